// Library-internal definition of a domain, shared by the single-domain API and the
// batch (whose instances are domains stepped by the batch kernel).
#pragma once
#include <string>
#include "surflbm.h"
#include "surflbm_step.cuh"

struct slbm_domain {
    slbm_params p;
    cudaStream_t stream = nullptr;
    slbm::Phys phys;
    double beta, kappa, lambda_s, W, kT, phi_b, M_phi, M_0;
    double wall_theta[2] = {90.0, 90.0}, wall_bsg[2] = {0, 0}, wall_bsl[2] = {0, 0}, wall_u[2] = {0, 0};
    long long N = 0;
    dim3 grid;
    long long total = 0;   // strips * ny, the rows the CTAs share out
    int cur = 0;
    long long n = 0;
    bool initialised = false;
    void* f[2] = {nullptr, nullptr};
    void* gd[2] = {nullptr, nullptr};
    void* hd[2] = {nullptr, nullptr};
    float2* gm[2] = {nullptr, nullptr};
    float2* hm[2] = {nullptr, nullptr};
    float* php[2] = {nullptr, nullptr};
    void* hist = nullptr;
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    slbm::Rec* recs = nullptr;  // [0], [1]: ring by step parity; [2]: diagnostic level; [3]: zeros
    double* fields = nullptr;   // 5 N doubles, allocated on first read
    size_t bytes = 0;
    std::string err = "no error";
};
