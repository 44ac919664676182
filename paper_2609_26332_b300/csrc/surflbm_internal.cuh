// Library-internal definition of a domain, shared by the single-domain API and the
// batch (whose instances are domains stepped by the batch kernel).
#pragma once
#include <string>
#include <vector>
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
    int exact_blocks = 0;   // grid of the exact-multiplier pass (EXACT mode only)
    long long total = 0;   // strips * ny, the rows the CTAs share out
    int band_h = 0;        // > 0: band-major split into pieces of band_h rows
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
    unsigned int* counter = nullptr;   // [0]: CTAs done in the current launch, [1]: error bits (ERR_*)
    slbm::Rec* recs = nullptr;  // [0], [1]: ring by step parity; [2]: diagnostic level; [3]: zeros
    double* fields = nullptr;   // 5 N doubles, allocated on first read
    size_t bytes = 0;
    // caller-owned device workspace (slbm_create_domain_ext): every buffer is carved from
    // it in the order of slbm_workspace_bytes and nothing is allocated or freed
    bool tma = false;                 // the step stages through TMA boxes (maps of both sides)
    bool mms = false;                 // manufactured-solution test (slbm_set_mms)
    double mms_u0x = 0.0;             // its uniform lattice velocity (initial state)
    slbm::TmaMaps maps[2];
    bool ext = false;
    unsigned char* ws = nullptr;
    size_t ws_size = 0, ws_off = 0;
    std::string err = "no error";
};

// cudaMalloc counted in the process-wide total that slbm_device_allocations reports; every
// device allocation of the library goes through it.
cudaError_t slbm_device_malloc(void** ptr, size_t bytes);

// Parameter checks (empty string: valid), derivation of the model constants and Phys, and
// one wall's Phys entries (surflbm_api.cu); also used by the three-dimensional domain.
std::string slbm_validate_params(const slbm_params* p);
void slbm_derive_phys(slbm_domain* d);
void slbm_wall_phys(slbm_domain* d, int w);

// The diagnostic pass of the current level into d->fields (phi, psi, ux, uy, p planes),
// reduced with the domain's own partials; queued on the domain's stream.
slbm_status diag_into_fields(slbm_domain* d);

// Exact discrete multiplier of the step just queued (surflbm_exact.cu): reduces the
// coefficients of H(A + lambda B) = H0 and overwrites lambda in the record of that step.
cudaError_t launch_exact_multiplier(slbm_domain* d);
int exact_multiplier_blocks(int precision, long long N);

// A batch of domains stepped by the tile-queue kernel (surflbm_batch.cu).
struct slbm_batch {
    int count = 0;
    int precision = 0;
    bool var = false;                 // some instance has variable density / viscosity
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<slbm_domain*> dom;
    std::vector<char> active;
    std::vector<long long> G0;        // batch step at each instance's time level 0
    long long G = 0;                  // host mirror of the device step counter
    int band_rows = 64, ctas_per_sm = 2, graph_steps = 32;
    int strip_width = 64;             // columns per strip: 64 (256 threads) or 32 (128 threads)
    // device tables
    slbm::InstDesc* d_inst = nullptr;
    slbm::Piece* d_pieces = nullptr;
    double* d_partials = nullptr;     // per instance: max pieces * NPART
    unsigned int* d_counters = nullptr;  // per instance
    unsigned int* d_queue = nullptr;  // [0]: queue, [1]: done
    long long* d_G = nullptr;
    std::vector<size_t> part_off;     // offset of each instance's partial slots (doubles)
    std::vector<int> max_pieces;
    int npieces = 0, nctas = 1;
    bool tables_valid = false;
    cudaGraphExec_t graph = nullptr;
    int graph_len = 0;
    // residual
    float* d_snap_base = nullptr;
    std::vector<size_t> snap_off;
    bool have_snap = false;
    char* d_res = nullptr;            // residual-check scratch (kept between checks)
    size_t res_bytes = 0;
    std::string err = "no error";
    size_t bytes = 0;
};
