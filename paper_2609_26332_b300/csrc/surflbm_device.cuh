// Device-side building blocks of the coupled LBM step (sm_103a).
//
// Lattice: D2Q9, velocities ordered rest, +x, +y, -x, -y, (+,+), (-,+), (-,-), (+,-);
// weights 4/9, 1/9, 1/36; c_s^2 = 1/3 (Sec. 3).
//
// Number formats used on the hot path (B300 runs FP64 at a small fraction of the FP32
// rate, so no per-population FP64 arithmetic appears here):
//  * ff      - float-float pair (hi + lo, ~48-bit significand) for the conserved zeroth
//              moments m of the two scalar sets and for exactly-summed source terms;
//  * fixed   - 32-bit integers in units of 2^-S: every population value that crosses a
//              node boundary is converted once, deterministically, so the sum of what a
//              node receives minus what it sends telescopes exactly over the grid;
//  * Stor<T> - storage of the moving populations / history: FP32, FP16 or BF16.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <mutex>

namespace slbm {

// Host: runs setup() once per device (with that device current) and caches its result;
// kernel attributes such as the dynamic shared-memory opt-in are per device.  Thread-safe.
struct PerDeviceOnce {
    std::mutex mtx;
    bool done[128] = {};
    cudaError_t result[128] = {};
    template <class F>
    cudaError_t operator()(F&& setup) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lock(mtx);
        if (!done[dev]) {
            result[dev] = setup();
            done[dev] = true;
        }
        return result[dev];
    }
};

__host__ __device__ constexpr int CXk(int k) { return (k == 1 || k == 5 || k == 8) ? 1 : ((k == 3 || k == 6 || k == 7) ? -1 : 0); }
__host__ __device__ constexpr int CYk(int k) { return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0); }
__host__ __device__ constexpr float Wk(int k) { return k == 0 ? 4.0f / 9.0f : (k < 5 ? 1.0f / 9.0f : 1.0f / 36.0f); }
// exact-sum weights for the FP64 initialisation (the FP32 weights do not sum to 1)
__host__ __device__ constexpr double WkD(int k) { return k == 0 ? 4.0 / 9.0 : (k < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
__host__ __device__ constexpr int OPPk(int k) { return k == 0 ? 0 : (k < 5 ? ((k + 1) % 4) + 1 : ((k - 3) % 4) + 5); }
// direction with the y component reversed (specular reflection at a y-wall)
__host__ __device__ constexpr int MIRYk(int k) {
    return k == 2 ? 4 : k == 4 ? 2 : k == 5 ? 8 : k == 8 ? 5 : k == 6 ? 7 : k == 7 ? 6 : k;
}

// fixed-point exponents of the exchanged populations: phi set |v| < 2, psi set |v| < 1
constexpr int SFIX_PHI = 30;
constexpr int SFIX_PSI = 31;

// ----------------------------------------------------------------- float-float
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    float t = __fadd_rn(a.lo, b.lo);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, t));
}
__device__ __forceinline__ ff ff_scale_pow2(ff a, float p) { return {__fmul_rn(a.hi, p), __fmul_rn(a.lo, p)}; }
__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }

// exact float-float value of an int32 fixed-point number K * 2^-S
__device__ __forceinline__ ff fixed_to_ff(int K, float inv_scale) {
    int kh = K & ~0xFFF;            // <= 20 significant bits: exact in FP32
    int kl = K - kh;                // 0 .. 4095
    return quick_two_sum(__fmul_rn((float)kh, inv_scale), __fmul_rn((float)kl, inv_scale));
}

// ------------------------------------------------------------------- storage
template <class T> struct Stor;
template <> struct Stor<float> {
    static constexpr float kScale = 1.0f, kInv = 1.0f;
    static __device__ __forceinline__ float ld(const float* p, long long i) { return __ldg(p + i); }
    static __device__ __forceinline__ float lds(const float* p, int i) { return p[i]; }
    // the stored number without the storage scale (times kInv gives the value)
    static __device__ __forceinline__ float lds_raw(const float* p, int i) { return p[i]; }
    static __device__ __forceinline__ float rnd(float v) { return v; }
    static __device__ __forceinline__ void st(float* p, long long i, float v) { p[i] = v; }
};
template <> struct Stor<__half> {
    // deviations are O(1e-6 .. 1e-2): a 2^10 scale keeps them in FP16's normal range
    static constexpr float kScale = 1024.0f, kInv = 1.0f / 1024.0f;
    static __device__ __forceinline__ float ld(const __half* p, long long i) {
        return __half2float(__ldg(p + i)) * kInv;
    }
    static __device__ __forceinline__ float lds(const __half* p, int i) { return __half2float(p[i]) * kInv; }
    static __device__ __forceinline__ float lds_raw(const __half* p, int i) { return __half2float(p[i]); }
    static __device__ __forceinline__ float rnd(float v) { return __half2float(__float2half_rn(v * kScale)) * kInv; }
    static __device__ __forceinline__ void st(__half* p, long long i, float v) { p[i] = __float2half_rn(v * kScale); }
};
template <> struct Stor<__nv_bfloat16> {
    static constexpr float kScale = 1.0f, kInv = 1.0f;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, long long i) {
        return __bfloat162float(__ldg(p + i));
    }
    static __device__ __forceinline__ float lds(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }
    static __device__ __forceinline__ float lds_raw(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }
    static __device__ __forceinline__ float rnd(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, long long i, float v) { p[i] = __float2bfloat16_rn(v); }
};

// --------------------------------------------------------- natural-moment MRT
// Raw moments [1, cx, cy, cx^2, cx cy, cy^2, cx^2 cy, cx cy^2, cx^2 cy^2] of nine
// populations via two 1D transforms (values at c = -1, 0, +1 -> sum, first, second).
__device__ __forceinline__ void raw_moments(const float* f, float* m) {
    // rows by cy: (cx = -1, 0, +1)
    const float r0[3] = {f[3], f[0], f[1]};
    const float rp[3] = {f[6], f[2], f[5]};
    const float rm[3] = {f[7], f[4], f[8]};
    float A0[3], A1[3], A2[3];  // x-moments for rows cy = -1, 0, +1
    const float* rows[3] = {rm, r0, rp};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        A0[r] = rows[r][0] + rows[r][1] + rows[r][2];
        A1[r] = rows[r][2] - rows[r][0];
        A2[r] = rows[r][2] + rows[r][0];
    }
    // y-moments
    m[0] = A0[0] + A0[1] + A0[2];
    m[2] = A0[2] - A0[0];
    m[5] = A0[2] + A0[0];
    m[1] = A1[0] + A1[1] + A1[2];
    m[4] = A1[2] - A1[0];
    m[7] = A1[2] + A1[0];
    m[3] = A2[0] + A2[1] + A2[2];
    m[6] = A2[2] - A2[0];
    m[8] = A2[2] + A2[0];
}
// inverse of raw_moments
__device__ __forceinline__ void from_raw_moments(const float* m, float* f) {
    // invert in y: for each x-moment a, values at cy = -1, 0, +1
    float A[3][3];  // A[a][row], row 0: cy=-1, 1: cy=0, 2: cy=+1
    const float mm[3][3] = {{m[0], m[2], m[5]}, {m[1], m[4], m[7]}, {m[3], m[6], m[8]}};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        A[a][1] = mm[a][0] - mm[a][2];
        A[a][2] = 0.5f * (mm[a][2] + mm[a][1]);
        A[a][0] = 0.5f * (mm[a][2] - mm[a][1]);
    }
    // invert in x for each row
    float v[3][3];  // v[row][cx+1]
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        v[r][1] = A[0][r] - A[2][r];
        v[r][2] = 0.5f * (A[2][r] + A[1][r]);
        v[r][0] = 0.5f * (A[2][r] - A[1][r]);
    }
    f[0] = v[1][1]; f[1] = v[1][2]; f[3] = v[1][0];
    f[2] = v[2][1]; f[5] = v[2][2]; f[6] = v[2][0];
    f[4] = v[0][1]; f[8] = v[0][2]; f[7] = v[0][0];
}

// pop <- pop - M^-1 S M (pop - eq) + M^-1 (I - S/2) M src   (Sec. 3); s in moment order
__device__ __forceinline__ void mrt_collide(float* pop, const float* eq, const float* src, const float* s) {
    float d[9], dm[9], sm[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k] = pop[k] - eq[k];
    raw_moments(d, dm);
    raw_moments(src, sm);
#pragma unroll
    for (int a = 0; a < 9; ++a) dm[a] = s[a] * dm[a] - (1.0f - 0.5f * s[a]) * sm[a];
    float back[9];
    from_raw_moments(dm, back);
#pragma unroll
    for (int k = 0; k < 9; ++k) pop[k] -= back[k];
}

}  // namespace slbm
