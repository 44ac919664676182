// Learned warm start: the conv encoder-decoder (forward, backward, Adam) built on the
// tcgen05 convolutions of ws_conv.cuh, the training-target extraction from relaxed
// lattice Boltzmann states, and the warm-start projection onto the cold start's
// conserved totals (sum psi, Eq. AC_psi's constraint; H = sum h_phi, Eq. conservation).
#include "surflbm_internal.cuh"
#include "surflbm_ws.h"
#include "ws_conv.cuh"
#include "ws_conv_tma.cuh"

#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace ws;
typedef __nv_bfloat16 bf16;

namespace {

__device__ unsigned int g_prim_err = 0;   // timeout flag of the conv primitive entry points

std::string g_ws_create_error = "no error";

// ================================================================== small kernels
constexpr int EW = 256;   // threads of the elementwise kernels

inline unsigned ew_grid(long long n) {
    long long g = (n + EW - 1) / EW;
    return (unsigned)(g < 1 ? 1 : (g > 148LL * 64 ? 148LL * 64 : g));
}

__global__ void flip_weights_kernel(const bf16* __restrict__ w, bf16* __restrict__ wt, int Cin, int Cout) {
    const long long n = (long long)Cout * 9 * Cin;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(e / (9 * Cin));
        const int r = (int)(e - (long long)co * 9 * Cin);
        const int tap = r / Cin, ci = r - tap * Cin;
        wt[((long long)ci * 9 + (8 - tap)) * Cout + co] = w[e];
    }
}

// FP32 master weights of one conv -> BF16 [Cout][9][Cin] and flipped [Cin][9][Cout]
__global__ void convert_kernel(const float* __restrict__ p, bf16* __restrict__ w, bf16* __restrict__ wt, int Cin,
                               int Cout) {
    const long long n = (long long)Cout * 9 * Cin;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(e / (9 * Cin));
        const int r = (int)(e - (long long)co * 9 * Cin);
        const int tap = r / Cin, ci = r - tap * Cin;
        const bf16 v = __float2bfloat16_rn(p[e]);
        w[e] = v;
        wt[((long long)ci * 9 + (8 - tap)) * Cout + co] = v;
    }
}

constexpr int CIN0 = 16;   // input channels: 5 parameters + 11 coordinate features

// network input [B][H][W][16] from parameter rows cond[idx[b]]
__global__ void input_kernel(const float* __restrict__ cond, const int* __restrict__ idx, int B, int H, int W,
                             bf16* __restrict__ x0) {
    const long long n = (long long)B * H * W;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(p % W);
        const long long t = p / W;
        const int y = (int)(t % H);
        const int b = (int)(t / H);
        const int s = idx ? idx[b] : b;
        const float* c = cond + (long long)s * 5;
        const float half = 0.5f * (float)H;
        const float X = ((float)x + 0.5f - 0.5f * (float)W) / half, Y = ((float)y + 0.5f) / half;
        float v[CIN0];
        v[0] = (c[0] - 90.0f) / 60.0f;
        v[1] = 2.0f * c[1] - 1.0f;
        v[2] = 2.0f * c[2] - 1.0f;
        v[3] = (c[3] - 0.0275f) / 0.0225f;
        v[4] = (c[4] - 0.07f) / 0.025f;
        v[5] = X;
        v[6] = Y;
        v[7] = 1.0f;
        v[8] = X * X;
        v[9] = Y * Y;
        v[10] = X * Y;
        v[11] = fabsf(X);
        v[12] = sinpif(0.5f * X);
        v[13] = cospif(0.5f * X);
        v[14] = sinpif(0.5f * Y);
        v[15] = cospif(0.5f * Y);
        uint4 o[2];
        __nv_bfloat162* ob = (__nv_bfloat162*)o;
#pragma unroll
        for (int i = 0; i < 8; ++i) ob[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        uint4* dst = (uint4*)(x0 + p * CIN0);
        dst[0] = o[0];
        dst[1] = o[1];
    }
}

__device__ __forceinline__ void unpack8(const uint4& u, float (&f)[8]) {
    const __nv_bfloat162* h = (const __nv_bfloat162*)&u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 u;
    __nv_bfloat162* h = (__nv_bfloat162*)&u;
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return u;
}

// 2 x 2 average pool: in [B][H][W][C] -> out [B][H/2][W/2][C]; one thread per 8 channels
__global__ void pool_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2, C8 = C / 8;
    const long long n = (long long)B * Ho * Wo * C8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c8 = (int)(e % C8);
        const long long q = e / C8;
        const int xo = (int)(q % Wo);
        const long long t = q / Wo;
        const int yo = (int)(t % Ho);
        const long long b = t / Ho;
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                float f[8];
                unpack8(*(const uint4*)(in + (((b * H + 2 * yo + dy) * W + 2 * xo + dx) * C + c8 * 8)), f);
#pragma unroll
                for (int i = 0; i < 8; ++i) s[i] += f[i];
            }
#pragma unroll
        for (int i = 0; i < 8; ++i) s[i] *= 0.25f;
        *(uint4*)(out + q * C + c8 * 8) = pack8(s);
    }
}

// out [B][H][W][Cu + Cs] = (nearest-upsampled up [B][H/2][W/2][Cu], skip [B][H][W][Cs])
__global__ void upcat_kernel(const bf16* __restrict__ up, const bf16* __restrict__ skip, bf16* __restrict__ out,
                             int B, int H, int W, int Cu, int Cs) {
    const int Ct = Cu + Cs, C8 = Ct / 8;
    const long long n = (long long)B * H * W * C8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C8) * 8;
        const long long p = e / C8;
        const int x = (int)(p % W);
        const long long t = p / W;
        const int y = (int)(t % H);
        const long long b = t / H;
        uint4 v;
        if (c < Cu) v = *(const uint4*)(up + (((b * (H / 2) + y / 2) * (W / 2) + x / 2) * Cu + c));
        else v = *(const uint4*)(skip + p * Cs + (c - Cu));
        *(uint4*)(out + p * Ct + c) = v;
    }
}

// gradient of the upsampled part: gout [B][H/2][W/2][Cu] = sum over the 2 x 2 children of
// gcat[..][0 .. Cu)
__global__ void unpool_back_kernel(const bf16* __restrict__ gcat, int Ct, bf16* __restrict__ gout, int B, int Hc,
                                   int Wc, int Cu) {
    const int C8 = Cu / 8, H = 2 * Hc, W = 2 * Wc;
    const long long n = (long long)B * Hc * Wc * C8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C8) * 8;
        const long long q = e / C8;
        const int xc = (int)(q % Wc);
        const long long t = q / Wc;
        const int yc = (int)(t % Hc);
        const long long b = t / Hc;
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                float f[8];
                unpack8(*(const uint4*)(gcat + (((b * H + 2 * yc + dy) * W + 2 * xc + dx) * Ct + c)), f);
#pragma unroll
                for (int i = 0; i < 8; ++i) s[i] += f[i];
            }
        *(uint4*)(gout + q * Cu + c) = pack8(s);
    }
}

// gradient at a skip tensor e [B][H][W][C] (a ReLU output feeding both a pool and a
// concat): gz = [e > 0] * gp[pooled parent] / 4 + gcat[.., off .. off + C)
__global__ void pool_back_kernel(const bf16* __restrict__ e_act, const bf16* __restrict__ gp,
                                 const bf16* __restrict__ gcat, int Ct, int off, bf16* __restrict__ gz, int B, int H,
                                 int W, int C) {
    const int C8 = C / 8;
    const long long n = (long long)B * H * W * C8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C8) * 8;
        const long long p = e / C8;
        const int x = (int)(p % W);
        const long long t = p / W;
        const int y = (int)(t % H);
        const long long b = t / H;
        float a[8], g[8], k[8];
        unpack8(*(const uint4*)(e_act + p * C + c), a);
        unpack8(*(const uint4*)(gp + (((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c)), g);
        unpack8(*(const uint4*)(gcat + p * Ct + off + c), k);
        float o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = (a[i] > 0.0f ? 0.25f * g[i] : 0.0f) + k[i];
        *(uint4*)(gz + p * C + c) = pack8(o);
    }
}

// gb[c] += sum_p dz[p][c]
__global__ void bias_grad_kernel(const bf16* __restrict__ dz, long long P, int C, float* __restrict__ gb) {
    __shared__ float s[256];
    for (int i = threadIdx.x; i < C; i += blockDim.x) s[i] = 0.0f;
    __syncthreads();
    const int per = blockDim.x / C > 0 ? blockDim.x / C : 1;   // pixels in flight per block
    const int c = threadIdx.x % C, lane_p = threadIdx.x / C;
    if (lane_p < per && threadIdx.x < per * C) {
        float acc = 0.0f;
        for (long long p = (long long)blockIdx.x * per + lane_p; p < P; p += (long long)gridDim.x * per)
            acc += __bfloat162float(dz[p * C + c]);
        atomicAdd(&s[c], acc);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C; i += blockDim.x) atomicAdd(gb + i, s[i]);
}

constexpr int HEAD_C = 32;

// head (1 x 1 conv 32 -> 2), loss and its gradient; targets [rows][2][H][W]
__global__ void head_train_kernel(const bf16* __restrict__ d0, const float* __restrict__ Wh, const float* __restrict__ bh,
                                  const float* __restrict__ targets, const int* __restrict__ idx, int B, int H, int W,
                                  bf16* __restrict__ gz, float* __restrict__ gWh, float* __restrict__ gbh,
                                  double* __restrict__ loss) {
    __shared__ float sW[2 * HEAD_C + 2];
    __shared__ float sacc[2 * HEAD_C + 2];
    __shared__ double sloss;
    for (int i = threadIdx.x; i < 2 * HEAD_C; i += blockDim.x) {
        sW[i] = Wh[i];
        sacc[i] = 0.0f;
    }
    if (threadIdx.x < 2) {
        sW[2 * HEAD_C + threadIdx.x] = bh[threadIdx.x];
        sacc[2 * HEAD_C + threadIdx.x] = 0.0f;
    }
    if (threadIdx.x == 0) sloss = 0.0;
    __syncthreads();
    const long long HW = (long long)H * W, n = (long long)B * HW;
    const float scale = 2.0f / (float)n;
    float acc[2 * HEAD_C + 2];
#pragma unroll
    for (int i = 0; i < 2 * HEAD_C + 2; ++i) acc[i] = 0.0f;
    double lsum = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        float h[HEAD_C];
#pragma unroll
        for (int q = 0; q < HEAD_C / 8; ++q) {
            float f[8];
            unpack8(*(const uint4*)(d0 + p * HEAD_C + 8 * q), f);
#pragma unroll
            for (int i = 0; i < 8; ++i) h[8 * q + i] = f[i];
        }
        float o0 = sW[2 * HEAD_C], o1 = sW[2 * HEAD_C + 1];
#pragma unroll
        for (int i = 0; i < HEAD_C; ++i) {
            o0 += sW[i] * h[i];
            o1 += sW[HEAD_C + i] * h[i];
        }
        const long long b = p / HW, q = p - b * HW;
        const long long s = idx ? idx[b] : b;
        const float r0 = o0 - targets[(2 * s) * HW + q], r1 = o1 - targets[(2 * s + 1) * HW + q];
        lsum += (double)r0 * r0 + (double)r1 * r1;
        const float g0 = scale * r0, g1 = scale * r1;
#pragma unroll
        for (int i = 0; i < HEAD_C; ++i) {
            acc[i] += g0 * h[i];
            acc[HEAD_C + i] += g1 * h[i];
        }
        acc[2 * HEAD_C] += g0;
        acc[2 * HEAD_C + 1] += g1;
#pragma unroll
        for (int q8 = 0; q8 < HEAD_C / 8; ++q8) {
            float f[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = 8 * q8 + i;
                f[i] = h[k] > 0.0f ? g0 * sW[k] + g1 * sW[HEAD_C + k] : 0.0f;
            }
            *(uint4*)(gz + p * HEAD_C + 8 * q8) = pack8(f);
        }
    }
#pragma unroll
    for (int i = 0; i < 2 * HEAD_C + 2; ++i) {
        float v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sacc[i], v);
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sloss, lsum);
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * HEAD_C; i += blockDim.x) atomicAdd(gWh + i, sacc[i]);
    if (threadIdx.x < 2) atomicAdd(gbh + threadIdx.x, sacc[2 * HEAD_C + threadIdx.x]);
    if (threadIdx.x == 0) atomicAdd(loss, sloss / (double)n);
}

// inference head: out [B][2][H][W] FP32
__global__ void head_fwd_kernel(const bf16* __restrict__ d0, const float* __restrict__ Wh, const float* __restrict__ bh,
                                int B, int H, int W, float* __restrict__ out) {
    const long long HW = (long long)H * W, n = (long long)B * HW;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        float o0 = bh[0], o1 = bh[1];
#pragma unroll
        for (int q = 0; q < HEAD_C / 8; ++q) {
            float f[8];
            unpack8(*(const uint4*)(d0 + p * HEAD_C + 8 * q), f);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                o0 += Wh[8 * q + i] * f[i];
                o1 += Wh[HEAD_C + 8 * q + i] * f[i];
            }
        }
        const long long b = p / HW, q = p - b * HW;
        out[(2 * b) * HW + q] = o0;
        out[(2 * b + 1) * HW + q] = o1;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// training target of one relaxed instance: phi and ln(psi / psi0)
__global__ void targets_kernel(const double* __restrict__ phi, const double* __restrict__ psi, long long N,
                               double psi0, int psi_on, float* __restrict__ t) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        t[i] = (float)phi[i];
        t[N + i] = psi_on ? (float)log(fmax(psi[i], 1e-12) / psi0) : 0.0f;
    }
}

// ---------------------------------------------------------------- warm-start projection
struct ProjArgs {
    const float* pred;      // [2][N]: phi, ln(psi / psi0)
    double* phi;            // out [N]
    double* psi;            // out [N]
    long long N;
    double phi_b, psi0, psi_target, q_target;
    int linear, psi_on;
    int* ok;                // out
};

__device__ double block_sum_d(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

__device__ __forceinline__ double q_of(double phi, double phi_b) {
    const double u = phi / phi_b;
    return 1.5 * u - 0.5 * u * u * u;
}

// one CTA per instance: scale psi to the target total; shift phi (clamped to the bulk
// values) by the constant that gives the target sum q(phi) (nonlinear; bisection on a
// monotone function) or sum phi (linear; closed form)
__global__ void project_kernel(const ProjArgs* __restrict__ args) {
    __shared__ double sh[32];
    const ProjArgs a = args[blockIdx.x];
    const long long N = a.N;
    bool finite = true;
    double s = 0.0;
    if (a.psi_on) {
        for (long long i = threadIdx.x; i < N; i += blockDim.x) {
            const double v = fmin(fmax(a.psi0 * exp((double)a.pred[N + i]), 1e-8), 0.9);
            finite = finite && isfinite(v);
            s += v;
        }
        s = block_sum_d(s, sh);
    }
    const double scale = (a.psi_on && s > 0.0) ? a.psi_target / s : 0.0;
    double c = 0.0, resid = 0.0;
    if (a.linear) {
        double t = 0.0;
        for (long long i = threadIdx.x; i < N; i += blockDim.x) t += (double)a.pred[i];
        t = block_sum_d(t, sh);
        c = (a.q_target - t) / (double)N;
    } else {
        double lo = -2.0 * a.phi_b, hi = 2.0 * a.phi_b;
        for (int it = 0; it < 64; ++it) {
            const double mid = 0.5 * (lo + hi);
            double t = 0.0;
            for (long long i = threadIdx.x; i < N; i += blockDim.x)
                t += q_of(fmin(fmax((double)a.pred[i] + mid, -a.phi_b), a.phi_b), a.phi_b);
            t = block_sum_d(t, sh) - a.q_target;
            if (t < 0.0) lo = mid;
            else hi = mid;
            resid = t;
        }
        c = 0.5 * (lo + hi);
    }
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        double ph = (double)a.pred[i] + c;
        if (!a.linear) ph = fmin(fmax(ph, -a.phi_b), a.phi_b);
        finite = finite && isfinite(ph);
        a.phi[i] = ph;
        if (a.psi_on) a.psi[i] = scale * fmin(fmax(a.psi0 * exp((double)a.pred[N + i]), 1e-8), 0.9);
    }
    const double bad = block_sum_d(finite ? 0.0 : 1.0, sh);
    if (threadIdx.x == 0)
        *a.ok = (bad == 0.0 && (!a.psi_on || s > 0.0) && fabs(resid) <= 1e-6 * (double)N + 1e-6) ? 1 : 0;
}

// ================================================================== conv launchers
// ring depth by width: the narrowest tiles (32 channels) take 3 stages, so three CTAs
// fit on an SM (measured: faster at 32 channels, slower at 64)
inline int mk_stages(int N) { return N <= 32 ? 3 : 4; }
inline int wg_stages(int C) { return C <= 32 ? 3 : 4; }

cudaError_t conv_attrs() {
    static slbm::PerDeviceOnce once;
    return once([] {
        const int mk = (int)(CONV_STAGES * mk_stage_bytes(256)), wg = (int)(CONV_STAGES * wg_stage_bytes(256));
        cudaError_t e = cudaFuncSetAttribute(conv_mk_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mk);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(conv_mk_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mk);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(conv_wg_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, wg);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(conv_wg_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, wg);
        return e;
    });
}

// ---- tensor-memory-accelerator convolution (ws_conv_tma.cuh)
PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
    static std::once_flag flag;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(flag, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

// channels per K block of the TMA convolution: 64, 32 or 16 (0: not supported)
int tma_kc(int C) { return C % 64 == 0 ? 64 : (C % 32 == 0 ? 32 : (C % 16 == 0 ? 16 : 0)); }

// pixel tile Wt x Ht x Bt = 128 that tiles the B x H x W grid exactly, or false
bool tma_tile(int B, int H, int W, int& Wt, int& Ht, int& Bt) {
    Wt = W < 128 ? W : 128;
    if (W % Wt || 128 % Wt) return false;
    const int rest = 128 / Wt;
    Ht = H < rest ? H : rest;
    if (H % Ht || rest % Ht) return false;
    Bt = rest / Ht;
    return B % Bt == 0;
}

constexpr int TC_SMEM_BUDGET = 110 * 1024;   // two CTAs per SM

cudaError_t tconv_attrs() {
    static slbm::PerDeviceOnce once;
    return once([] {
        // the ring (at most TC_SMEM_BUDGET bytes: 2 stages of the widest tiles take 96 KB) and
        // 1 KB of alignment slack
        cudaError_t e = cudaFuncSetAttribute(conv_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BUDGET + 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_wg_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BUDGET + 1024);
        return e;
    });
}

// the TMA convolution when the shapes allow it (true), else false (nothing launched)
bool launch_tconv(const bf16* x, const bf16* w, const float* bias, const bf16* mask, bf16* y, int B, int H, int W,
                  int C, int N, int relu, unsigned int* err, cudaStream_t st, cudaError_t* res) {
    int Wt, Ht, Bt;
    const int KC = tma_kc(C);
    auto enc = tma_encode_fn();
    if (!enc || KC == 0 || N % 16 || N < 16 || N > 256 || !tma_tile(B, H, W, Wt, Ht, Bt)) return false;
    const CUtensorMapSwizzle sw = KC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                           : (KC == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    CUtensorMap mx, mw;
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const cuuint64_t xd[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t xs[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t xb[4] = {(cuuint32_t)KC, (cuuint32_t)Wt, (cuuint32_t)Ht, (cuuint32_t)Bt};
    const cuuint64_t wd[2] = {(cuuint64_t)9 * C, (cuuint64_t)N};
    const cuuint64_t ws_[1] = {(cuuint64_t)9 * C * 2};
    const cuuint32_t wb[2] = {(cuuint32_t)KC, (cuuint32_t)N};
    if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x), xd, xs, xb, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(w), wd, ws_, wb, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    cudaError_t e = tconv_attrs();
    if (e != cudaSuccess) {
        *res = e;
        return true;
    }
    TConvArgs a;
    a.bias = bias; a.mask = mask; a.y = y;
    a.B = B; a.H = H; a.W = W; a.C = C; a.N = N; a.relu = relu;
    a.Wt = Wt; a.Ht = Ht; a.Bt = Bt; a.KC = KC;
    a.a_bytes = 128u * (uint32_t)KC * 2u;
    a.b_bytes = (((uint32_t)N * (uint32_t)KC * 2u) + 1023u) & ~1023u;
    const uint32_t sb = a.a_bytes + a.b_bytes;
    int stages = (int)(TC_SMEM_BUDGET / sb);
    stages = stages > TC_MAX_STAGES ? TC_MAX_STAGES : stages;
    if (stages < 2) return false;
    a.stages = stages;
    a.err = err;
    const size_t smem = (size_t)stages * sb + 1024;
    // persistent grid: the CTAs that fit at once (two accumulators of N columns each in the
    // 512 columns of tensor memory, and the shared-memory ring), at most one per tile
    int dev = 0, sms = 148, smem_sm = 233472;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // per CTA: the dynamic ring, ~1 KB of static barriers and the 1 KB the runtime reserves
    int per = (int)((size_t)smem_sm / (smem + 2048));
    const int by_tmem = (int)(512u / (2u * tmem_cols_for(N)));
    if (per > by_tmem) per = by_tmem;
    if (per < 1) per = 1;
    const long long tiles = (long long)B * H * W / 128;
    const unsigned grid = (unsigned)(tiles < (long long)per * sms ? tiles : (long long)per * sms);
    conv_tma_kernel<<<grid, TC_THREADS, smem, st>>>(mx, mw, a);
    *res = cudaGetLastError();
    return true;
}

cudaError_t launch_mk(const bf16* x, const bf16* w, const float* bias, const bf16* mask, bf16* y, int B, int H, int W,
                      int C, int N, int relu, unsigned int* err, cudaStream_t st) {
    cudaError_t te = cudaSuccess;
    if (launch_tconv(x, w, bias, mask, y, B, H, W, C, N, relu, err, st, &te)) return te;
    cudaError_t e = conv_attrs();
    if (e != cudaSuccess) return e;
    MKArgs a{x, w, bias, mask, y, B, H, W, C, N, relu, err};
    const long long P = (long long)B * H * W;
    const unsigned grid = (unsigned)((P + 127) / 128);
    if (mk_stages(N) == 3) conv_mk_kernel<3><<<grid, CONV_THREADS, 3 * mk_stage_bytes(N), st>>>(a);
    else conv_mk_kernel<4><<<grid, CONV_THREADS, 4 * mk_stage_bytes(N), st>>>(a);
    return cudaGetLastError();
}

// the TMA weight gradient when the shapes allow it (true), else false (nothing launched);
// C = Cin, N = Cout
bool launch_twg(const bf16* x, const bf16* dz, float* dw, int B, int H, int W, int C, int N, unsigned int* err,
                cudaStream_t st, cudaError_t* res) {
    auto enc = tma_encode_fn();
    const int Wb = W < 64 ? W : 64;
    if (!enc || W % Wb || 64 % Wb || C % 16 || N % 16 || C > 256 || N > 128) return false;
    // with both channel counts below 64 every box row is at most 64 bytes and the copy engine's
    // per-row rate bounds the kernel below the cp.async one (measured: 627 vs 436 us for
    // 32 -> 32 at 1 M pixels)
    if (C < 64 && N < 64) return false;
    const int Hb = 64 / Wb;
    if (H % Hb) return false;
    const int swap = (C <= 128 && C > N) ? 1 : 0;
    const int Mv = swap ? C : N, Nn = swap ? N : C;
    const int awA = tma_kc(Mv), awB = tma_kc(Nn);
    if (awA == 0 || awB == 0) return false;
    // 4-D views [B][H][W][C], boxes of AW channels x Wb x Hb pixels, swizzled by the atom width
    auto sw_of = [](int aw) {
        return aw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (aw == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    };
    auto make = [&](CUtensorMap* m, const bf16* t, int ch, int aw) {
        const cuuint64_t d[4] = {(cuuint64_t)ch, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t str[3] = {(cuuint64_t)ch * 2, (cuuint64_t)W * ch * 2, (cuuint64_t)H * W * ch * 2};
        const cuuint32_t box[4] = {(cuuint32_t)aw, (cuuint32_t)Wb, (cuuint32_t)Hb, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(t), d, str, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw_of(aw), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap mdz, mx;
    if (!make(&mdz, dz, N, swap ? awB : awA) || !make(&mx, x, C, swap ? awA : awB)) return false;
    cudaError_t e = tconv_attrs();
    if (e != cudaSuccess) {
        *res = e;
        return true;
    }
    TWGArgs a;
    a.dw = dw; a.B = B; a.H = H; a.W = W; a.Cin = C; a.Cout = N; a.Wb = Wb; a.Hb = Hb; a.swap = swap;
    a.awA = awA; a.awB = awB;
    a.a_bytes = 16u * 1024u;
    a.b_bytes = (uint32_t)Nn * 128u;
    const uint32_t sb = a.a_bytes + ((a.b_bytes + 1023u) & ~1023u);
    a.b_bytes = sb - a.a_bytes;
    int stages = (int)(TC_SMEM_BUDGET / sb);
    stages = stages > TC_MAX_STAGES ? TC_MAX_STAGES : stages;
    if (stages < 2) return false;
    a.stages = stages;
    a.err = err;
    a.nkb_total = (int)((long long)B * H * W / 64);
    // about two CTAs per SM over the 9 taps
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long splits = (2LL * sms + 8) / 9;
    if (splits > a.nkb_total) splits = a.nkb_total;
    a.kb_per_cta = (int)((a.nkb_total + splits - 1) / splits);
    const dim3 grid((unsigned)((a.nkb_total + a.kb_per_cta - 1) / a.kb_per_cta), 9);
    conv_wg_tma_kernel<<<grid, TC_THREADS, (size_t)stages * sb + 1024, st>>>(mdz, mx, a);
    *res = cudaGetLastError();
    return true;
}

cudaError_t launch_wg(const bf16* x, const bf16* dz, float* dw, int B, int H, int W, int C, int N, unsigned int* err,
                      cudaStream_t st) {
    cudaError_t te = cudaSuccess;
    if (launch_twg(x, dz, dw, B, H, W, C, N, err, st, &te)) return te;
    cudaError_t e = conv_attrs();
    if (e != cudaSuccess) return e;
    const long long P = (long long)B * H * W;
    const long long splits = 33;   // 33 x 9 taps ~ 2 CTAs per SM
    long long ppc = (P + splits - 1) / splits;
    ppc = ((ppc + 63) / 64) * 64;
    if (ppc < 256) ppc = 256;
    WGArgs a{x, dz, dw, B, H, W, C, N, ppc, err};
    dim3 grid((unsigned)((P + ppc - 1) / ppc), 9);
    if (wg_stages(C) == 3) conv_wg_kernel<3><<<grid, CONV_THREADS, 3 * wg_stage_bytes(C), st>>>(a);
    else conv_wg_kernel<4><<<grid, CONV_THREADS, 4 * wg_stage_bytes(C), st>>>(a);
    return cudaGetLastError();
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

unsigned int* prim_err() {
    void* p = nullptr;
    return cudaGetSymbolAddress(&p, g_prim_err) == cudaSuccess ? (unsigned int*)p : nullptr;
}

// ================================================================== network
struct ConvSpec {
    int level, cin, cout;
};
constexpr int NCONV = 14;
constexpr ConvSpec SPECS[NCONV] = {{0, CIN0, 32}, {0, 32, 32},   {1, 32, 64},   {1, 64, 64},   {2, 64, 128},
                                   {2, 128, 128}, {3, 128, 128}, {3, 128, 128}, {2, 256, 128}, {2, 128, 128},
                                   {1, 192, 64},  {1, 64, 64},   {0, 96, 32},   {0, 32, 32}};

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct slbm_ws {
    int H = 0, W = 0, maxB = 0;
    cudaStream_t stream = nullptr;
    long long nparam = 0;
    long long w_off[NCONV], b_off[NCONV], hw_off = 0, hb_off = 0;
    float* params = nullptr;   // FP32 master
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long adam_t = 0;
    bf16* wb[NCONV];           // [Cout][9][Cin]
    bf16* wt[NCONV];           // [Cin][9][Cout] flipped
    // activations (BF16 NHWC, max batch)
    bf16* x0 = nullptr;
    bf16* y[NCONV];
    bf16 *p0 = nullptr, *p1 = nullptr, *p2 = nullptr, *c2 = nullptr, *c1 = nullptr, *c0 = nullptr;
    bf16* gz[NCONV];
    bf16 *gp0 = nullptr, *gp1 = nullptr, *gp2 = nullptr, *gc2 = nullptr, *gc1 = nullptr, *gc0 = nullptr;
    const bf16* in[NCONV];
    double* d_loss = nullptr;
    unsigned int* d_err = nullptr;
    float* d_cond = nullptr;   // warm-start scratch: parameter rows
    float* d_pred = nullptr;   // [maxB][2][H][W]
    ProjArgs* d_proj = nullptr;
    int* d_ok = nullptr;
    size_t bytes = 0;
    std::vector<void*> allocs;
    std::string err = "no error";
};

namespace {

slbm_status wfail(slbm_ws* n, slbm_status s, const std::string& m) {
    if (n) n->err = m;
    else g_ws_create_error = m;
    return s;
}
slbm_status wcuda(slbm_ws* n, cudaError_t e, const char* what) {
    return wfail(n, SLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t walloc(slbm_ws* n, T** p, size_t count) {
    void* q = nullptr;
    const size_t b = count * sizeof(T);
    cudaError_t e = slbm_device_malloc((void**)&q, b ? b : 16);
    if (e == cudaSuccess) {
        n->allocs.push_back(q);
        n->bytes += b;
        *p = (T*)q;
    }
    return e;
}

long long pix(const slbm_ws* n, int level, int B) { return (long long)B * (n->H >> level) * (n->W >> level); }

cudaError_t refresh_weights(slbm_ws* n) {
    for (int i = 0; i < NCONV; ++i) {
        const long long cnt = (long long)SPECS[i].cout * 9 * SPECS[i].cin;
        convert_kernel<<<ew_grid(cnt), EW, 0, n->stream>>>(n->params + n->w_off[i], n->wb[i], n->wt[i], SPECS[i].cin,
                                                            SPECS[i].cout);
    }
    return cudaGetLastError();
}

// forward pass for B samples (rows idx of cond)
cudaError_t forward(slbm_ws* n, const float* cond, const int* idx, int B) {
    cudaStream_t st = n->stream;
    const int H = n->H, W = n->W;
    input_kernel<<<ew_grid(pix(n, 0, B)), EW, 0, st>>>(cond, idx, B, H, W, n->x0);
    cudaError_t e = cudaGetLastError();
    auto conv = [&](int i) {
        if (e != cudaSuccess) return;
        const int l = SPECS[i].level;
        e = launch_mk(n->in[i], n->wb[i], n->params + n->b_off[i], nullptr, n->y[i], B, H >> l, W >> l, SPECS[i].cin,
                      SPECS[i].cout, 1, n->d_err, st);
    };
    auto pool = [&](const bf16* a, bf16* o, int l, int C) {
        if (e != cudaSuccess) return;
        pool_kernel<<<ew_grid(pix(n, l + 1, B) * C / 8), EW, 0, st>>>(a, o, B, H >> l, W >> l, C);
        e = cudaGetLastError();
    };
    auto upcat = [&](const bf16* up, const bf16* skip, bf16* o, int l, int Cu, int Cs) {
        if (e != cudaSuccess) return;
        upcat_kernel<<<ew_grid(pix(n, l, B) * (Cu + Cs) / 8), EW, 0, st>>>(up, skip, o, B, H >> l, W >> l, Cu, Cs);
        e = cudaGetLastError();
    };
    conv(0); conv(1); pool(n->y[1], n->p0, 0, 32);
    conv(2); conv(3); pool(n->y[3], n->p1, 1, 64);
    conv(4); conv(5); pool(n->y[5], n->p2, 2, 128);
    conv(6); conv(7); upcat(n->y[7], n->y[5], n->c2, 2, 128, 128);
    conv(8); conv(9); upcat(n->y[9], n->y[3], n->c1, 1, 128, 64);
    conv(10); conv(11); upcat(n->y[11], n->y[1], n->c0, 0, 64, 32);
    conv(12); conv(13);
    return e;
}

// backward pass after head_train_kernel wrote gz[13]; gradients accumulate into n->grad
cudaError_t backward(slbm_ws* n, int B) {
    cudaStream_t st = n->stream;
    const int H = n->H, W = n->W;
    cudaError_t e = cudaSuccess;
    // input gradient of conv i into out (N = cin), masked by the conv's input when that
    // input is a ReLU output (or a concatenation of ReLU outputs)
    auto dgrad = [&](int i, bf16* out, bool mask) {
        if (e != cudaSuccess) return;
        const int l = SPECS[i].level;
        e = launch_mk(n->gz[i], n->wt[i], nullptr, mask ? n->in[i] : nullptr, out, B, H >> l, W >> l, SPECS[i].cout,
                      SPECS[i].cin, 0, n->d_err, st);
    };
    auto unpool = [&](const bf16* gcat, int Ct, bf16* out, int lc, int Cu) {
        if (e != cudaSuccess) return;
        unpool_back_kernel<<<ew_grid(pix(n, lc, B) * Cu / 8), EW, 0, st>>>(gcat, Ct, out, B, H >> lc, W >> lc, Cu);
        e = cudaGetLastError();
    };
    auto poolb = [&](const bf16* act, const bf16* gp, const bf16* gcat, int Ct, int off, bf16* out, int l, int C) {
        if (e != cudaSuccess) return;
        pool_back_kernel<<<ew_grid(pix(n, l, B) * C / 8), EW, 0, st>>>(act, gp, gcat, Ct, off, out, B, H >> l, W >> l, C);
        e = cudaGetLastError();
    };
    dgrad(13, n->gz[12], true);
    dgrad(12, n->gc0, true);
    unpool(n->gc0, 96, n->gz[11], 1, 64);
    dgrad(11, n->gz[10], true);
    dgrad(10, n->gc1, true);
    unpool(n->gc1, 192, n->gz[9], 2, 128);
    dgrad(9, n->gz[8], true);
    dgrad(8, n->gc2, true);
    unpool(n->gc2, 256, n->gz[7], 3, 128);
    dgrad(7, n->gz[6], true);
    dgrad(6, n->gp2, false);
    poolb(n->y[5], n->gp2, n->gc2, 256, 128, n->gz[5], 2, 128);
    dgrad(5, n->gz[4], true);
    dgrad(4, n->gp1, false);
    poolb(n->y[3], n->gp1, n->gc1, 192, 128, n->gz[3], 1, 64);
    dgrad(3, n->gz[2], true);
    dgrad(2, n->gp0, false);
    poolb(n->y[1], n->gp0, n->gc0, 96, 64, n->gz[1], 0, 32);
    dgrad(1, n->gz[0], true);
    for (int i = 0; i < NCONV && e == cudaSuccess; ++i) {
        const int l = SPECS[i].level;
        e = launch_wg(n->in[i], n->gz[i], n->grad + n->w_off[i], B, H >> l, W >> l, SPECS[i].cin, SPECS[i].cout,
                      n->d_err, st);
        if (e != cudaSuccess) break;
        const long long P = pix(n, l, B);
        long long blocks = (P + 63) / 64;
        if (blocks > 1184) blocks = 1184;
        bias_grad_kernel<<<(unsigned)blocks, EW, 0, st>>>(n->gz[i], P, SPECS[i].cout, n->grad + n->b_off[i]);
        e = cudaGetLastError();
    }
    return e;
}

slbm_status check_err(slbm_ws* n) {
    unsigned int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, n->d_err, sizeof(h), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) return wcuda(n, e, "network");
    if (h) {
        cudaMemsetAsync(n->d_err, 0, sizeof(unsigned int), n->stream);
        return wfail(n, SLBM_ECUDA, "tensor-core wait timed out in a conv kernel");
    }
    return SLBM_OK;
}

slbm_status loss_grad(slbm_ws* n, const float* cond, const float* targets, const int* idx, int B, double* loss) {
    if (!cond || !targets || B < 1 || B > n->maxB) return wfail(n, SLBM_EINVAL, "need cond, targets and 1 <= B <= max_batch");
    cudaError_t e = cudaMemsetAsync(n->grad, 0, n->nparam * sizeof(float), n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->d_loss, 0, sizeof(double), n->stream);
    if (e == cudaSuccess) e = forward(n, cond, idx, B);
    if (e == cudaSuccess) {
        long long blocks = (pix(n, 0, B) + EW - 1) / EW;
        if (blocks > 148 * 4) blocks = 148 * 4;
        head_train_kernel<<<(unsigned)blocks, EW, 0, n->stream>>>(n->y[13], n->params + n->hw_off,
                                                                   n->params + n->hb_off, targets, idx, B, n->H, n->W,
                                                                   n->gz[13], n->grad + n->hw_off,
                                                                   n->grad + n->hb_off, n->d_loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward(n, B);
    if (e != cudaSuccess) return wcuda(n, e, "loss_grad launch");
    double h = 0.0;
    e = cudaMemcpyAsync(&h, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream);
    if (e != cudaSuccess) return wcuda(n, e, "loss readback");
    slbm_status s = check_err(n);
    if (s) return s;
    if (loss) *loss = h;
    if (!std::isfinite(h)) return wfail(n, SLBM_EUNSTABLE, "loss is not finite");
    return SLBM_OK;
}

slbm_status adam(slbm_ws* n, float lr, float b1, float b2, float eps) {
    n->adam_t += 1;
    const double c1 = 1.0 / (1.0 - std::pow((double)b1, (double)n->adam_t));
    const double c2 = 1.0 / (1.0 - std::pow((double)b2, (double)n->adam_t));
    adam_kernel<<<ew_grid(n->nparam), EW, 0, n->stream>>>(n->params, n->grad, n->adam_m, n->adam_v, n->nparam, lr, b1, b2,
                                                          eps, (float)c1, (float)c2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = refresh_weights(n);
    return e == cudaSuccess ? SLBM_OK : wcuda(n, e, "adam");
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------- primitives
slbm_status slbm_conv3x3_forward(const uint16_t* x, const uint16_t* w, const float* bias, uint16_t* y, int B, int H,
                                 int W, int Cin, int Cout, int relu, void* stream) {
    if (!x || !w || !y || B < 1 || H < 1 || W < 1 || Cin < 8 || Cin % 8 || Cout < 16 || Cout > 256 || Cout % 16)
        return SLBM_EINVAL;
    if (!aligned16(x) || !aligned16(w) || !aligned16(y)) return SLBM_EINVAL;
    unsigned int* err = prim_err();
    if (!err) return SLBM_ECUDA;
    return launch_mk((const bf16*)x, (const bf16*)w, bias, nullptr, (bf16*)y, B, H, W, Cin, Cout, relu, err,
                     (cudaStream_t)stream) == cudaSuccess ? SLBM_OK : SLBM_ECUDA;
}

slbm_status slbm_conv3x3_flip_weights(const uint16_t* w, uint16_t* wt, int Cin, int Cout, void* stream) {
    if (!w || !wt || Cin < 1 || Cout < 1) return SLBM_EINVAL;
    const long long cnt = (long long)Cout * 9 * Cin;
    flip_weights_kernel<<<ew_grid(cnt), EW, 0, (cudaStream_t)stream>>>((const bf16*)w, (bf16*)wt, Cin, Cout);
    return cudaGetLastError() == cudaSuccess ? SLBM_OK : SLBM_ECUDA;
}

slbm_status slbm_conv3x3_input_grad(const uint16_t* dy, const uint16_t* wt, const uint16_t* mask, uint16_t* dx, int B,
                                    int H, int W, int Cin, int Cout, void* stream) {
    if (!dy || !wt || !dx || B < 1 || H < 1 || W < 1 || Cout < 8 || Cout % 8 || Cin < 16 || Cin > 256 || Cin % 16)
        return SLBM_EINVAL;
    if (!aligned16(dy) || !aligned16(wt) || !aligned16(dx) || (mask && !aligned16(mask))) return SLBM_EINVAL;
    unsigned int* err = prim_err();
    if (!err) return SLBM_ECUDA;
    return launch_mk((const bf16*)dy, (const bf16*)wt, nullptr, (const bf16*)mask, (bf16*)dx, B, H, W, Cout, Cin, 0,
                     err, (cudaStream_t)stream) == cudaSuccess ? SLBM_OK : SLBM_ECUDA;
}

slbm_status slbm_conv3x3_weight_grad(const uint16_t* x, const uint16_t* dy, float* dw, int B, int H, int W, int Cin,
                                     int Cout, void* stream) {
    if (!x || !dy || !dw || B < 1 || H < 1 || W < 1 || Cout < 8 || Cout > 128 || Cout % 8 || Cin < 16 || Cin > 256 ||
        Cin % 16)
        return SLBM_EINVAL;
    if (!aligned16(x) || !aligned16(dy)) return SLBM_EINVAL;
    unsigned int* err = prim_err();
    if (!err) return SLBM_ECUDA;
    return launch_wg((const bf16*)x, (const bf16*)dy, dw, B, H, W, Cin, Cout, err, (cudaStream_t)stream) == cudaSuccess
               ? SLBM_OK
               : SLBM_ECUDA;
}

slbm_status slbm_conv_error(int* flag) {
    if (!flag) return SLBM_EINVAL;
    unsigned int* err = prim_err();
    if (!err) return SLBM_ECUDA;
    unsigned int h = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(h));
    *flag = (int)h;
    return e == cudaSuccess ? SLBM_OK : SLBM_ECUDA;
}

// ---------------------------------------------------------------- network
slbm_status slbm_ws_create(int ny, int nx, int max_batch, unsigned long long seed, void* stream, slbm_ws** out) {
    if (!out) return wfail(nullptr, SLBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (ny < 8 || nx < 8 || ny % 8 || nx % 8 || max_batch < 1)
        return wfail(nullptr, SLBM_EINVAL, "need ny, nx multiples of 8 and max_batch >= 1");
    slbm_ws* n = new (std::nothrow) slbm_ws();
    if (!n) return wfail(nullptr, SLBM_ENOMEM, "host allocation failed");
    n->H = ny;
    n->W = nx;
    n->maxB = max_batch;
    n->stream = (cudaStream_t)stream;
    long long off = 0;
    for (int i = 0; i < NCONV; ++i) {
        n->w_off[i] = off;
        off += (long long)SPECS[i].cout * 9 * SPECS[i].cin;
        n->b_off[i] = off;
        off += SPECS[i].cout;
    }
    n->hw_off = off;
    off += 2 * HEAD_C;
    n->hb_off = off;
    off += 2;
    n->nparam = off;
    const int B = max_batch;
    auto P = [&](int l) { return (size_t)pix(n, l, B); };
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t cnt) {
        if (e == cudaSuccess) e = walloc(n, p, cnt);
    };
    A(&n->params, off); A(&n->grad, off); A(&n->adam_m, off); A(&n->adam_v, off);
    for (int i = 0; i < NCONV; ++i) {
        A(&n->wb[i], (size_t)SPECS[i].cout * 9 * SPECS[i].cin);
        A(&n->wt[i], (size_t)SPECS[i].cout * 9 * SPECS[i].cin);
        A(&n->y[i], P(SPECS[i].level) * SPECS[i].cout);
        A(&n->gz[i], P(SPECS[i].level) * SPECS[i].cout);
    }
    A(&n->x0, P(0) * CIN0);
    A(&n->p0, P(1) * 32); A(&n->p1, P(2) * 64); A(&n->p2, P(3) * 128);
    A(&n->c2, P(2) * 256); A(&n->c1, P(1) * 192); A(&n->c0, P(0) * 96);
    A(&n->gp0, P(1) * 32); A(&n->gp1, P(2) * 64); A(&n->gp2, P(3) * 128);
    A(&n->gc2, P(2) * 256); A(&n->gc1, P(1) * 192); A(&n->gc0, P(0) * 96);
    A(&n->d_loss, 1); A(&n->d_err, 1);
    A(&n->d_cond, (size_t)B * 5); A(&n->d_pred, P(0) * 2);
    A(&n->d_proj, (size_t)B); A(&n->d_ok, (size_t)B);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_ws_create_error = std::string("network allocation: ") + cudaGetErrorString(e);
        slbm_ws_destroy(n);
        return e == cudaErrorMemoryAllocation ? SLBM_ENOMEM : SLBM_ECUDA;
    }
    const bf16* ins[NCONV] = {n->x0, n->y[0], n->p0, n->y[2], n->p1, n->y[4], n->p2,
                              n->y[6], n->c2, n->y[8], n->c1, n->y[10], n->c0, n->y[12]};
    for (int i = 0; i < NCONV; ++i) n->in[i] = ins[i];
    // He-uniform weights, zero biases; head Glorot-uniform
    std::vector<float> h(off, 0.0f);
    uint64_t s = seed;
    auto uni = [&]() { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); };
    for (int i = 0; i < NCONV; ++i) {
        const double bound = std::sqrt(6.0 / (9.0 * SPECS[i].cin));
        for (long long k = 0; k < (long long)SPECS[i].cout * 9 * SPECS[i].cin; ++k)
            h[n->w_off[i] + k] = (float)((2.0 * uni() - 1.0) * bound);
    }
    for (int k = 0; k < 2 * HEAD_C; ++k) h[n->hw_off + k] = (float)((2.0 * uni() - 1.0) * std::sqrt(6.0 / (HEAD_C + 2)));
    *out = n;
    slbm_status st = slbm_ws_set_params(n, h.data());
    if (st) {
        g_ws_create_error = n->err;
        slbm_ws_destroy(n);
        *out = nullptr;
    }
    return st;
}

long long slbm_ws_param_count(const slbm_ws* n) { return n ? n->nparam : 0; }

slbm_status slbm_ws_get_params(slbm_ws* n, float* host) {
    if (!n || !host) return n ? wfail(n, SLBM_EINVAL, "host is NULL") : SLBM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(host, n->params, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? SLBM_OK : wcuda(n, e, "get_params");
}

slbm_status slbm_ws_set_params(slbm_ws* n, const float* host) {
    if (!n || !host) return n ? wfail(n, SLBM_EINVAL, "host is NULL") : SLBM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(n->params, host, n->nparam * sizeof(float), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_m, 0, n->nparam * sizeof(float), n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_v, 0, n->nparam * sizeof(float), n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->d_err, 0, sizeof(unsigned int), n->stream);
    if (e == cudaSuccess) e = refresh_weights(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    n->adam_t = 0;
    return e == cudaSuccess ? SLBM_OK : wcuda(n, e, "set_params");
}

slbm_status slbm_ws_forward(slbm_ws* n, const float* cond, int B, float* out) {
    if (!n) return SLBM_EINVAL;
    if (!cond || !out || B < 1 || B > n->maxB) return wfail(n, SLBM_EINVAL, "need cond, out and 1 <= B <= max_batch");
    cudaError_t e = forward(n, cond, nullptr, B);
    if (e == cudaSuccess) {
        head_fwd_kernel<<<ew_grid(pix(n, 0, B)), EW, 0, n->stream>>>(n->y[13], n->params + n->hw_off,
                                                                      n->params + n->hb_off, B, n->H, n->W, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return wcuda(n, e, "forward");
    return check_err(n);
}

slbm_status slbm_ws_loss_grad(slbm_ws* n, const float* cond, const float* targets, const int* idx, int B,
                              double* loss, float* grad) {
    if (!n) return SLBM_EINVAL;
    slbm_status s = loss_grad(n, cond, targets, idx, B, loss);
    if (s || !grad) return s;
    cudaError_t e = cudaMemcpyAsync(grad, n->grad, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? SLBM_OK : wcuda(n, e, "gradient readback");
}

slbm_status slbm_ws_adam(slbm_ws* n, float lr, float beta1, float beta2, float eps) {
    if (!n) return SLBM_EINVAL;
    if (!(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return wfail(n, SLBM_EINVAL, "bad Adam hyper-parameters");
    return adam(n, lr, beta1, beta2, eps);
}

slbm_status slbm_ws_train_step(slbm_ws* n, const float* cond, const float* targets, const int* idx, int B, float lr,
                               double* loss) {
    if (!n) return SLBM_EINVAL;
    slbm_status s = loss_grad(n, cond, targets, idx, B, loss);
    if (s) return s;
    return slbm_ws_adam(n, lr, 0.9f, 0.999f, 1e-8f);
}

slbm_status slbm_ws_batch_targets(slbm_ws* n, slbm_batch* b, int idx, double psi0, float* targets) {
    if (!n) return SLBM_EINVAL;
    if (!b || !targets || idx < 0 || idx >= b->count || !(psi0 > 0.0))
        return wfail(n, SLBM_EINVAL, "need a batch, an instance index, psi0 > 0 and a target buffer");
    slbm_domain* d = b->dom[idx];
    if (d->p.ny != n->H || d->p.nx != n->W) return wfail(n, SLBM_EINVAL, "instance grid differs from the network's");
    if (!d->fields) return wfail(n, SLBM_ESTATE, "instance never initialised");
    // fields of the current level into the instance's own field buffer (its own partials)
    slbm_status s = diag_into_fields(d);
    if (s) return wfail(n, s, d->err);
    targets_kernel<<<ew_grid(d->N), EW, 0, d->stream>>>(d->fields, d->fields + d->N, d->N, psi0, d->p.psi_on, targets);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return e == cudaSuccess ? SLBM_OK : wcuda(n, e, "targets");
}

slbm_status slbm_ws_warm_start(slbm_ws* n, slbm_batch* b, const int* which, const float* cond, int count,
                               int* accepted) {
    if (!n) return SLBM_EINVAL;
    if (!b || !which || !cond || count < 0) return wfail(n, SLBM_EINVAL, "need a batch, instance list and parameters");
    for (int k = 0; k < count; ++k) {
        const int i = which[k];
        if (i < 0 || i >= b->count) return wfail(n, SLBM_EINVAL, "instance index out of range");
        const slbm_domain* d = b->dom[i];
        if (d->p.ny != n->H || d->p.nx != n->W) return wfail(n, SLBM_EINVAL, "instance grid differs from the network's");
        if (!d->initialised || d->n != 0 || !d->fields)
            return wfail(n, SLBM_ESTATE, "instance must hold its cold start (initialised, no step taken)");
    }
    for (int k0 = 0; k0 < count; k0 += n->maxB) {
        const int B = count - k0 < n->maxB ? count - k0 : n->maxB;
        std::vector<ProjArgs> pa(B);
        for (int k = 0; k < B; ++k) {
            slbm_domain* d = b->dom[which[k0 + k]];
            slbm_totals t;
            slbm_status s = slbm_read_totals(d, &t);    // totals of the cold start
            if (s) return wfail(n, s, d->err);
            ProjArgs& a = pa[k];
            a.pred = n->d_pred + (size_t)k * 2 * d->N;
            a.phi = d->fields;
            a.psi = d->fields + d->N;
            a.N = d->N;
            a.phi_b = d->phi_b;
            a.psi0 = cond[(size_t)(k0 + k) * 5 + 3];
            a.psi_target = t.psi_total;
            a.linear = d->p.constraint == SLBM_CONSTRAINT_LINEAR;
            a.q_target = a.linear ? t.phi_total : t.Q_phi;
            a.psi_on = d->p.psi_on;
            a.ok = n->d_ok + k;
        }
        cudaError_t e = cudaMemcpyAsync(n->d_cond, cond + (size_t)k0 * 5, (size_t)B * 5 * sizeof(float),
                                        cudaMemcpyHostToDevice, n->stream);
        if (e != cudaSuccess) return wcuda(n, e, "warm start upload");
        slbm_status s = slbm_ws_forward(n, n->d_cond, B, n->d_pred);
        if (s) return s;
        e = cudaMemcpyAsync(n->d_proj, pa.data(), (size_t)B * sizeof(ProjArgs), cudaMemcpyHostToDevice, n->stream);
        if (e == cudaSuccess) {
            project_kernel<<<B, 1024, 0, n->stream>>>(n->d_proj);
            e = cudaGetLastError();
        }
        std::vector<int> ok(B, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ok.data(), n->d_ok, B * sizeof(int), cudaMemcpyDeviceToHost, n->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
        if (e != cudaSuccess) return wcuda(n, e, "warm start projection");
        for (int k = 0; k < B; ++k) {
            const int i = which[k0 + k];
            slbm_domain* d = b->dom[i];
            // on failure the instance keeps its cold-start state (the projection wrote
            // only the field scratch, not the populations)
            if (ok[k]) {
                s = slbm_batch_init_fields_device(b, i, d->fields, d->fields + d->N);
                if (s) return wfail(n, s, slbm_batch_last_error(b));
            }
            if (accepted) accepted[k0 + k] = ok[k];
        }
    }
    return SLBM_OK;
}

size_t slbm_ws_device_bytes(const slbm_ws* n) { return n ? n->bytes : 0; }
const char* slbm_ws_last_error(const slbm_ws* n) { return n ? n->err.c_str() : g_ws_create_error.c_str(); }

void slbm_ws_destroy(slbm_ws* n) {
    if (!n) return;
    for (void* p : n->allocs) cudaFree(p);
    delete n;
}

}  // extern "C"
