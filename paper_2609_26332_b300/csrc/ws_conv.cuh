// 3 x 3 convolutions (stride 1, zero padding 1, NHWC, BF16 operands, FP32 accumulation)
// as implicit GEMMs on the tcgen05 tensor cores.
//
//   conv_mk_kernel   M = pixels (128 per CTA), N = output channels, K = 9 taps x C inputs:
//                    forward (bias, ReLU) and input gradient (flipped, transposed weights;
//                    output multiplied by a ReLU mask)
//   conv_wg_kernel   M = output channels (zero-padded to 128), N = input channels of one
//                    tap, K = pixels (split over CTAs, FP32 atomics into the weight gradient)
//
// Operands are gathered by the CTA's threads with 16-byte cp.async (zero fill outside the
// image) straight into the core-matrix layout, four-stage ring; one thread issues the MMAs
// and commits each stage to an mbarrier that frees it.  Every wait is bounded: on timeout
// the kernel raises the error flag, drains what it issued, frees tensor memory and exits.
#pragma once
#include "ws_tc.cuh"

namespace ws {

constexpr int CONV_THREADS = 128;
constexpr int CONV_STAGES = 4;      // deepest ring; 32-channel tiles use 3 (three CTAs per SM)
constexpr uint32_t A_STAGE_BYTES = 128 * 64 * 2;     // 128 rows x 64 K-elements
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;      // 2 s: far beyond any legitimate wait

enum { ERR_TIMEOUT = 1 };

__host__ __device__ inline uint32_t tmem_cols_for(int n) { return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : 256u; }
__host__ __device__ inline uint32_t mk_stage_bytes(int n) { return A_STAGE_BYTES + (uint32_t)n * 128u; }
__host__ __device__ inline uint32_t wg_stage_bytes(int c) { return A_STAGE_BYTES + (uint32_t)c * 128u; }

struct MKArgs {
    const __nv_bfloat16* x;     // [P][C] gathered input, P = B H W
    const __nv_bfloat16* w;     // [N][9][C] (tap = 3 (dy + 1) + (dx + 1))
    const float* bias;          // [N] or null
    const __nv_bfloat16* mask;  // [P][N] or null: outputs where mask <= 0 are zeroed
    __nv_bfloat16* y;           // [P][N]
    int B, H, W, C, N;
    int relu;
    unsigned int* err;
};

struct WGArgs {
    const __nv_bfloat16* x;     // [P][C] input of the layer
    const __nv_bfloat16* dz;    // [P][N] gradient of the layer's pre-activation output
    float* dw;                  // [N][9][C], accumulated
    int B, H, W, C, N;
    long long pix_per_cta;      // multiple of 64
    unsigned int* err;
};

// ------------------------------------------------------------------ shared pipeline pieces
struct Pipe {
    uint64_t bar[CONV_STAGES];
    uint32_t tmem;
    int abort;
    int last;                   // last committed K block
};

__device__ __forceinline__ void pipe_open(Pipe& S, uint32_t ncols) {
    const int tid = threadIdx.x;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < CONV_STAGES; ++s) mbar_init(&S.bar[s], 1);
        S.abort = 0;
        S.last = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) tmem_alloc(&S.tmem, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// drain after the main loop: wait (bounded) for the last committed MMA group
template <int STAGES>
__device__ __forceinline__ bool pipe_drain(Pipe& S, unsigned int* err) {
    cp_wait<0>();
    __syncthreads();
    const int last = S.last;
    bool ok = !S.abort;
    if (last >= 0) {
        const bool done = mbar_wait(&S.bar[last % STAGES], (uint32_t)(last / STAGES) & 1u, WAIT_LIMIT_NS);
        if (!done) {
            ok = false;
            atomicOr(err, ERR_TIMEOUT);
        }
    }
    tc_fence_after();
    return ok;
}

__device__ __forceinline__ void pipe_close(Pipe& S, uint32_t ncols) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(S.tmem, ncols);
    }
}

// one K block (64 elements = 4 MMAs of K = 16) from stage s
__device__ __forceinline__ void issue_block(uint32_t tmem, uint32_t sA, uint32_t sB, uint32_t a_lbo, uint32_t a_sbo,
                                            uint32_t b_lbo, uint32_t b_sbo, uint32_t idesc, bool first) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint64_t ad = smem_desc(sA + (uint32_t)j * 2u * a_lbo, a_lbo, a_sbo);
        const uint64_t bd = smem_desc(sB + (uint32_t)j * 2u * b_lbo, b_lbo, b_sbo);
        mma_bf16(tmem, ad, bd, idesc, (first && j == 0) ? 0u : 1u);
    }
}

// ------------------------------------------------------------------ forward / input gradient
// A (pixels x K, K-major): core matrix (row group g, K chunk c) at c * 2048 + g * 128.
// B (N x K, K-major):      core matrix (row group h, K chunk c) at c * 16 N + h * 128.
template <int STAGES>
__global__ void __launch_bounds__(CONV_THREADS, 1) conv_mk_kernel(const MKArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Pipe S;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int N = a.N, C = a.C, CB = C >> 3, KC = 9 * CB, NKB = (KC + 7) >> 3;
    const long long P = (long long)a.B * a.H * a.W;
    const long long m = (long long)blockIdx.x * 128 + tid;
    const uint32_t stage = mk_stage_bytes(N), ncols = tmem_cols_for(N);
    const uint32_t sbase = smem_u32(smem);
    pipe_open(S, ncols);
    const uint32_t tmem = S.tmem;

    const bool mvalid = m < P;
    int px = 0, py = 0;
    long long pimg = 0;
    if (mvalid) {
        px = (int)(m % a.W);
        const long long t = m / a.W;
        py = (int)(t % a.H);
        pimg = t / a.H;
    }
    // gather set-up, once per thread: the own pixel's element offset, which of the 9 taps
    // land inside the image, and the weight rows this thread copies
    const __nv_bfloat16* own = a.x + (mvalid ? m * C : 0);
    unsigned vmask = 0;
    if (mvalid) {
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = py + t / 3 - 1, xx = px + t % 3 - 1;
            if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) vmask |= 1u << t;
        }
    }
    const long long rowC = (long long)a.W * C;
    const bool brow0 = tid < N, brow1 = tid + CONV_THREADS < N;
    const __nv_bfloat16* wrow0 = brow0 ? a.w + (size_t)tid * KC * 8 : a.w;
    const __nv_bfloat16* wrow1 = brow1 ? a.w + (size_t)(tid + CONV_THREADS) * KC * 8 : a.w;
    auto tap_offset = [&](int tap) { return (long long)(tap / 3 - 1) * rowC + (long long)(tap % 3 - 1) * C; };
    auto load = [&](int kb) {
        const uint32_t sA = sbase + (uint32_t)(kb % STAGES) * stage, sB = sA + A_STAGE_BYTES;
        const int kc = kb * 8;
        int tap = kc / CB, cb = kc - tap * CB;
        long long toff = tap_offset(tap);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int k = kc + c;
            const bool kv = k < KC;
            const bool v = kv && ((vmask >> tap) & 1u);
            cp16_ca(sA + (uint32_t)c * 2048u + (uint32_t)tid * 16u, v ? own + toff + cb * 8 : a.x, v);
            const uint32_t bdst = sB + (uint32_t)c * (uint32_t)(16 * N) + (uint32_t)tid * 16u;
            if (brow0) cp16_cg(bdst, kv ? wrow0 + (size_t)k * 8 : a.w, kv);
            if (brow1) cp16_cg(bdst + (uint32_t)CONV_THREADS * 16u, kv ? wrow1 + (size_t)k * 8 : a.w, kv);
            if (++cb == CB) {
                cb = 0;
                ++tap;
                toff = tap_offset(tap);
            }
        }
    };

    const uint32_t idesc = idesc_bf16(128, N, false, false);
    for (int kb = 0; kb < STAGES - 1; ++kb) {
        if (kb < NKB) load(kb);
        cp_commit();
    }
    for (int kb = 0; kb < NKB; ++kb) {
        cp_wait<STAGES - 2>();
        fence_async_smem();
        __syncthreads();
        if (S.abort) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t sA = sbase + (uint32_t)(kb % STAGES) * stage;
            issue_block(tmem, sA, sA + A_STAGE_BYTES, 2048u, 128u, (uint32_t)(16 * N), 128u, idesc, kb == 0);
            mma_commit(&S.bar[kb % STAGES]);
            S.last = kb;
        }
        const int kn = kb + STAGES - 1;
        if (kn < NKB) {
            bool ok = true;
            if (kb >= 1) ok = mbar_wait(&S.bar[(kb - 1) % STAGES], (uint32_t)((kb - 1) / STAGES) & 1u, WAIT_LIMIT_NS);
            if (ok) load(kn);
            else {
                S.abort = 1;
                atomicOr(a.err, ERR_TIMEOUT);
            }
        }
        cp_commit();
    }
    const bool ok = pipe_drain<STAGES>(S, a.err);
    if (ok) {
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int j = 0; j < N / 16; ++j) {
            float v[16];
            tmem_ld16(trow + (uint32_t)(16 * j), v);
            if (mvalid) {
                const size_t off = (size_t)m * N + 16 * j;
                if (a.bias) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += a.bias[16 * j + i];
                }
                if (a.relu) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.0f);
                }
                if (a.mask) {
                    const uint4* mp = (const uint4*)(a.mask + off);
                    uint4 mv[2] = {mp[0], mp[1]};
                    const __nv_bfloat16* mb = (const __nv_bfloat16*)mv;
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = __bfloat162float(mb[i]) > 0.0f ? v[i] : 0.0f;
                }
                uint4 ov[2];
                __nv_bfloat162* ob = (__nv_bfloat162*)ov;
#pragma unroll
                for (int i = 0; i < 8; ++i) ob[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                uint4* yp = (uint4*)(a.y + off);
                yp[0] = ov[0];
                yp[1] = ov[1];
            }
        }
    }
    pipe_close(S, ncols);
}

// ------------------------------------------------------------------ weight gradient
// A (Cout x pixels, MN-major): core matrix (channel group g, pixel group q) at q * 2048 + g * 128.
// B (Cin x pixels, MN-major):  core matrix (channel group h, pixel group q) at q * 16 C + h * 128.
// grid: (pixel splits, 9 taps)
template <int STAGES>
__global__ void __launch_bounds__(CONV_THREADS, 1) conv_wg_kernel(const WGArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Pipe S;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int C = a.C, Co = a.N, tap = blockIdx.y;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long long P = (long long)a.B * a.H * a.W;
    const long long p0 = (long long)blockIdx.x * a.pix_per_cta;
    const long long p1 = p0 + a.pix_per_cta < P ? p0 + a.pix_per_cta : P;
    const int NKB = p1 > p0 ? (int)((p1 - p0 + 63) / 64) : 0;
    const uint32_t stage = wg_stage_bytes(C), ncols = tmem_cols_for(C);
    const uint32_t sbase = smem_u32(smem);
    // rows Co..127 of A stay zero in every stage
    for (int s = 0; s < STAGES; ++s) {
        unsigned char* sa = smem + (size_t)s * stage;
        for (int q = 0; q < 8; ++q)
            for (int g = Co / 8 + (tid >> 3); g < 16; g += CONV_THREADS / 8)
                *(uint4*)(sa + q * 2048 + g * 128 + (tid & 7) * 16) = make_uint4(0, 0, 0, 0);
    }
    pipe_open(S, ncols);
    const uint32_t tmem = S.tmem;

    const int pl = tid & 63, gsub = tid >> 6;
    // this thread's pixel of K block 0; every block advances it by 64 pixels
    int cx = 0, cy = 0;
    {
        const long long p = p0 + pl;
        cx = (int)(p % a.W);
        cy = (int)((p / a.W) % a.H);
    }
    long long pcur = p0 + pl;
    const uint32_t qoffA = (uint32_t)(pl >> 3) * 2048u + (uint32_t)(pl & 7) * 16u;
    const uint32_t qoffB = (uint32_t)(pl >> 3) * (uint32_t)(16 * C) + (uint32_t)(pl & 7) * 16u;
    const long long dxy = (long long)dy * a.W + dx;
    auto load = [&](int kb) {   // called with kb = 0, 1, 2, ... in order
        const uint32_t sA = sbase + (uint32_t)(kb % STAGES) * stage, sB = sA + A_STAGE_BYTES;
        const bool pv = pcur < p1;
        const int yy = cy + dy, xx = cx + dx;
        const bool xv = pv && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
        const long long xoff = xv ? (pcur + dxy) * C : 0;
        for (int g = gsub; g < Co / 8; g += 2)
            cp16_cg(sA + qoffA + (uint32_t)g * 128u, pv ? a.dz + (size_t)pcur * Co + g * 8 : a.dz, pv);
        for (int h = gsub; h < C / 8; h += 2)
            cp16_ca(sB + qoffB + (uint32_t)h * 128u, xv ? a.x + xoff + h * 8 : a.x, xv);
        pcur += 64;
        cx += 64;
        while (cx >= a.W) {
            cx -= a.W;
            if (++cy == a.H) cy = 0;
        }
    };

    const uint32_t idesc = idesc_bf16(128, C, true, true);
    for (int kb = 0; kb < STAGES - 1; ++kb) {
        if (kb < NKB) load(kb);
        cp_commit();
    }
    for (int kb = 0; kb < NKB; ++kb) {
        cp_wait<STAGES - 2>();
        fence_async_smem();
        __syncthreads();
        if (S.abort) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t sA = sbase + (uint32_t)(kb % STAGES) * stage;
            issue_block(tmem, sA, sA + A_STAGE_BYTES, 2048u, 128u, (uint32_t)(16 * C), 128u, idesc, kb == 0);
            mma_commit(&S.bar[kb % STAGES]);
            S.last = kb;
        }
        const int kn = kb + STAGES - 1;
        if (kn < NKB) {
            bool ok = true;
            if (kb >= 1) ok = mbar_wait(&S.bar[(kb - 1) % STAGES], (uint32_t)((kb - 1) / STAGES) & 1u, WAIT_LIMIT_NS);
            if (ok) load(kn);
            else {
                S.abort = 1;
                atomicOr(a.err, ERR_TIMEOUT);
            }
        }
        cp_commit();
    }
    const bool ok = pipe_drain<STAGES>(S, a.err);
    if (ok && NKB > 0) {
        const int co = warp * 32 + (tid & 31);
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int j = 0; j < C / 16; ++j) {
            float v[16];
            tmem_ld16(trow + (uint32_t)(16 * j), v);
            if (co < Co) {
                float* dst = a.dw + ((size_t)co * 9 + tap) * C + 16 * j;
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(dst + i, v[i]);
            }
        }
    }
    pipe_close(S, ncols);
}

}  // namespace ws
