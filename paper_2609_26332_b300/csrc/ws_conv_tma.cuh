// 3 x 3 convolution (stride 1, zero padding 1, NHWC, BF16 operands, FP32 accumulation) as an
// implicit GEMM fed by the tensor-memory accelerator: M = 128 pixels per CTA, N = output
// channels (16..256, one tensor-memory column each), K = 9 taps x C input channels in blocks
// of KC = 64, 32 or 16 channels.
//
// With NHWC activations the channel is the innermost tensor dimension, so the operand of
// tap (dy, dx) for a tile of pixels is one box of the 4-D tensor [B][H][W][C] at the shifted
// coordinates (c0, x0 + dx, y0 + dy, b0): the innermost coordinate stays a multiple of KC
// (16-byte aligned), the spatial ones may be -1 or one past the edge, where the copy fills
// zeros (the convolution's padding).  The pixel tile is Wt x Ht x Bt = 128 (a row segment,
// several rows, or several images of a small field).  The weights [N][9][C] are a 2-D tensor
// [N][9 C] read as one KC x N box per K block.  Boxes land 128-, 64- or 32-byte swizzled
// (KC = 64, 32, 16), the canonical K-major layouts of the tcgen05 shared-memory descriptors.
//
// Roles (persistent CTAs, six warps): one lane of warp 0 issues the boxes into a ring of
// stages (each completing a "full" mbarrier with its byte count); one lane of warp 1 waits
// for a full stage, issues the KC / 16 MMAs and commits them to the stage's "empty"
// mbarrier, which frees it for the producer; tile i accumulates into one of two tensor-memory
// buffers, whose "acc_full" commit hands it to the four epilogue warps (bias / ReLU / mask,
// BF16 stores), which free it through "acc_empty".  Every wait is bounded: on timeout the
// error flag is raised, the role stops, copies already issued are waited for (bounded),
// tensor memory is freed and the CTA exits.
#pragma once
#include <cuda.h>   // CUtensorMap (type only)
#include "ws_conv.cuh"

namespace ws {

constexpr int TC_THREADS = 192;   // producer warp, MMA warp, four epilogue warps
constexpr int TC_MAX_STAGES = 8;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
            dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor of a swizzled K-major operand: start address, leading
// byte offset 16 (unused by the swizzled K-major layouts), stride byte offset = the distance
// between 8-row groups, layout type (2: 128-byte swizzle, 4: 64-byte, 6: 32-byte)
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t saddr, uint32_t sbo, uint32_t layout) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)layout << 61;
    return d;
}

struct TConvArgs {
    const float* bias;            // [N] or null
    const __nv_bfloat16* mask;    // [P][N] or null: outputs where mask <= 0 are zeroed
    __nv_bfloat16* y;             // [P][N]
    int B, H, W, C, N, relu;
    int Wt, Ht, Bt;               // pixel tile, Wt Ht Bt = 128
    int KC;                       // channels per K block: 64, 32 or 16
    int stages;                   // ring depth, <= TC_MAX_STAGES
    uint32_t a_bytes, b_bytes;    // bytes of the A and B tiles of a stage (multiples of 1024)
    unsigned int* err;
};

// Persistent, warp-specialised: CTA b takes tiles b, b + gridDim.x, ...  Warp 0 (one lane)
// streams the boxes of every tile's K blocks through the ring; warp 1 (one lane) issues the
// MMAs of tile i into accumulator buffer i % 2 of tensor memory and commits "acc_full";
// warps 2..5 read a full accumulator (warp w holds the lane quarter w % 4, i.e. pixels
// 32 (w % 4) ..), write the epilogue and arrive on "acc_empty", so the epilogue of one tile
// runs while the next tile's blocks stream in.
__global__ void __launch_bounds__(TC_THREADS, 1)
    conv_tma_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw, const TConvArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;   // swizzle atoms on 1024-byte boundaries
    const int S = a.stages;
    const uint32_t stage_bytes = a.a_bytes + a.b_bytes;
    const uint32_t ncols = tmem_cols_for(a.N);   // one accumulator; two are allocated
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);   // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_base, 2 * ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    const int nW = a.W / a.Wt, nH = a.H / a.Ht;
    const int ntiles = nW * nH * (a.B / a.Bt);
    const int CB = a.C / a.KC, NKB = 9 * CB;
    auto tile_origin = [&](int t, int& x0, int& y0, int& b0) {
        const int xt = t % nW;
        t /= nW;
        x0 = xt * a.Wt;
        y0 = (t % nH) * a.Ht;
        b0 = (t / nH) * a.Bt;
    };

    if (warp == 0) {
        if (lane == 0) {
            // producer: every K block of every tile of this CTA through the ring
            int last[TC_MAX_STAGES];
            for (int s = 0; s < S; ++s) last[s] = -1;
            long long g = 0;   // blocks issued by this CTA
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int x0, y0, b0;
                tile_origin(t, x0, y0, b0);
                for (int kb = 0; kb < NKB; ++kb, ++g) {
                    const int s = (int)(g % S);
                    if (g >= S && !mbar_wait(&empty[s], (uint32_t)(g / S - 1) & 1u, WAIT_LIMIT_NS)) {
                        ok = false;
                        atomicOr(a.err, ERR_TIMEOUT);
                        break;
                    }
                    const int tap = kb / CB, cb = kb - tap * CB;
                    const uint32_t sA = base + (uint32_t)s * stage_bytes;
                    mbar_expect_tx(&full[s], stage_bytes);
                    tma_load_4d(sA, &mx, cb * a.KC, x0 + tap % 3 - 1, y0 + tap / 3 - 1, b0, &full[s]);
                    tma_load_2d(sA + a.a_bytes, &mw, tap * a.C + cb * a.KC, 0, &full[s]);
                    last[s] = (int)(g / S);
                }
            }
            // copies issued must land before the CTA leaves (they already have unless a wait ran out)
            for (int s = 0; s < S; ++s)
                if (last[s] >= 0) mbar_wait(&full[s], (uint32_t)last[s] & 1u, WAIT_LIMIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile i of this CTA accumulates into buffer i % 2
            const uint32_t layout = a.KC == 64 ? 2u : (a.KC == 32 ? 4u : 6u);
            const uint32_t sbo = 16u * (uint32_t)a.KC;   // 8 rows of KC two-byte channels
            const uint32_t idesc = idesc_bf16(128, a.N, false, false);
            long long g = 0;
            bool ok = true;
            int li = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++li) {
                const int ab = li & 1;
                if (li >= 2 && !mbar_wait(&acc_empty[ab], (uint32_t)(li / 2 - 1) & 1u, WAIT_LIMIT_NS)) {
                    atomicOr(a.err, ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)ab * ncols;
                for (int kb = 0; kb < NKB; ++kb, ++g) {
                    const int s = (int)(g % S);
                    if (!mbar_wait(&full[s], (uint32_t)(g / S) & 1u, WAIT_LIMIT_NS)) {
                        ok = false;
                        atomicOr(a.err, ERR_TIMEOUT);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sA = base + (uint32_t)s * stage_bytes, sB = sA + a.a_bytes;
                    for (int j = 0; j < a.KC / 16; ++j)
                        mma_bf16(acc, smem_desc_sw(sA + 32u * j, sbo, layout), smem_desc_sw(sB + 32u * j, sbo, layout),
                                 idesc, (kb | j) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                mma_commit(&acc_full[ab]);   // arrives once this tile's MMAs have completed
            }
        }
    } else {
        // epilogue warps 2..5: lane quarter q of the accumulator = pixels 32 q .. 32 q + 31
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int ww = m % a.Wt, hh = (m / a.Wt) % a.Ht, bb = m / (a.Wt * a.Ht);
        int li = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++li) {
            const int ab = li & 1;
            const bool ok = mbar_wait(&acc_full[ab], (uint32_t)(li / 2) & 1u, WAIT_LIMIT_NS);
            __syncwarp();
            if (!ok) {
                if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            int x0, y0, b0;
            tile_origin(t, x0, y0, b0);
            const long long p = ((long long)(b0 + bb) * a.H + (y0 + hh)) * a.W + (x0 + ww);
            const uint32_t trow = tmem + (uint32_t)ab * ncols + ((uint32_t)(q * 32) << 16);
            for (int j = 0; j < a.N / 16; ++j) {
                float v[16];
                tmem_ld16(trow + (uint32_t)(16 * j), v);
                const size_t off = (size_t)p * a.N + 16 * j;
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
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * ncols);
    }
}

}  // namespace ws
