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

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(
            dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
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

// shared-memory matrix descriptor of a swizzled MN-major operand: leading byte offset =
// the distance between swizzle atoms along M / N, stride byte offset = the distance between
// 8-row groups along K
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
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

namespace ws {

// ------------------------------------------------------------------ weight gradient on TMA
// dW[co][tap][ci] = sum_p dz[p][co] x[p + s_tap][ci] (zero outside the image), one GEMM per
// tap with K = pixels: D (M x N) += A (M x 64 pixels) B (N x 64 pixels)^T per K block.  Both
// operands are MN-major in NHWC memory (channels contiguous per pixel).  An operand of a K
// block is AW-channel boxes of the 4-D view [B][H][W][C] (AW = 64, 32 or 16 channels, the
// swizzle atom width: 128, 64 or 32 bytes), each landing as 64 pixel rows x 2 AW bytes,
// swizzled: the canonical MN-major layout whose atoms are 8 pixel rows x 2 AW bytes, with
// the descriptor's leading byte offset = the distance between channel atoms (one box,
// 128 AW bytes) and its stride byte offset = the distance between 8-pixel groups (16 AW
// bytes).  The x operand's boxes sit at the tap-shifted pixel coordinates (zero fill outside
// the image).  M rows are the 128 accumulator lanes: the operand with the larger channel
// count that fits (<= 128) takes M ("swap": x in A, dz in B); its atoms past the channel
// count stay zero in every stage.  grid (splits, 9 taps): CTA (s, t) reduces a contiguous
// range of K blocks of tap t and adds its partial result to dw with FP32 atomics.
struct TWGArgs {
    float* dw;                    // [Cout][9][Cin], accumulated
    int B, H, W, Cin, Cout;
    int Wb, Hb;                   // pixel box, Wb Hb = 64
    int swap;                     // 1: A = x (M = Cin), B = dz (N = Cout); 0: A = dz, B = x
    int awA, awB;                 // atom widths (channels) of the A and B operands
    int nkb_total, kb_per_cta;
    int stages;
    uint32_t a_bytes, b_bytes;    // stage bytes of A (128 rows: 16 KB) and B (N x 128 bytes, 1 KB rounded)
    unsigned int* err;
};

__device__ __forceinline__ uint32_t sw_layout(int aw) { return aw == 64 ? 2u : (aw == 32 ? 4u : 6u); }

__global__ void __launch_bounds__(TC_THREADS, 1)
    conv_wg_tma_kernel(const __grid_constant__ CUtensorMap mdz, const __grid_constant__ CUtensorMap mx, const TWGArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES], done;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - smem_u32(smem_raw));
    const int S = a.stages;
    const uint32_t stage_bytes = a.a_bytes + a.b_bytes;
    const int Mv = a.swap ? a.Cin : a.Cout, N = a.swap ? a.Cout : a.Cin;
    const int nA = Mv / a.awA, nB = N / a.awB;
    const uint32_t boxA = 128u * (uint32_t)a.awA, boxB = 128u * (uint32_t)a.awB;   // bytes of one box
    const uint32_t ncols = tmem_cols_for(N);
    const int tap = blockIdx.y, dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int kb0 = blockIdx.x * a.kb_per_cta;
    const int kb1 = kb0 + a.kb_per_cta < a.nkb_total ? kb0 + a.kb_per_cta : a.nkb_total;
    // A atoms past the M channels stay zero in every stage
    for (int s = 0; s < S; ++s) {
        unsigned char* sa = gbase + (size_t)s * stage_bytes;
        for (uint32_t i = (uint32_t)nA * boxA / 16u + tid; i < a.a_bytes / 16u; i += TC_THREADS)
            *(uint4*)(sa + (size_t)i * 16) = make_uint4(0, 0, 0, 0);
    }
    fence_async_smem();
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_base, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int nWb = a.W / a.Wb, nHb = a.H / a.Hb;
    const CUtensorMap* mapA = a.swap ? &mx : &mdz;
    const CUtensorMap* mapB = a.swap ? &mdz : &mx;
    const int sxA = a.swap ? dx : 0, syA = a.swap ? dy : 0, sxB = a.swap ? 0 : dx, syB = a.swap ? 0 : dy;

    if (warp == 0) {
        if (lane == 0) {
            int last[TC_MAX_STAGES];
            for (int s = 0; s < S; ++s) last[s] = -1;
            for (int kb = kb0, g = 0; kb < kb1; ++kb, ++g) {
                const int s = g % S;
                if (g >= S && !mbar_wait(&empty[s], (uint32_t)(g / S - 1) & 1u, WAIT_LIMIT_NS)) {
                    atomicOr(a.err, ERR_TIMEOUT);
                    break;
                }
                int t = kb;
                const int xb = t % nWb;
                t /= nWb;
                const int yb = t % nHb, b = t / nHb;
                const int px = xb * a.Wb, py = yb * a.Hb;
                const uint32_t sA = base + (uint32_t)s * stage_bytes, sB = sA + a.a_bytes;
                mbar_expect_tx(&full[s], (uint32_t)nA * boxA + (uint32_t)nB * boxB);
                for (int i = 0; i < nA; ++i)
                    tma_load_4d(sA + (uint32_t)i * boxA, mapA, i * a.awA, px + sxA, py + syA, b, &full[s]);
                for (int i = 0; i < nB; ++i)
                    tma_load_4d(sB + (uint32_t)i * boxB, mapB, i * a.awB, px + sxB, py + syB, b, &full[s]);
                last[s] = g / S;
            }
            for (int s = 0; s < S; ++s)
                if (last[s] >= 0) mbar_wait(&full[s], (uint32_t)last[s] & 1u, WAIT_LIMIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, N, true, true);
            const uint32_t la = sw_layout(a.awA), lb = sw_layout(a.awB);
            for (int kb = kb0, g = 0; kb < kb1; ++kb, ++g) {
                const int s = g % S;
                if (!mbar_wait(&full[s], (uint32_t)(g / S) & 1u, WAIT_LIMIT_NS)) {
                    atomicOr(a.err, ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t sA = base + (uint32_t)s * stage_bytes, sB = sA + a.a_bytes;
                // 4 MMAs of K = 16 pixel rows: two 8-row groups (16 AW bytes apart) each
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t da = smem_desc_mn(sA + 32u * a.awA * j, boxA, 16u * a.awA, la);
                    const uint64_t db = smem_desc_mn(sB + 32u * a.awB * j, boxB, 16u * a.awB, lb);
                    mma_bf16(tmem, da, db, idesc, (g | j) ? 1u : 0u);
                }
                mma_commit(&empty[s]);
            }
            mma_commit(&done);
        }
    }
    __syncwarp();
    const bool ok = kb1 > kb0 && mbar_wait(&done, 0u, WAIT_LIMIT_NS);
    tc_fence_after();
    __syncwarp();
    if (ok && warp >= 2) {
        const int q = warp & 3;
        const int row = q * 32 + lane;   // accumulator lane: channel of the M operand
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
        for (int j = 0; j < N / 16; ++j) {
            float v[16];
            tmem_ld16(trow + (uint32_t)(16 * j), v);
            if (row < Mv) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = 16 * j + i;
                    const int co = a.swap ? n : row, ci = a.swap ? row : n;
                    atomicAdd(a.dw + ((size_t)co * 9 + tap) * a.Cin + ci, v[i]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

}  // namespace ws
