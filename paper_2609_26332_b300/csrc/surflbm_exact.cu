// Exact discrete multiplier (the constraint of Sec. 2, H(phi) = sum h_phi(phi), imposed on
// the lattice field instead of through the continuous projection of Eq. eq15).
//
// After step n, phi^{n+1} is affine in lambda^n: the multiplier enters the phi populations
// only as w_i a M_phi lambda h'(phi^n) (a = 1.5, or 1 on the first step), and the step
// kernel leaves that term to the next launch, which adds it to each node's zeroth moment
// before the pull.  So, from the stored post-collision state,
//     phi^{n+1}(x) = A(x) + lambda B(x),
//     A = the pull with the term left out (the step kernel's own fixed-point exchange),
//     B = sum_k w_k a M_phi h'(phi^n(x_k)),  x_k the node the k-th link pulls from
//         (its mirror across a wall, as in the specular scalar walls),
// and H(A + lambda B) = H(phi^0) is a cubic in lambda (h = 1/2 + g, g cubic in phi; linear
// for the linear constraint).  One pass reduces the four coefficients in float-float per
// thread and FP64 across blocks; the last block takes Newton steps from the step kernel's
// estimate and overwrites lambda^n in the record of the level, which the next step reads.
#include "surflbm_internal.cuh"

using namespace slbm;

namespace {

constexpr int EX_THREADS = NTHREADS;
constexpr int EX_TX = 32, EX_TY = EX_THREADS / EX_TX;

template <class T>
struct ExactArgs {
    int nx, ny;
    long long N;
    const T* gd;            // deviations of the phi set, planes k = 1..8 (post-collision, step n)
    const float2* gm;       // its zeroth moments (float-float)
    const float* php;       // phi^n
    double* partials;       // [gridDim][NPART]
    unsigned int* counter;
    Rec* rec;               // record of level n: in lam (estimate), H0, a; out lam
    Phys P;
};

// the fixed-point value node c sends in direction k without the deferred term
// (the step kernel's stage K with a zero multiplier coefficient)
template <class T>
__device__ __forceinline__ int sent_fixed(const ExactArgs<T>& a, long long c, int k, float2 m, float scl) {
    const float wsc = __fmul_rn(k < 5 ? Wk(1) : Wk(5), scl);
    return __float2int_rn(__fmaf_rn(Stor<T>::ld(a.gd, (long long)(k - 1) * a.N + c), scl, __fmul_rn(wsc, m.x)));
}

template <class T>
__global__ void __launch_bounds__(EX_THREADS) exact_multiplier_kernel(const ExactArgs<T> a) {
    const Phys& P = a.P;
    const float scl = (float)(1u << SFIX_PHI), isc = 1.0f / scl;
    const float coef = (float)(a.rec->a * P.M_phi_d);     // a M_phi
    ff acc[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) acc[q] = {0.0f, 0.0f};
    // tiles of EX_TX x EX_TY cells with a one-node halo: each node's eight sent fixed-point
    // values, h'(phi^n) and zeroth moment are evaluated once into shared memory (phase 1),
    // then every cell sums what it sends and receives from there (phase 2)
    constexpr int HX = EX_TX + 2, HN = HX * (EX_TY + 2);
    __shared__ int sKs[8][HN];
    __shared__ float sHp[HN];
    __shared__ float2 sM[HN];
    const int ntx = (a.nx + EX_TX - 1) / EX_TX, nty = (a.ny + EX_TY - 1) / EX_TY;
    const int tx = threadIdx.x % EX_TX, ty = threadIdx.x / EX_TX;
    for (int t = blockIdx.x; t < ntx * nty; t += gridDim.x) {
        const int ty0 = t / ntx;
        const int x0 = (t - ty0 * ntx) * EX_TX, y0 = ty0 * EX_TY;
        __syncthreads();   // the previous tile's phase 2 has read the shared arrays
        for (int q = threadIdx.x; q < HN; q += EX_THREADS) {
            const int hy = q / HX, hx = q - hy * HX;
            const int gy = y0 - 1 + hy;
            if (gy < 0 || gy >= a.ny) continue;   // beyond a wall: the links use mirrors in the own row
            int gx = (x0 - 1 + hx) % a.nx;
            if (gx < 0) gx += a.nx;
            const long long sidx = (long long)gy * a.nx + gx;
            const float2 m = a.gm[sidx];
            sM[q] = m;
#pragma unroll
            for (int k = 1; k < 9; ++k) sKs[k - 1][q] = sent_fixed(a, sidx, k, m, scl);
            sHp[q] = P.linear ? 1.0f : hprime(a.php[sidx], P);
        }
        __syncthreads();
        const int x = x0 + tx, y = y0 + ty;
        if (x >= a.nx || y >= a.ny) continue;
        const int q0 = (ty + 1) * HX + (tx + 1);
        const float2 m = sM[q0];
        int ksum = 0;
#pragma unroll
        for (int k = 1; k < 9; ++k) ksum += sKs[k - 1][q0];
        int krecv = 0;
        // h' = 1 for the linear constraint: the term's total is exactly N a M_phi lambda
        // (the fixed-point exchange telescopes), so its distribution need not be summed
        float bsum = P.linear ? 1.0f : Wk(0) * sHp[q0];
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            const int sy = y - CYk(k);
            const bool out = sy < 0 || sy >= a.ny;   // specular: the mirrored direction of the own row
            const int qs = (ty + 1 - (out ? 0 : CYk(k))) * HX + (tx + 1 - CXk(k));
            krecv += sKs[(out ? MIRYk(k) : k) - 1][qs];
            if (!P.linear) bsum = __fmaf_rn(Wk(k), sHp[qs], bsum);
        }
        const ff A = ff_add(ff_add({m.x, m.y}, fixed_to_ff(-ksum, isc)), fixed_to_ff(krecv, isc));
        const float B = coef * bsum;
        if (P.linear) {
            acc[0] = ff_add(acc[0], A);
            acc[1] = ff_add_f(acc[1], B);
        } else {
            const float u = (A.hi + A.lo) * P.inv_phi_b, v = B * P.inv_phi_b;
            // Q(u + lambda v) with Q = (3u - u^3)/2 = 2 g, expanded in lambda
            acc[0] = ff_add_f(acc[0], 1.5f * u - 0.5f * u * u * u);
            acc[1] = ff_add_f(acc[1], 1.5f * v * (1.0f - u * u));
            acc[2] = ff_add_f(acc[2], -1.5f * u * v * v);
            acc[3] = ff_add_f(acc[3], -0.5f * v * v * v);
        }
    }

    __shared__ double s_blk[NPART], s_tot[NPART];
    __shared__ bool s_last;
    block_sum(acc, s_blk);
    if (threadIdx.x < NPART) a.partials[(long long)blockIdx.x * NPART + threadIdx.x] = s_blk[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ordered_sum(a.partials, gridDim.x, s_tot);
    if (threadIdx.x == 0) {
        Rec* r = a.rec;
        // target of the cubic: sum Q(phi^0) = 2 H0 - N (nonlinear), sum phi^0 = H0 (linear)
        const double target = P.linear ? r->H0 : 2.0 * r->H0 - P.Nd;
        const double p0 = s_tot[0] - target;
        // linear constraint: the pull adds a M_phi lambda to every node in float-float, so the
        // slope is N a M_phi exactly
        const double p1 = P.linear ? P.Nd * r->a * P.M_phi_d : s_tot[1], p2 = s_tot[2], p3 = s_tot[3];
        // |f| at the rounding level of the difference that makes p0 also counts as a root
        // (a root at lambda ~ 0 never meets the relative step test)
        const double f_tol = 1e-14 * (fabs(s_tot[0]) + fabs(target));
        double lam = r->lam;
        int it = 0;
        bool converged = !(p1 != 0.0);   // no multiplier term (M_phi = 0): nothing to solve
        for (; it < 50 && !converged; ++it) {   // Newton from the continuous estimate (bounded)
            const double f = p0 + lam * (p1 + lam * (p2 + lam * p3));
            if (fabs(f) <= f_tol) { converged = true; break; }
            const double fp = p1 + lam * (2.0 * p2 + 3.0 * lam * p3);
            if (!(fp != 0.0)) break;
            const double dl = f / fp;
            lam -= dl;
            converged = fabs(dl) <= 1e-15 * fabs(lam);
        }
        r->pad[0] = r->lam;          // the estimate the root was started from
        // iterations taken, or -1: no root found (the estimate stays)
        r->pad[1] = (converged && isfinite(lam)) ? (double)it : -1.0;
        if (converged && isfinite(lam)) r->lam = lam;
        *a.counter = 0u;
        __threadfence();
    }
}

template <class T>
cudaError_t launch_exact_t(slbm_domain* d) {
    ExactArgs<T> a;
    // state after the step just launched: the buffers it wrote
    const int o = d->cur ^ 1;
    a.nx = d->p.nx; a.ny = d->p.ny; a.N = d->N;
    a.gd = (const T*)d->gd[o]; a.gm = d->gm[o]; a.php = d->php[o];
    a.partials = d->partials;
    a.counter = d->counter;
    a.rec = d->recs + (d->n & 1);
    a.P = d->phys;
    // the partials buffer was sized for max(step grid, this grid) at creation
    exact_multiplier_kernel<T><<<d->exact_blocks, EX_THREADS, 0, d->stream>>>(a);
    return cudaGetLastError();
}

template <class T>
int exact_blocks_t(long long N) {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, exact_multiplier_kernel<T>, EX_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long need = (N + EX_THREADS - 1) / EX_THREADS;   // about the number of tiles
    const long long slots = (long long)sms * per_sm;
    return (int)(need < slots ? (need > 0 ? need : 1) : slots);
}

}  // namespace

// grid of the reduction pass: every resident slot (the pass is latency-bound: each cell
// gathers 16 fixed-point values from 9 nodes), at most one CTA per 256 cells
int exact_multiplier_blocks(int precision, long long N) {
    switch (precision) {
        case SLBM_FP16DEV: return exact_blocks_t<__half>(N);
        case SLBM_BF16DEV: return exact_blocks_t<__nv_bfloat16>(N);
        default: return exact_blocks_t<float>(N);
    }
}

cudaError_t launch_exact_multiplier(slbm_domain* d) {
    switch (d->p.precision) {
        case SLBM_FP16DEV: return launch_exact_t<__half>(d);
        case SLBM_BF16DEV: return launch_exact_t<__nv_bfloat16>(d);
        default: return launch_exact_t<float>(d);
    }
}
