// The fused stream-collide kernel of the coupled LBM step and its helpers.
//
// One launch advances every cell by one time step (pull scheme, Sec. 3):
//   phase 1  pull the two scalar sets on the tile plus a 2-node ring, giving
//            phi and psi exactly in float-float (fixed-point exchange);
//   phase 2  wall ghost rows (Eq. boundary) and the chemical potentials
//            mu_phi, mu_psi (Eqs. eq_muphi, eq_mupsi) on the tile plus a 1-node ring;
//   phase 3  per interior cell: force (Eq. eq_Fs0), flow pull with bounce-back walls,
//            velocity and pressure, equilibria, sources and the MRT/BGK collisions of
//            all three sets; store; FP64 block partials of the global integrals;
//   tail     the last block to finish reduces the partials in a fixed order and
//            resolves lambda_phi (Eq. eq15) and mubar_psi (Eq. AC_psi).
//
// lambda^n and mubar^n enter the step-n populations only as w_i * (scalar at the node)
// in the source w_i (R + dt/2 dR/dt); that term lands entirely on the stored zeroth
// moment, so it is applied by the next launch when it pulls (a deferred correction
// algebraically identical to applying it in this step) and no grid-wide barrier is needed.
#pragma once
#include "surflbm_device.cuh"

namespace slbm {

constexpr int TX = 32;          // tile width (cells)
constexpr int TY = 16;          // tile height
constexpr int NTHREADS = 256;   // 32 x 8 threads, two cells each
constexpr int R2X = TX + 4, R2Y = TY + 4;
constexpr int R1X = TX + 2, R1Y = TY + 2;
constexpr int NPART = 9;        // doubles per block partial

// indices of the block partials / reduced quantities
enum { P_S1 = 0, P_S2, P_S3, P_Q, P_PHI, P_PSI, P_KIN, P_CLAMP, P_RANGE };

struct Phys {
    float beta, kappa, lambda_s, W, kT, phi_b, inv_phi_b, M_phi, M_psi, M_0, eta_phi, eta_psi;
    float rho_l, rho_g, nu_l, nu_g, Gx, Gy;
    float sf[5], sg[5], sh[5];   // (s0, s1, s2, s3, s4) per set; s2 of the flow set = 1/tau_f
    int mrt_f, mrt_g, mrt_h;      // 0: all rates equal (BGK path)
    int var_nu;                   // nu_l != nu_g
    float wcos[2], wA[2], wB[2], uw[2];
    float psi_clamp;
    int psi_on, linear, target;
    double Nd;                    // number of cells
    double M_phi_d, M_psi_d;
};

// reduced record of one time level (written by the last block)
struct Rec {
    double lam, mpsi_mubar, a, S1, S2, S3, Q, H, phi_tot, psi_tot, kin, clamps, range, H0;
    double pad[2];
};

template <class T>
struct StepArgs {
    int nx, ny;
    long long N;
    // state in (post-collision of the previous step) and out
    const T* f_in; const T* gd_in; const float2* gm_in; const T* hd_in; const float2* hm_in; const float* php_in;
    T* f_out; T* gd_out; float2* gm_out; T* hd_out; float2* hm_out; float* php_out;
    T* hist;                      // 6 planes, updated in place
    double* partials;             // [gridDim][NPART]
    unsigned int* counter;
    const Rec* rec_prev;          // time level n-1 (zeros before the first step)
    Rec* rec_out;                 // time level n
    int first;                    // this is the first step after initialisation
    // DIAG outputs (device, double)
    double* o_phi; double* o_psi; double* o_ux; double* o_uy; double* o_p;
    Phys P;
};

__device__ __forceinline__ int wrapx(int x, int nx) {
    x %= nx;
    return x < 0 ? x + nx : x;
}

// h_phi'(phi) = g'(phi) = 3/(4 phi_b) (1 - phi^2/phi_b^2), or 1 for the linear constraint
__device__ __forceinline__ float hprime(float phi, const Phys& P) {
    if (P.linear) return 1.0f;
    float u = phi * P.inv_phi_b;
    return 0.75f * P.inv_phi_b * (1.0f - u * u);
}

// fixed-point value of the population leaving `node` in direction k:
// v = d_k(node) + w_k * hi(m~(node)), converted once with round-to-nearest
__device__ __forceinline__ int kval(float d, float w, float mh, float scale, int& range) {
    float v = __fadd_rn(d, __fmul_rn(w, mh));
    float sv = __fmul_rn(v, scale);
    range |= !(fabsf(sv) < 2147483000.0f);
    return __float2int_rn(sv);
}

// m~ = m + correction of the deferred multiplier term of the previous step
template <bool PHISET>
__device__ __forceinline__ ff mtilde(const float2* __restrict__ m, const float* __restrict__ php, long long c,
                                     float qcoef, ff cuni, const Phys& P) {
    float2 mv = __ldg(m + c);
    ff r = {mv.x, mv.y};
    if (PHISET) {
        if (qcoef != 0.0f) r = ff_add_f(r, __fmul_rn(qcoef, hprime(__ldg(php + c), P)));
    } else {
        r = ff_add(r, cuni);
    }
    return r;
}

// Pull one scalar set at (x, y): returns the zeroth moment exactly (float-float) and,
// if Kin != nullptr, the eight received fixed-point populations.  Walls: specular.
template <class T, bool PHISET>
__device__ __forceinline__ ff pull_scalar(const T* __restrict__ d, const float2* __restrict__ m,
                                          const float* __restrict__ php, int x, int y, int nx, int ny,
                                          long long N, float qcoef, ff cuni, const Phys& P, int* Kin,
                                          int& range) {
    const float scale = PHISET ? (float)(1u << SFIX_PHI) : 2147483648.0f;
    const float inv_scale = 1.0f / scale;
    const long long c = (long long)y * nx + x;
    ff mself = mtilde<PHISET>(m, php, c, qcoef, cuni, P);
    int ksum = 0;
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        ksum -= kval(Stor<T>::ld(d, (long long)(k - 1) * N + c), Wk(k), mself.hi, scale, range);
        int sy = y - CYk(k);
        int sx = wrapx(x - CXk(k), nx);
        int kk = k;
        if (sy < 0 || sy >= ny) { sy = y; kk = MIRYk(k); }
        long long sc = (long long)sy * nx + sx;
        ff ms = mtilde<PHISET>(m, php, sc, qcoef, cuni, P);
        int kin = kval(Stor<T>::ld(d, (long long)(kk - 1) * N + sc), Wk(kk), ms.hi, scale, range);
        ksum += kin;
        if (Kin) Kin[k] = kin;
    }
    return ff_add(mself, fixed_to_ff(ksum, inv_scale));
}

// wetting / adsorption ghost values (Eq. boundary, reading c2): phi_G = phi_w - (df_w/dphi)/kappa,
// psi_G = psi_w - (df_w/dpsi)/lambda_s, derivatives evaluated at the wall-row values
__device__ __forceinline__ void wall_ghost(float ph, float ps, int w, const Phys& P, float& phG, float& psG) {
    float psc = P.psi_on ? fminf(fmaxf(ps, P.psi_clamp), 1.0f - P.psi_clamp) : 0.0f;
    float L = P.psi_on ? log1pf(-psc) : 0.0f;
    float u = ph * P.inv_phi_b;
    float gp = 0.75f * P.inv_phi_b * (1.0f - u * u);
    float gv = 0.75f * u - 0.25f * u * u * u;
    float dfdphi = -(P.wcos[w] + L * P.wA[w]) * gp;
    float dfdpsi = (P.wA[w] * gv - 0.5f * P.wB[w]) / (1.0f - psc);
    phG = P.kappa > 0.0f ? ph - dfdphi / P.kappa : ph;
    psG = (P.lambda_s > 0.0f && P.psi_on) ? ps - dfdpsi / P.lambda_s : ps;
}

// warp reduction of a float-float pair
__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, w);
    }
    return v;
}

// Block reduction of NPART float-float accumulators into partials[blockIdx], then the
// last block reduces all partials in fixed order and resolves the multipliers.
template <class T>
__device__ void finish_reduction(ff (&acc)[NPART], const StepArgs<T>& A, bool diag) {
    __shared__ double s_w[NPART][NTHREADS / 32];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
        ff v = warp_sum_ff(acc[q]);
        if (lane == 0) s_w[q][warp] = ff_to_d(v);
    }
    __syncthreads();
    const int nblocks = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x < NPART) {
        double s = 0.0;
        for (int w = 0; w < NTHREADS / 32; ++w) s += s_w[threadIdx.x][w];
        A.partials[(long long)bid * NPART + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(A.counter, 1u);
        s_last = (prev == (unsigned)(nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // fixed-order reduction: warp q sums quantity q (and q + 8), lanes stride the blocks
    __shared__ double s_tot[NPART];
    for (int q = warp; q < NPART; q += NTHREADS / 32) {
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32) s += ((volatile double*)A.partials)[(long long)b * NPART + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) s_tot[q] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const Phys& P = A.P;
        Rec r = {};
        r.S1 = s_tot[P_S1];
        r.S2 = s_tot[P_S2];
        r.S3 = s_tot[P_S3];
        r.Q = s_tot[P_Q];
        r.phi_tot = s_tot[P_PHI];
        r.psi_tot = s_tot[P_PSI];
        r.kin = s_tot[P_KIN];
        r.clamps = s_tot[P_CLAMP];
        r.range = s_tot[P_RANGE];
        r.H = P.linear ? r.phi_tot : 0.5 * P.Nd + 0.5 * r.Q;
        r.H0 = A.first ? r.H : A.rec_prev->H0;
        double lam = 0.0;
        if (r.S2 > 0.0) {
            lam = r.S1 / r.S2;
            if (P.target && P.M_phi_d > 0.0) lam = (r.S1 + (r.H0 - r.H) / P.M_phi_d) / r.S2;
        }
        r.lam = lam;
        r.mpsi_mubar = P.psi_on ? -r.S3 / P.Nd : 0.0;
        r.a = diag ? 0.0 : (A.first ? 1.0 : 1.5);
        *A.rec_out = r;
        *A.counter = 0u;
        __threadfence();
    }
}

// ------------------------------------------------------------------- the step
// DIAG = true: same moments / forces / velocity / pressure, no collision, writes the
// macroscopic fields and the reduced totals of the current time level.
template <class T, bool DIAG>
__global__ void __launch_bounds__(NTHREADS) step_kernel(const StepArgs<T> A) {
    const Phys& P = A.P;
    const int nx = A.nx, ny = A.ny;
    const long long N = A.N;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x;

    __shared__ float s_ph[R2Y][R2X], s_pl[R2Y][R2X], s_sh[R2Y][R2X], s_sl[R2Y][R2X];
    __shared__ float s_mu[R1Y][R1X], s_mp[R1Y][R1X];
    __shared__ float s_gphi[2][R2X], s_gpsi[2][R2X];

    // deferred multiplier terms of time level n-1
    const Rec rp = *A.rec_prev;
    const float qcoef = (float)(rp.a * P.M_phi_d * rp.lam);
    const double cu_d = rp.a * rp.mpsi_mubar;
    ff cuni;
    cuni.hi = (float)cu_d;
    cuni.lo = (float)(cu_d - (double)cuni.hi);
    int range = 0;

    // ---------------- phase 1: phi, psi on the tile + 2-ring
    for (int idx = tid; idx < R2X * R2Y; idx += NTHREADS) {
        const int lx = idx % R2X, ly = idx / R2X;
        const int gy = y0 - 2 + ly;
        if (gy < 0 || gy >= ny) continue;
        const int gx = wrapx(x0 - 2 + lx, nx);
        ff ph = pull_scalar<T, true>(A.gd_in, A.gm_in, A.php_in, gx, gy, nx, ny, N, qcoef, cuni, P, nullptr, range);
        s_ph[ly][lx] = ph.hi;
        s_pl[ly][lx] = ph.lo;
        if (P.psi_on) {
            ff ps = pull_scalar<T, false>(A.hd_in, A.hm_in, A.php_in, gx, gy, nx, ny, N, 0.0f, cuni, P, nullptr, range);
            s_sh[ly][lx] = ps.hi;
            s_sl[ly][lx] = ps.lo;
        } else {
            s_sh[ly][lx] = 0.0f;
            s_sl[ly][lx] = 0.0f;
        }
    }
    __syncthreads();

    // ---------------- phase 2a: ghost rows beyond the walls
    const int lyb = 2 - y0;            // local row of grid row 0
    const int lyt = ny - 1 - y0 + 2;   // local row of grid row ny-1
    for (int lx = tid; lx < R2X; lx += NTHREADS) {
        if (lyb >= 0 && lyb < R2Y) wall_ghost(s_ph[lyb][lx], s_sh[lyb][lx], 0, P, s_gphi[0][lx], s_gpsi[0][lx]);
        if (lyt >= 0 && lyt < R2Y) wall_ghost(s_ph[lyt][lx], s_sh[lyt][lx], 1, P, s_gphi[1][lx], s_gpsi[1][lx]);
    }
    __syncthreads();

    // ---------------- phase 2b: chemical potentials on the tile + 1-ring
    float clamps = 0.0f;
    for (int idx = tid; idx < R1X * R1Y; idx += NTHREADS) {
        const int l1x = idx % R1X, l1y = idx / R1X;
        const int lx = l1x + 1, ly = l1y + 1;
        const int gy = y0 - 1 + l1y;
        if (gy < 0 || gy >= ny) continue;
        const float phi = s_ph[ly][lx], psi = s_sh[ly][lx];
        float lapG_phi = 0.0f, lapG_psi = 0.0f;
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            const int ny_ = gy + CYk(k);
            float vphi, vpsi;
            if (ny_ < 0) { vphi = s_gphi[0][lx + CXk(k)]; vpsi = s_gpsi[0][lx + CXk(k)]; }
            else if (ny_ >= ny) { vphi = s_gphi[1][lx + CXk(k)]; vpsi = s_gpsi[1][lx + CXk(k)]; }
            else { vphi = s_ph[ly + CYk(k)][lx + CXk(k)]; vpsi = s_sh[ly + CYk(k)][lx + CXk(k)]; }
            lapG_phi += Wk(k) * (vphi - phi);
            lapG_psi += Wk(k) * (vpsi - psi);
        }
        lapG_phi *= 6.0f;
        lapG_psi *= 6.0f;
        s_mu[l1y][l1x] = 4.0f * P.beta * (1.0f - psi) * (phi * phi * phi - phi) - P.kappa * lapG_phi + P.W * psi * phi;
        if (P.psi_on) {
            float psc = fminf(fmaxf(psi, P.psi_clamp), 1.0f - P.psi_clamp);
            float om = 1.0f - phi * phi;
            s_mp[l1y][l1x] = P.kT * logf(psc / (1.0f - psc)) - P.lambda_s * lapG_psi - P.beta * om * om +
                             0.5f * P.W * phi * phi;
        } else {
            s_mp[l1y][l1x] = 0.0f;
        }
    }
    __syncthreads();

    // ---------------- phase 3: interior cells
    ff acc[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) acc[q] = {0.0f, 0.0f};

    const int tx = tid & 31, tyb = tid >> 5;
#pragma unroll 1
    for (int sub = 0; sub < 2; ++sub) {
        const int ty = tyb + 8 * sub;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= nx || gy >= ny) continue;
        const long long c = (long long)gy * nx + gx;
        const int lx = tx + 2, ly = ty + 2, l1x = tx + 1, l1y = ty + 1;
        const ff phff = {s_ph[ly][lx], s_pl[ly][lx]};
        const ff psff = {s_sh[ly][lx], s_sl[ly][lx]};
        const float phi = phff.hi, psi = psff.hi;

        // gradients (mirror ghosts for mu and rho), Neumann Laplacians and wall flux
        float gmx = 0.f, gmy = 0.f, gpx = 0.f, gpy = 0.f, grx = 0.f, gry = 0.f;
        float lapN_phi = 0.f, lapN_psi = 0.f, wf_phi = 0.f, wf_psi = 0.f;
        const float drho = (P.rho_l - P.rho_g) * 0.5f * P.inv_phi_b;
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            const int cx = CXk(k), cy = CYk(k);
            const int ny_ = gy + cy;
            const bool out = (ny_ < 0 || ny_ >= ny);
            const int oy = out ? 0 : cy;   // mirror: same row
            const float mu = s_mu[l1y + oy][l1x + cx];
            const float mp = s_mp[l1y + oy][l1x + cx];
            const float vphi = s_ph[ly + oy][lx + cx];
            const float vpsi = s_sh[ly + oy][lx + cx];
            const float w3 = 3.0f * Wk(k);
            gmx += w3 * cx * mu; gmy += w3 * cy * mu;
            gpx += w3 * cx * mp; gpy += w3 * cy * mp;
            grx += w3 * cx * vphi; gry += w3 * cy * vphi;
            lapN_phi += Wk(k) * (vphi - phi);
            lapN_psi += Wk(k) * (vpsi - psi);
            if (out) {
                const int w = ny_ < 0 ? 0 : 1;
                wf_phi += Wk(k) * (s_gphi[w][lx + cx] - vphi);
                wf_psi += Wk(k) * (s_gpsi[w][lx + cx] - vpsi);
            }
        }
        grx *= drho; gry *= drho;
        lapN_phi *= 6.0f; lapN_psi *= 6.0f; wf_phi *= 6.0f; wf_psi *= 6.0f;
        const float Fx = -phi * gmx - psi * gpx + P.Gx;
        const float Fy = -phi * gmy - psi * gpy + P.Gy;
        const float chi = 0.5f * (phi * P.inv_phi_b + 1.0f);
        const float rho = P.rho_g + (P.rho_l - P.rho_g) * chi;

        // flow pull with halfway bounce-back and the moving-wall term
        float f[9];
        const float php_self = __ldg(A.php_in + c);
        const float rho_w = P.rho_g + (P.rho_l - P.rho_g) * 0.5f * (php_self * P.inv_phi_b + 1.0f);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int sy = gy - CYk(k);
            if (sy < 0 || sy >= ny) {
                const int o = OPPk(k);
                const int w = sy < 0 ? 0 : 1;
                f[k] = Stor<T>::ld(A.f_in, (long long)o * N + c) - 6.0f * Wk(o) * rho_w * CXk(o) * P.uw[w];
            } else {
                const int sx = wrapx(gx - CXk(k), nx);
                f[k] = Stor<T>::ld(A.f_in, (long long)k * N + (long long)sy * nx + sx);
            }
        }
        float jx = 0.f, jy = 0.f, fsum = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            jx += CXk(k) * f[k];
            jy += CYk(k) * f[k];
            if (k) fsum += f[k];
        }
        const float inv_rho = 1.0f / rho;
        const float ux = (jx + 0.5f * Fx) * inv_rho;
        const float uy = (jy + 0.5f * Fy) * inv_rho;
        const float usq = ux * ux + uy * uy;
        const float ugr = ux * grx + uy * gry;
        const float pres = (1.0f / 3.0f) / (1.0f - Wk(0)) * (fsum + 0.5f * ugr - rho * Wk(0) * usq * 1.5f);

        const float hp = hprime(phi, P);
        float mu_self = s_mu[l1y][l1x];
        if (P.psi_on) clamps += (psi < P.psi_clamp || psi > 1.0f - P.psi_clamp) ? 1.0f : 0.0f;

        // accumulate the global integrals at this time level
        acc[P_S1] = ff_add_f(acc[P_S1], hp * mu_self);
        acc[P_S2] = ff_add_f(acc[P_S2], hp * hp);
        {
            const float u = phi * P.inv_phi_b;
            acc[P_Q] = ff_add_f(acc[P_Q], 1.5f * u - 0.5f * u * u * u);
        }
        acc[P_PHI] = ff_add(acc[P_PHI], phff);
        acc[P_PSI] = ff_add(acc[P_PSI], psff);
        acc[P_KIN] = ff_add_f(acc[P_KIN], 0.5f * rho * usq);
        range |= !(fabsf(ux) < 1.0f && fabsf(uy) < 1.0f && fabsf(phi) < 2.0f && fabsf(pres) < 1e3f);

        if (DIAG) {
            if (A.o_phi) {
                A.o_phi[c] = ff_to_d(phff);
                A.o_psi[c] = ff_to_d(psff);
                A.o_ux[c] = (double)ux;
                A.o_uy[c] = (double)uy;
                A.o_p[c] = (double)pres;
            }
            // S3 of the diagnostic level: the free reaction term as the next step would form it
            if (P.psi_on) {
                float psc = fminf(fmaxf(psi, P.psi_clamp), 1.0f - P.psi_clamp);
                float om = 1.0f - phi * phi;
                float Rf = P.M_psi * (-P.kT * logf(psc / (1.0f - psc)) + P.beta * om * om - 0.5f * P.W * phi * phi +
                                      P.lambda_s * wf_psi) - P.M_0 * lapN_psi;
                acc[P_S3] = ff_add_f(acc[P_S3], Stor<T>::rnd(Rf));
            }
            continue;
        }

        // ---- flow collision (Sec. 3): f^eq, source F_{i,1}
        {
            float feq[9], src[9];
            const float p3 = 3.0f * pres;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float cu = CXk(k) * ux + CYk(k) * uy;
                const float cF = CXk(k) * Fx + CYk(k) * Fy;
                const float cg = CXk(k) * grx + CYk(k) * gry;
                feq[k] = p3 * (Wk(k) - (k == 0 ? 1.0f : 0.0f)) + rho * Wk(k) * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq);
                src[k] = Wk(k) * (ugr + 3.0f * cF + 3.0f * (cu * cg - (1.0f / 3.0f) * ugr));
            }
            float s2 = P.sf[2];
            if (P.var_nu) {
                const float nu = P.nu_g + (P.nu_l - P.nu_g) * chi;
                s2 = 1.0f / (3.0f * nu + 0.5f);
            }
            if (P.mrt_f) {
                float s[9];
                s[0] = P.sf[0] > 0.f ? P.sf[0] : s2;
                s[1] = s[2] = P.sf[1] > 0.f ? P.sf[1] : s2;
                s[3] = s[4] = s[5] = s2;
                s[6] = s[7] = P.sf[3] > 0.f ? P.sf[3] : s2;
                s[8] = P.sf[4] > 0.f ? P.sf[4] : s2;
                mrt_collide(f, feq, src, s);
            } else {
                const float a = 1.0f - 0.5f * s2;
#pragma unroll
                for (int k = 0; k < 9; ++k) f[k] = f[k] - s2 * (f[k] - feq[k]) + a * src[k];
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) Stor<T>::st(A.f_out, (long long)k * N + c, f[k]);
        }

        // ---- history of the source terms (Sec. 3, backward differences)
        const float phux = phi * ux, phuy = phi * uy, psux = psi * ux, psuy = psi * uy;
        float dphux = 0.f, dphuy = 0.f, dpsux = 0.f, dpsuy = 0.f, Rp_phi = 0.f, Rp_psi = 0.f;
        if (!A.first) {
            Rp_phi = Stor<T>::ld(A.hist, 0 * N + c);
            Rp_psi = Stor<T>::ld(A.hist, 1 * N + c);
            dphux = phux - Stor<T>::ld(A.hist, 2 * N + c);
            dphuy = phuy - Stor<T>::ld(A.hist, 3 * N + c);
            dpsux = psux - Stor<T>::ld(A.hist, 4 * N + c);
            dpsuy = psuy - Stor<T>::ld(A.hist, 5 * N + c);
        }

        // ---- phase-field set
        {
            // R_phi without the lambda^n term (deferred), with the wall flux of reading c2
            const float Rf = Stor<T>::rnd(P.M_phi * (-4.0f * P.beta * (1.0f - psi) * (phi * phi * phi - phi) -
                                                     P.W * psi * phi + P.kappa * wf_phi));
            // dR = R + (R - R_prev)/2, exact in float-float; minus the lambda^{n-1} part of R_prev
            ff dR;
            if (A.first) {
                dR = {Rf, 0.0f};
            } else {
                ff t = two_sum(Rf, -Rp_phi);
                dR = ff_add_f(ff_scale_pow2(t, 0.5f), Rf);
                const float lam_part = (float)(0.5 * P.M_phi_d * rp.lam) * hprime(php_self, P);
                dR = ff_add_f(dR, -lam_part);
            }
            const float dRf = dR.hi + dR.lo;
            int Kin[9];
            int rdummy = 0;
            (void)pull_scalar<T, true>(A.gd_in, A.gm_in, A.php_in, gx, gy, nx, ny, N, qcoef, cuni, P, Kin, rdummy);
            const float inv_scale = 1.0f / (float)(1u << SFIX_PHI);
            float g[9];
            float gs = 0.f;
#pragma unroll
            for (int k = 1; k < 9; ++k) { g[k] = (float)Kin[k] * inv_scale; gs += g[k]; }
            g[0] = phi - gs;
            float geq[9], src[9];
            const float a3x = 3.0f * dphux, a3y = 3.0f * dphuy;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                geq[k] = Wk(k) * P.eta_phi * phi + (k == 0 ? (1.0f - P.eta_phi) * phi : 0.0f) +
                         Wk(k) * 3.0f * (CXk(k) * phux + CYk(k) * phuy);
                src[k] = Wk(k) * (CXk(k) * a3x + CYk(k) * a3y);
            }
            if (P.mrt_g) {
                float s[9];
                const float s1 = P.sg[1];
                s[0] = P.sg[0] > 0.f ? P.sg[0] : s1;
                s[1] = s[2] = s1;
                s[3] = s[4] = s[5] = P.sg[2] > 0.f ? P.sg[2] : s1;
                s[6] = s[7] = P.sg[3] > 0.f ? P.sg[3] : s1;
                s[8] = P.sg[4] > 0.f ? P.sg[4] : s1;
                mrt_collide(g, geq, src, s);
            } else {
                const float s1 = P.sg[1], a = 1.0f - 0.5f * s1;
#pragma unroll
                for (int k = 0; k < 9; ++k) g[k] = g[k] - s1 * (g[k] - geq[k]) + a * src[k];
            }
            const ff mstar = ff_add(phff, dR);
            float2 mo;
            mo.x = mstar.hi;
            mo.y = mstar.lo;
            A.gm_out[c] = mo;
#pragma unroll
            for (int k = 1; k < 9; ++k)
                Stor<T>::st(A.gd_out, (long long)(k - 1) * N + c, g[k] + Wk(k) * dRf - Wk(k) * mstar.hi);
            A.php_out[c] = phi;
            Stor<T>::st(A.hist, 0 * N + c, Rf);
            Stor<T>::st(A.hist, 2 * N + c, phux);
            Stor<T>::st(A.hist, 3 * N + c, phuy);
        }

        // ---- surfactant set
        if (P.psi_on) {
            const float psc = fminf(fmaxf(psi, P.psi_clamp), 1.0f - P.psi_clamp);
            const float om = 1.0f - phi * phi;
            const float Rf = Stor<T>::rnd(P.M_psi * (-P.kT * logf(psc / (1.0f - psc)) + P.beta * om * om -
                                                     0.5f * P.W * phi * phi + P.lambda_s * wf_psi) -
                                          P.M_0 * lapN_psi);
            acc[P_S3] = ff_add_f(acc[P_S3], Rf);
            ff dR;
            if (A.first) {
                dR = {Rf, 0.0f};
            } else {
                ff t = two_sum(Rf, -Rp_psi);
                dR = ff_add_f(ff_scale_pow2(t, 0.5f), Rf);
                const double hm = -0.5 * rp.mpsi_mubar;
                ff hmf;
                hmf.hi = (float)hm;
                hmf.lo = (float)(hm - (double)hmf.hi);
                dR = ff_add(dR, hmf);
            }
            const float dRf = dR.hi + dR.lo;
            int Kin[9];
            int rdummy = 0;
            (void)pull_scalar<T, false>(A.hd_in, A.hm_in, A.php_in, gx, gy, nx, ny, N, 0.0f, cuni, P, Kin, rdummy);
            const float inv_scale = 1.0f / 2147483648.0f;
            float h[9];
            float hs = 0.f;
#pragma unroll
            for (int k = 1; k < 9; ++k) { h[k] = (float)Kin[k] * inv_scale; hs += h[k]; }
            h[0] = psi - hs;
            float heq[9], src[9];
            const float a3x = 3.0f * dpsux, a3y = 3.0f * dpsuy;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                heq[k] = Wk(k) * P.eta_psi * psi + (k == 0 ? (1.0f - P.eta_psi) * psi : 0.0f) +
                         Wk(k) * 3.0f * (CXk(k) * psux + CYk(k) * psuy);
                src[k] = Wk(k) * (CXk(k) * a3x + CYk(k) * a3y);
            }
            if (P.mrt_h) {
                float s[9];
                const float s1 = P.sh[1];
                s[0] = P.sh[0] > 0.f ? P.sh[0] : s1;
                s[1] = s[2] = s1;
                s[3] = s[4] = s[5] = P.sh[2] > 0.f ? P.sh[2] : s1;
                s[6] = s[7] = P.sh[3] > 0.f ? P.sh[3] : s1;
                s[8] = P.sh[4] > 0.f ? P.sh[4] : s1;
                mrt_collide(h, heq, src, s);
            } else {
                const float s1 = P.sh[1], a = 1.0f - 0.5f * s1;
#pragma unroll
                for (int k = 0; k < 9; ++k) h[k] = h[k] - s1 * (h[k] - heq[k]) + a * src[k];
            }
            const ff mstar = ff_add(psff, dR);
            float2 mo;
            mo.x = mstar.hi;
            mo.y = mstar.lo;
            A.hm_out[c] = mo;
#pragma unroll
            for (int k = 1; k < 9; ++k)
                Stor<T>::st(A.hd_out, (long long)(k - 1) * N + c, h[k] + Wk(k) * dRf - Wk(k) * mstar.hi);
            Stor<T>::st(A.hist, 1 * N + c, Rf);
            Stor<T>::st(A.hist, 4 * N + c, psux);
            Stor<T>::st(A.hist, 5 * N + c, psuy);
        }
    }
    acc[P_CLAMP] = {clamps, 0.0f};
    acc[P_RANGE] = {(float)range, 0.0f};
    finish_reduction<T>(acc, A, DIAG);
}

}  // namespace slbm
