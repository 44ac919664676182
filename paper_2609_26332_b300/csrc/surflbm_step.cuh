// The fused stream-collide kernel of the coupled LBM step and its helpers.
//
// Each CTA owns a strip of TX columns and a segment of rows (pieces of bands of rows,
// neighbouring strips marched together), and marches up the segment RB rows at a time
// through a software pipeline kept in shared-memory rings (12 rows for the fixed-point
// populations and m~, 8 for phi / psi and mu):
//   stage K    for every source node of the rows seven ahead, the eight populations it
//              sends, converted once to 32-bit fixed point (both scalar sets), in the same
//              barrier interval as stage PHI (disjoint rows);
//   stage PHI  pull: phi, psi of the rows two ahead, exactly, as float-float
//              (m~ + received - sent, an integer sum that telescopes over the grid);
//   stage MU   chemical potentials mu_phi, mu_psi (Eqs. eq_muphi, eq_mupsi) one row ahead,
//              with the wall ghost rows of Eq. boundary;
//   stage COLLIDE  per cell: force (Eq. eq_Fs0), flow pull with bounce-back walls, u, p,
//              equilibria, sources and the MRT/BGK collisions of the three sets (Sec. 3),
//              stores, and the FP64-reduced global integrals.
// The last CTA to finish reduces the block partials in a fixed order and resolves
// lambda_phi (Eq. eq15) and mubar_psi (Eq. AC_psi).
//
// lambda^n and mubar^n enter the step-n populations only as w_i * (scalar at the node)
// in the source w_i (R + dt/2 dR/dt); that term lands entirely on the stored zeroth
// moment, so the next launch applies it when it pulls (a deferred correction,
// algebraically identical to applying it in this step) and no grid-wide barrier is needed.
#pragma once
#include <cuda.h>   // CUtensorMap (type only; maps are encoded through the runtime's driver entry point)
#include <type_traits>
#include "surflbm_device.cuh"

namespace slbm {

constexpr int NPART = 13;        // doubles per block partial

// tensor maps of one side of the ping-pong state (kernel parameter, __grid_constant__)
struct TmaMaps {   // CUtensorMap is 64-byte aligned
    CUtensorMap dev[2];   // deviation planes of phi, psi: [8][ny][nx], box {WW, RB, 8}
    CUtensorMap mom[2];   // zeroth moments: float2 [ny][nx] as 32-bit [ny][2 nx], box {2 WW, RB}
    CUtensorMap php;      // previous phi [ny][nx], box {WW, RB}
    CUtensorMap f;        // flow populations [9][ny][nx], box {WW, RB, 1}
};

// bound of every mbarrier wait of the step (global-timer nanoseconds)
constexpr unsigned long long TMA_WAIT_NS = 2000000000ull;
// bits of the step's error word
constexpr unsigned int ERR_TMA_WAIT = 1u;

// indices of the block partials / reduced quantities
enum { P_S1 = 0, P_S2, P_S3, P_Q, P_PHI, P_PSI, P_KIN, P_CLAMP, P_RANGE, P_EF, P_DPHI2, P_PHI2, P_SR };

struct Phys {
    float beta, kappa, lambda_s, W, kT, phi_b, inv_phi_b, M_phi, M_psi, M_0, eta_phi, eta_psi;
    float rho_l, rho_g, nu_l, nu_g, Gx, Gy;
    float sf[5], sg[5], sh[5];   // (s0, s1, s2, s3, s4) per set; s2 of the flow set = 1/tau_f
    int mrt_f, mrt_g, mrt_h;      // 0: all rates equal (BGK path)
    int var_nu;                   // nu_l != nu_g
    float wcos[2], uw[2];
    // per wall: sigma_sg,0 beta_sg, sigma_sl,0 beta_sl, sigma_sg,0, sigma_sl,0 and the
    // ln(1 - psi) below which each tension sits on its Remark-1 cap (-1e30: never)
    float wSg[2], wSl[2], wS0g[2], wS0l[2], wLg[2], wLl[2];
    float psi_clamp;
    int psi_on, linear, target;
    // manufactured-solution test (MMS kernels only): physical amplitude, advection speed,
    // mobility, beta, kappa, k_B T, W, node spacing and time step
    float mms_a, mms_u, mms_M, mms_beta, mms_kappa, mms_kT, mms_W, mms_dx, mms_dt;
    double Nd;                    // number of cells
    double M_phi_d, M_psi_d;
};

// reduced record of one time level (written by the last block)
struct Rec {
    double lam, mpsi_mubar, a, S1, S2, S3, Q, H, phi_tot, psi_tot, kin, clamps, range, H0;
    double ef;              // discrete free energy (diagnostic level only)
    double dphi2, phi2;     // sum (phi^n - phi^{n-1})^2 and sum (phi^n)^2 (diagnostic level only)
    double pad[3];
};

template <class T>
struct StepArgs {
    int nx, ny;
    long long N;
    long long total;              // strips * ny: the strip-major rows shared out among the CTAs
    int band_h;                   // > 0: band-major pieces of band_h rows (see the split below)
    // state in (post-collision of the previous step) and out
    const T* f_in; const T* gd_in; const float2* gm_in; const T* hd_in; const float2* hm_in; const float* php_in;
    T* f_out; T* gd_out; float2* gm_out; T* hd_out; float2* hm_out; float* php_out;
    T* hist;                      // 6 planes, updated in place
    double* partials;             // [gridDim][NPART]
    unsigned int* counter;
    unsigned int* err;            // error bits (ERR_*), or null
    const Rec* rec_prev;          // time level n-1 (zeros before the first step)
    Rec* rec_out;                 // time level n
    int first;                    // this is the first step after initialisation
    long long level;              // time level of the populations the launch collides
    // DIAG outputs (device, double; may be null)
    double* o_phi; double* o_psi; double* o_ux; double* o_uy; double* o_p;
    Phys P;
};

// One instance of a batch (device memory, read-only during a launch).
struct InstDesc {
    const void* f[2]; const void* gd[2]; const void* hd[2];      // ping-pong population buffers
    const float2* gm[2]; const float2* hm[2]; const float* php[2];
    void* hist;
    Rec* recs;                 // [0], [1]: ring by step parity; [2]: diagnostic; [3]: zeros
    double* partials;          // npieces * NPART partial sums of the current launch
    unsigned int* counter;     // pieces of this instance finished in the current launch
    int nx, ny, npieces, pad;
    long long N;
    long long G0;              // batch step counter at this instance's time level 0
    Phys P;
};
// One piece of the batch tile queue: rows [y0, y1) of strip `strip` of instance `inst`;
// `slot` is the piece's index among its instance's pieces.
struct Piece {
    int inst, strip, y0, y1, slot, pad0, pad1, pad2;
};
struct BatchArgs {
    const InstDesc* inst;
    const Piece* pieces;
    int npieces;
    unsigned int* queue;       // next piece (reset by the last CTA of each launch)
    unsigned int* done;        // CTAs finished in this launch
    long long* G;              // batch step counter, advanced by the last CTA of each launch
};

__device__ __forceinline__ int wrapx(int x, int nx) {
    x %= nx;
    return x < 0 ? x + nx : x;
}
// x within [-nx, 2nx): one conditional correction
__device__ __forceinline__ int wrap1(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for the phase of the given parity; false after TMA_WAIT_NS
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > TMA_WAIT_NS) return false;
    }
}
// generic-proxy shared-memory accesses ordered before later async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// y component of c_k for a runtime k
__device__ __forceinline__ int CYk_rt(int k) { return (k == 2 || k == 5 || k == 6) ? 1 : ((k == 4 || k == 7 || k == 8) ? -1 : 0); }

// c_k . (ax, ay) with the zero lattice components folded away at compile time (IEEE
// arithmetic may not drop 0 * x, so the generic form would pay for every zero)
__device__ __forceinline__ float cdot(int k, float ax, float ay) {
    const int cx = CXk(k), cy = CYk(k);
    if (cx == 0 && cy == 0) return 0.0f;
    if (cy == 0) return cx > 0 ? ax : -ax;
    if (cx == 0) return cy > 0 ? ay : -ay;
    const float t = cx > 0 ? ax : -ax;
    return cy > 0 ? t + ay : t - ay;
}
// acc + sgn * v for a compile-time integer sign in {-1, 0, 1}
__device__ __forceinline__ float addc(float acc, int sgn, float v) {
    return sgn == 0 ? acc : (sgn > 0 ? acc + v : acc - v);
}

// h_phi'(phi) = g'(phi) = 3/(4 phi_b) (1 - phi^2/phi_b^2), or 1 for the linear constraint
// liquid fraction of the density / viscosity interpolation, clipped to [0, 1] (the bulk
// |phi| exceeds phi_b(psi_b) where the bulk surfactant is below psi_b)
__device__ __forceinline__ float liquid_fraction(float phi, const Phys& P) {
    return fminf(fmaxf(0.5f * (phi * P.inv_phi_b + 1.0f), 0.0f), 1.0f);
}

__device__ __forceinline__ float hprime(float phi, const Phys& P) {
    if (P.linear) return 1.0f;
    float u = __fmul_rn(phi, P.inv_phi_b);
    return __fmul_rn(__fmul_rn(0.75f, P.inv_phi_b), __fsub_rn(1.0f, __fmul_rn(u, u)));
}

// wetting / adsorption ghost values (Eq. boundary, closed by ghost rows): phi_G = phi_w - (df_w/dphi)/kappa,
// psi_G = psi_w - (df_w/dpsi)/lambda_s, derivatives evaluated at the wall-row values
__device__ __forceinline__ void wall_ghost(float ph, float ps, int w, const Phys& P, float& phG, float& psG) {
    float psc = P.psi_on ? fminf(fmaxf(ps, P.psi_clamp), 1.0f - P.psi_clamp) : 0.0f;
    float L = P.psi_on ? log1pf(-psc) : 0.0f;
    float u = ph * P.inv_phi_b;
    float gp = 0.75f * P.inv_phi_b * (1.0f - u * u);
    float gv = 0.75f * u - 0.25f * u * u * u;
    // f_w = (1/2 - g) sigma_sg + (1/2 + g) sigma_sl, sigma_s,a = sigma_s,a,0 (1 + beta_a L)
    // (Eq. langmuir) or sigma_s,a,0 / 2 on the cap (Remark 1)
    const bool on_sg = L > P.wLg[w], on_sl = L > P.wLl[w];
    const float st_sg = on_sg ? P.wSg[w] * L : -0.5f * P.wS0g[w];
    const float st_sl = on_sl ? P.wSl[w] * L : -0.5f * P.wS0l[w];
    float dfdphi = -(P.wcos[w] + st_sg - st_sl) * gp;
    float dfdpsi = -((0.5f - gv) * (on_sg ? P.wSg[w] : 0.0f) + (0.5f + gv) * (on_sl ? P.wSl[w] : 0.0f)) /
                   (1.0f - psc);
    phG = P.kappa > 0.0f ? ph - dfdphi / P.kappa : ph;
    psG = (P.lambda_s > 0.0f && P.psi_on) ? ps - dfdpsi / P.lambda_s : ps;
}

// wall free-energy density f_w(phi, psi) of wall w (Eq. fw0 with the Langmuir-Szyszkowski
// tensions of Eq. langmuir, capped as in wall_ghost): (1/2 - g) sigma_sg + (1/2 + g) sigma_sl
__device__ __forceinline__ float wall_energy(float ph, float ps, int w, const Phys& P) {
    const float psc = P.psi_on ? fminf(fmaxf(ps, P.psi_clamp), 1.0f - P.psi_clamp) : 0.0f;
    const float L = P.psi_on ? log1pf(-psc) : 0.0f;
    const float u = ph * P.inv_phi_b;
    const float gv = 0.75f * u - 0.25f * u * u * u;
    const float st_sg = L > P.wLg[w] ? P.wSg[w] * L : -0.5f * P.wS0g[w];
    const float st_sl = L > P.wLl[w] ? P.wSl[w] * L : -0.5f * P.wS0l[w];
    return -(P.wcos[w] + st_sg - st_sl) * gv + 0.5f * (st_sg + st_sl) + 0.5f * (P.wS0g[w] + P.wS0l[w]);
}

// Manufactured sources of Sec. 4.1 on the channel (lattice units per step) at node (gx, y)
// and time level n: with X = 2 pi (x - u t), Y = 2 pi y and a = A e^{-t},
//   phi^e = a sin X cos Y,  psi^e = 1/2 + 0.05 e^{-2t} cos X cos Y
// are exact solutions of the phi and psi equations with the linear multipliers when
//   S_phi = -phi^e + M mu_phi^e                       (the mean of mu_phi^e is 0)
//   S_psi = -2 (psi^e - 1/2) + M (mu_psi^e - mean mu_psi^e),
//   mean mu_psi^e = -beta (1 - a^2/2 + 9 a^4/64) + W a^2/8   (lambda_s = 0).
__device__ __forceinline__ void mms_source(const Phys& P, long long n, int gx, int y, float& s_phi, float& s_psi) {
    const float t = (float)n * P.mms_dt;
    const float x = (float)gx * P.mms_dx, yy = ((float)y + 0.5f) * P.mms_dx;
    float sX, cX;
    sincospif(2.0f * (x - P.mms_u * t), &sX, &cX);
    const float cY = cospif(2.0f * yy);
    const float a = P.mms_a * expf(-t);
    const float pe = a * sX * cY;
    const float qe = 0.5f + 0.05f * expf(-2.0f * t) * cX * cY;
    const float lap = -8.0f * 9.8696044f * pe;   // nabla^2 of the mode: -8 pi^2 phi^e
    const float mu_phi = 4.0f * P.mms_beta * (1.0f - qe) * (pe * pe * pe - pe) + P.mms_W * qe * pe - P.mms_kappa * lap;
    const float om = 1.0f - pe * pe;
    const float mu_psi = P.mms_kT * logf(qe / (1.0f - qe)) - P.mms_beta * om * om + 0.5f * P.mms_W * pe * pe;
    const float a2 = a * a;
    const float mbar = -P.mms_beta * (1.0f - 0.5f * a2 + 9.0f / 64.0f * a2 * a2) + 0.125f * P.mms_W * a2;
    s_phi = P.mms_dt * (-pe + P.mms_M * mu_phi);
    s_psi = P.mms_dt * (-2.0f * (qe - 0.5f) + P.mms_M * (mu_psi - mbar));
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

// The time-level record from the reduced sums: lambda_phi (Eq. eq15, or the target reading),
// M_psi mubar_psi = -sum R_psi / N (Eq. AC_psi with the stored free reaction terms), H, H0.
__device__ __forceinline__ Rec resolve_rec(const Phys& P, int first, const Rec* rec_prev, const double* tot, bool diag) {
    Rec r = {};
    r.S1 = tot[P_S1];
    r.S2 = tot[P_S2];
    r.S3 = tot[P_S3];
    r.Q = tot[P_Q];
    r.phi_tot = tot[P_PHI];
    r.psi_tot = tot[P_PSI];
    r.kin = tot[P_KIN];
    r.clamps = tot[P_CLAMP];
    r.range = tot[P_RANGE];
    r.ef = tot[P_EF];
    r.dphi2 = tot[P_DPHI2];
    r.phi2 = tot[P_PHI2];
    r.H = P.linear ? r.phi_tot : 0.5 * P.Nd + 0.5 * r.Q;
    r.H0 = first ? r.H : rec_prev->H0;
    double lam = 0.0;
    if (P.linear && P.M_phi_d > 0.0) {
        // linear constraint: M_phi lambda = -(sum of the stored free reaction terms) / N, which
        // is the mean potential of Eq. eq15 with h' = 1 (the free terms sum to -M_phi sum
        // mu_phi because the Neumann Laplacian of the lattice diffusion sums to zero); taken
        // over the stored values, the multiplier's uniform term cancels them exactly and
        // sum phi is conserved to float-float rounding, as sum psi is through mubar_psi
        lam = -tot[P_SR] / (P.Nd * P.M_phi_d);
        if (P.target) lam += (r.H0 - r.H) / (P.Nd * P.M_phi_d);
    } else if (r.S2 > 0.0) {
        lam = r.S1 / r.S2;
        if (P.target && P.M_phi_d > 0.0) lam = (r.S1 + (r.H0 - r.H) / P.M_phi_d) / r.S2;
    }
    r.lam = lam;
    r.mpsi_mubar = P.psi_on ? -r.S3 / P.Nd : 0.0;
    r.a = diag ? 0.0 : (first ? 1.0 : 1.5);
    return r;
}

// compile-time loop: f(integral_constant<int, I>) for I in [B, E); the lattice tables
// then fold to constants in every direction-dependent expression
template <int I, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < E) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, E>(static_cast<F&&>(f));
    }
}

// The strip-width-dependent part (tile constants, shared-memory layout, block reductions,
// the step kernel): 64-column strips here; the batch also instantiates 32-column strips.
#define SLBM_TILE_TX 64
#include "surflbm_step_tile.inc"
#undef SLBM_TILE_TX

}  // namespace slbm
