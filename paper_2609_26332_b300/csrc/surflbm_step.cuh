// The fused stream-collide kernel of the coupled LBM step and its helpers.
//
// Each CTA owns a strip of TX columns and a segment of rows, and marches up the
// segment RB rows at a time through a software pipeline kept in shared memory rings
// of 8 rows (row y lives in slot y & 7):
//   stage K    for every source node of the next rows, the eight populations it sends,
//              converted once to 32-bit fixed point (both scalar sets);
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

constexpr int TX = 64;           // strip width (cells)
constexpr int RB = 4;            // rows per pipeline iteration
constexpr int NTHREADS = TX * RB;
constexpr int RING = 8;          // ring depth (rows)
constexpr int KX = TX + 6;       // columns of the fixed-point ring (3-node halo)
constexpr int PX = TX + 4;       // columns of the phi / psi ring (2-node halo)
constexpr int MX = TX + 2;       // columns of the mu ring (1-node halo)
constexpr int NPART = 13;        // doubles per block partial

// Raw source rows are staged with cp.async through a 16-byte aligned window of WW
// columns starting at x0 - WOFF (covers the K-ring columns x0 - 3 .. x0 + TX + 2).
constexpr int WOFF = 8;
constexpr int WW = TX + 16;

// dynamic shared memory layout (bytes)
constexpr size_t SM_K = 2ull * 8 * RING * KX * sizeof(int);      // fixed-point populations
constexpr size_t SM_MT = 2ull * RING * KX * sizeof(float2);      // m~ of every ring node
constexpr size_t SM_P = 4ull * RING * PX * sizeof(float);        // phi, psi (float-float)
constexpr size_t SM_M = 2ull * RING * MX * sizeof(float);        // mu_phi, mu_psi
template <class T> struct Staging {
    static constexpr size_t D_ROW = 16ull * WW * sizeof(T);      // 16 deviation planes
    static constexpr size_t M_ROW = 2ull * WW * sizeof(float2);   // two zeroth-moment planes
    static constexpr size_t P_ROW = 1ull * WW * sizeof(float);    // phi of the previous step
    static constexpr size_t ROW = D_ROW + M_ROW + P_ROW;
    static constexpr size_t BUF = RB * ROW;
    static constexpr size_t BYTES = 2 * BUF;
};
template <class T> constexpr size_t smem_bytes() { return SM_K + SM_MT + SM_P + SM_M + Staging<T>::BYTES; }

// Tensor-memory-access (TMA) staging of one domain (nx a multiple of TX): tile copies
// (cp.async.bulk.tensor) land in shared memory box by box, each set of boxes completing an
// mbarrier; the lane 0s of the warps share the issue.
//   K      single buffer: rows [r, r + RB) of the window x0 - WOFF .. + WW of the 8 + 8
//          deviation planes [plane][row][col], the two zeroth-moment planes [row][col]
//          (float2) and the previous phi [row][col], read by stage K;
//   F[2]   double buffer: rows [r - c_ky, r - c_ky + RB) of flow plane k, so that local row
//          rr holds the pull source of the collide row r + rr, read by the collide.
// The two strips at the periodic seam have WOFF window columns outside [0, nx), which the
// boxes fill with zeros; their periodic images arrive by cp.async in the side buffers
// (K side: [plane][row][WOFF]; F side[2]: [plane][row][WOFF]) and the readers take those
// columns from there.
template <class T> struct TmaStage {
    static constexpr size_t DEV = 8ull * RB * WW * sizeof(T);
    static constexpr size_t MOM = 1ull * RB * WW * sizeof(float2);
    static constexpr size_t PHP = 1ull * RB * WW * sizeof(float);
    static constexpr size_t K_BYTES = 2 * DEV + 2 * MOM + PHP;
    static constexpr size_t FPL = 1ull * RB * WW * sizeof(T);
    static constexpr size_t F_BYTES = 9 * FPL;
    // side buffers of the seam strips (WOFF columns)
    static constexpr size_t SDEV = 8ull * RB * WOFF * sizeof(T);
    static constexpr size_t SMOM = 1ull * RB * WOFF * sizeof(float2);
    static constexpr size_t SPHP = 1ull * RB * WOFF * sizeof(float);
    static constexpr size_t SK_BYTES = 2 * SDEV + 2 * SMOM + SPHP;
    static constexpr size_t SF_BYTES = 9ull * RB * WOFF * sizeof(T);
    // offsets from the stage base
    static constexpr size_t O_DEV0 = 0, O_DEV1 = DEV, O_MOM0 = 2 * DEV, O_MOM1 = 2 * DEV + MOM, O_PHPK = 2 * DEV + 2 * MOM;
    static constexpr size_t O_F0 = K_BYTES, O_F1 = K_BYTES + F_BYTES;
    static constexpr size_t O_SK = K_BYTES + 2 * F_BYTES;
    static constexpr size_t O_SDEV0 = O_SK, O_SDEV1 = O_SK + SDEV, O_SMOM0 = O_SK + 2 * SDEV,
                            O_SMOM1 = O_SK + 2 * SDEV + SMOM, O_SPHP = O_SK + 2 * SDEV + 2 * SMOM;
    static constexpr size_t O_SF0 = O_SK + SK_BYTES, O_SF1 = O_SK + SK_BYTES + SF_BYTES;
    static constexpr size_t BYTES = K_BYTES + 2 * F_BYTES + SK_BYTES + 2 * SF_BYTES;
    static_assert(DEV % 128 == 0 && MOM % 128 == 0 && PHP % 128 == 0 && FPL % 128 == 0, "boxes on 128-byte boundaries");
    static_assert(SDEV % 16 == 0 && SMOM % 16 == 0 && SPHP % 16 == 0 && SF_BYTES % 16 == 0, "16-byte cp.async chunks");
};
template <class T> constexpr size_t smem_bytes_tma() { return SM_K + SM_MT + SM_P + SM_M + TmaStage<T>::BYTES; }
static_assert((SM_K + SM_MT + SM_P + SM_M) % 128 == 0, "stage base on a 128-byte boundary");
// two CTAs per SM: 228 KB of shared memory per SM, 1 KB reserved and ~1 KB static per CTA
static_assert(smem_bytes_tma<float>() + 2048 <= 233472 / 2, "two CTAs per SM");

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

// CTA sum of NPART float-float accumulators; the FP64 result is in s_blk (all threads).
__device__ __forceinline__ void block_sum(ff (&acc)[NPART], double* s_blk) {
    __shared__ double s_w[NPART][NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
        ff v = warp_sum_ff(acc[q]);
        if (lane == 0) s_w[q][warp] = ff_to_d(v);
    }
    __syncthreads();
    if (threadIdx.x < NPART) {
        double t = 0.0;
        for (int w = 0; w < NTHREADS / 32; ++w) t += s_w[threadIdx.x][w];
        s_blk[threadIdx.x] = t;
    }
    __syncthreads();
}

// Partial sums of `nparts` producers (slot-major, NPART each) reduced in a fixed order by
// the calling CTA: warp w sums quantities w, w + 8 with lanes striding the slots.
__device__ __forceinline__ void ordered_sum(const double* partials, int nparts, double* s_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q < NPART; q += NTHREADS / 32) {
        double t = 0.0;
        for (int b = lane; b < nparts; b += 32) t += ((volatile const double*)partials)[(long long)b * NPART + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_tot[q] = t;
    }
    __syncthreads();
}

// Single domain: block partials to partials[blockIdx], then the last CTA to finish
// reduces all of them in fixed order and resolves the record of the time level.
template <class T>
__device__ void finish_reduction(ff (&acc)[NPART], const StepArgs<T>& A, bool diag) {
    __shared__ double s_blk[NPART], s_tot[NPART];
    __shared__ bool s_last;
    block_sum(acc, s_blk);
    const int nblocks = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x < NPART) A.partials[(long long)bid * NPART + threadIdx.x] = s_blk[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(A.counter, 1u) == (unsigned)(nblocks - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ordered_sum(A.partials, nblocks, s_tot);
    if (threadIdx.x == 0) {
        *A.rec_out = resolve_rec(A.P, A.first, A.rec_prev, s_tot, diag);
        *A.counter = 0u;
        __threadfence();
    }
}

// ring accessors
#define KR(s, k, y, col) sK[(((s) * 8 + ((k) - 1)) * RING + ((y) & (RING - 1))) * KX + (col)]
#define MT(s, y, col) sMT[((s) * RING + ((y) & (RING - 1))) * KX + (col)]
#define PH(y, col) sPh[((y) & (RING - 1)) * PX + (col)]
#define PL(y, col) sPl[((y) & (RING - 1)) * PX + (col)]
#define SH(y, col) sSh[((y) & (RING - 1)) * PX + (col)]
#define SL(y, col) sSl[((y) & (RING - 1)) * PX + (col)]
#define MU(y, col) sMu[((y) & (RING - 1)) * MX + (col)]
#define MP(y, col) sMp[((y) & (RING - 1)) * MX + (col)]

// received fixed-point population in direction k at (row y, K-ring column kc); walls: specular
__device__ __forceinline__ int k_in(const int* __restrict__ sK, int s, int k, int y, int kc, int ny) {
    const int sy = y - CYk(k);
    if (sy < 0 || sy >= ny) return KR(s, MIRYk(k), y, kc - CXk(k));
    return KR(s, k, sy, kc - CXk(k));
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

// ------------------------------------------------------------------- the step
// DIAG = true: same moments / forces / velocity / pressure, no collision, writes the
// macroscopic fields and the reduced totals of the current time level.
// VARRHO = false: uniform density and viscosity (no density-gradient terms).
// Work split: the strips x rows of the grid, ordered strip-major, are cut into gridDim.x
// contiguous ranges of equal length; a CTA marches its range (one or two strip pieces).
// TMA = true (single domains whose rows are 16-byte multiples): the staged rows of stage K
// and the collide's flow populations, history and previous phi arrive by TMA boxes
// (TmaStage), issued one iteration ahead by one thread; false: cp.async staging of the
// stage-K rows and direct global loads in the collide (batches, odd or narrow grids).
// MMS = true: the manufactured-solution test of Sec. 4.1 on the channel (verification
// only): no force acts on the flow, and the sources S_phi, S_psi that make the travelling
// decaying modes exact are added to R_phi, R_psi (mms_source).
template <class T, bool DIAG, bool VARRHO, bool BATCH, bool TMA = false, bool MMS = false>
__global__ void __launch_bounds__(NTHREADS, 2)
    step_kernel(const StepArgs<T> A, const BatchArgs B, const __grid_constant__ TmaMaps M) {
    static_assert(!(TMA && BATCH), "the batch kernel stages with cp.async");
    static_assert(!(MMS && (BATCH || VARRHO)), "the manufactured-solution test is a uniform-density single domain");
    extern __shared__ __align__(128) unsigned char smem[];
    int* sK = (int*)smem;
    float2* sMT = (float2*)(smem + SM_K);
    float* sPh = (float*)(smem + SM_K + SM_MT);
    float* sPl = sPh + RING * PX;
    float* sSh = sPl + RING * PX;
    float* sSl = sSh + RING * PX;
    float* sMu = (float*)(smem + SM_K + SM_MT + SM_P);
    float* sMp = sMu + RING * MX;
    unsigned char* sStg = smem + SM_K + SM_MT + SM_P + SM_M;
    using ST = Staging<T>;
    using TS = TmaStage<T>;
    unsigned char* sTma = sStg;   // TMA path: the stage boxes (TmaStage layout) start here
    __shared__ __align__(8) uint64_t s_bar[3];   // TMA path: [0] stage-K boxes, [1 + b] flow boxes of buffer b
    uint32_t phK = 0, phF0 = 0, phF1 = 0;        // parity of the next phase of each
    if (TMA && threadIdx.x == 0) {
        mbar_init1(&s_bar[0]);
        mbar_init1(&s_bar[1]);
        mbar_init1(&s_bar[2]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    int fbuf = 0;          // TMA path: flow buffer of the current iteration
    int seam = 0;          // TMA path: 0, or -1 / +1 for the strip at the left / right seam

    // physical parameters: the kernel argument for one domain, a shared copy of the
    // current instance's parameters in batch mode
    __shared__ Phys sP;
    const Phys& P = BATCH ? sP : A.P;
    const int tid = threadIdx.x;
    const float sc_phi = (float)(1u << SFIX_PHI), sc_psi = 2147483648.0f;
    const float isc_phi = 1.0f / sc_phi, isc_psi = 1.0f / sc_psi;

    // piece context: grid, state buffers, time level (set per domain or per batch piece)
    int nx = A.nx, ny = A.ny, first = A.first;
    long long N = A.N;
    const T* f_in = A.f_in; const T* gd_in = A.gd_in; const T* hd_in = A.hd_in;
    const float2* gm_in = A.gm_in; const float2* hm_in = A.hm_in; const float* php_in = A.php_in;
    T* f_out = A.f_out; T* gd_out = A.gd_out; T* hd_out = A.hd_out;
    float2* gm_out = A.gm_out; float2* hm_out = A.hm_out; float* php_out = A.php_out;
    T* hist = A.hist;
    const Rec* rec_prev = A.rec_prev;

    // deferred multiplier terms of time level n-1 (FP64 only here, once per piece)
    float inv_rho_l = 0.f, qcoef = 0.f, lam_half = 0.f;
    ff cuni = {0.f, 0.f}, mub_half = {0.f, 0.f};
    ff clin = {0.f, 0.f}, lin_half = {0.f, 0.f};   // linear constraint: a M lambda and -M lambda / 2 (uniform)
    int nsets = 1;
    auto set_level = [&]() {
        const Rec rp = *rec_prev;
        inv_rho_l = 1.0f / P.rho_l;
        qcoef = (float)(rp.a * P.M_phi_d * rp.lam);
        const double cu = rp.a * rp.mpsi_mubar;
        cuni.hi = (float)cu;
        cuni.lo = (float)(cu - (double)cuni.hi);
        lam_half = (float)(0.5 * P.M_phi_d * rp.lam);
        const double hm = -0.5 * rp.mpsi_mubar;
        mub_half.hi = (float)hm;
        mub_half.lo = (float)(hm - (double)mub_half.hi);
        const double cl = rp.a * P.M_phi_d * rp.lam, hl = -0.5 * P.M_phi_d * rp.lam;
        clin.hi = (float)cl;
        clin.lo = (float)(cl - (double)clin.hi);
        lin_half.hi = (float)hl;
        lin_half.lo = (float)(hl - (double)lin_half.hi);
        nsets = P.psi_on ? 2 : 1;
    };
    int range = 0;
    float clamps = 0.0f, s1acc = 0.0f, s2acc = 0.0f, kinacc = 0.0f;
    ff acc[NPART];
    auto reset_acc = [&]() {
#pragma unroll
        for (int q = 0; q < NPART; ++q) acc[q] = {0.0f, 0.0f};
        range = 0;
        clamps = s1acc = s2acc = kinacc = 0.0f;
    };
    auto pack_acc = [&]() {
        acc[P_CLAMP] = {clamps, 0.0f};
        acc[P_RANGE] = {(float)range, 0.0f};
        acc[P_S1] = {s1acc, 0.0f};
        acc[P_S2] = {s2acc, 0.0f};
        acc[P_KIN] = {kinacc, 0.0f};
    };
    if (!BATCH) set_level();
    reset_acc();

    int x0 = 0, ys = 0, ye = 0;
    bool vec = false;
    constexpr int VEC = (16 / sizeof(T)) > 4 ? (16 / sizeof(T)) : 4;

    // ------------------------------------------------------------------ stages
    // 16-byte staging path: a staged row is PER_ROW chunks (16 deviation planes, 2 moment
    // planes, phi_prev); this thread always moves chunks q = tid and tid + NTHREADS of every
    // row.  Their shared-memory offsets, sources at row 0 and source row strides depend only
    // on the piece's window, so they are set once per piece (a 16-byte chunk never straddles
    // the periodic seam: window start and nx are multiples of the elements per chunk, so
    // each chunk is fetched from its wrapped column).
    constexpr int CD = (int)(WW * sizeof(T) / 16);    // 16-byte chunks per deviation row
    constexpr int CM = (int)(WW * sizeof(float2) / 16);
    constexpr int PER_ROW = 16 * CD + 2 * CM + (int)(WW * sizeof(float) / 16);
    static_assert(PER_ROW <= 2 * NTHREADS, "two staging chunks per thread and row");
    const unsigned char* csrc[2] = {nullptr, nullptr};
    int cdst[2] = {0, 0}, cstride[2] = {0, 0};   // stride 0: no chunk
    auto prep_chunks = [&]() {
        const int ws = x0 - WOFF;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            int q = tid + j * NTHREADS;
            cstride[j] = 0;
            if (q >= PER_ROW) continue;
            if (q < 16 * CD) {
                const int pl = q / CD, ch = q - pl * CD;
                csrc[j] = (const unsigned char*)((pl < 8 ? gd_in : hd_in) + (long long)(pl & 7) * N +
                                                 wrap1(ws + ch * (int)(16 / sizeof(T)), nx));
                cdst[j] = pl * WW * (int)sizeof(T) + ch * 16;
                cstride[j] = nx * (int)sizeof(T);
            } else if ((q -= 16 * CD) < 2 * CM) {
                const int pl = q / CM, ch = q - pl * CM;
                csrc[j] = (const unsigned char*)((pl == 0 ? gm_in : hm_in) + wrap1(ws + 2 * ch, nx));
                cdst[j] = (int)ST::D_ROW + pl * WW * (int)sizeof(float2) + ch * 16;
                cstride[j] = nx * (int)sizeof(float2);
            } else {
                q -= 2 * CM;
                csrc[j] = (const unsigned char*)(php_in + wrap1(ws + 4 * q, nx));
                cdst[j] = (int)(ST::D_ROW + ST::M_ROW) + q * 16;
                cstride[j] = nx * (int)sizeof(float);
            }
        }
    };

    // staging: raw rows [r0, r0 + nrow) of (16 deviation planes, 2 moment planes, phi_prev)
    // for window columns x0 - WOFF .. x0 - WOFF + WW - 1, into buffer b
    auto issue = [&](int b, int r0, int nrow) {
        unsigned char* base = sStg + (size_t)b * ST::BUF;
        const int ws = x0 - WOFF;
        if (vec) {
            for (int rr = 0; rr < nrow; ++rr) {
                const int y = r0 + rr;
                if (y < 0 || y >= ny) continue;
                unsigned char* row = base + (size_t)rr * ST::ROW;
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (cstride[j]) cp_async16(row + cdst[j], csrc[j] + (long long)y * cstride[j]);
            }
            cp_async_commit();
        } else {
            // strips touching the periodic seam or unaligned grids: element-wise copy
            const int items = nrow * WW;
            for (int it = tid; it < items; it += NTHREADS) {
                const int rr = it / WW, col = it - rr * WW;
                const int y = r0 + rr;
                if (y < 0 || y >= ny) continue;
                unsigned char* row = base + (size_t)rr * ST::ROW;
                const long long cidx = (long long)y * nx + wrapx(ws + col, nx);
                T* dd = (T*)row;
#pragma unroll
                for (int pl = 0; pl < 8; ++pl) {
                    dd[pl * WW + col] = gd_in[(long long)pl * N + cidx];
                    dd[(pl + 8) * WW + col] = hd_in[(long long)pl * N + cidx];
                }
                float2* mm = (float2*)(row + ST::D_ROW);
                mm[col] = gm_in[cidx];
                mm[WW + col] = hm_in[cidx];
                ((float*)(row + ST::D_ROW + ST::M_ROW))[col] = php_in[cidx];
            }
        }
    };

    // stage K from staging buffer b holding rows [r0, r0 + NROW)
    auto stageK = [&](auto nrow_c, int b, int r0) {
        constexpr int NROW = decltype(nrow_c)::value;
        const unsigned char* base = sStg + (size_t)b * ST::BUF;
        const int items = NROW * KX * nsets;
        for (int it = tid; it < items; it += NTHREADS) {
            const int kc = it % KX;
            const int rest = it / KX;
            const int rr = rest % NROW;
            const int s = rest / NROW;
            const int y = r0 + rr;
            if (y < 0 || y >= ny) continue;
            const int col = kc + (WOFF - 3);
            const unsigned char* row = base + (size_t)rr * ST::ROW;
            const float2 mv = ((const float2*)(row + ST::D_ROW))[s * WW + col];
            ff mt = {mv.x, mv.y};
            if (s == 0) {
                if (P.linear) {
                    mt = ff_add(mt, clin);
                } else if (qcoef != 0.0f) {
                    const float php = ((const float*)(row + ST::D_ROW + ST::M_ROW))[col];
                    mt = ff_add_f(mt, __fmul_rn(qcoef, hprime(php, P)));
                }
            } else {
                mt = ff_add(mt, cuni);
            }
            const T* dd = (const T*)row + (size_t)(8 * s) * WW + col;
            const float scl = s == 0 ? sc_phi : sc_psi;
            // fixed point of v = d + w mh: K = rint(d * 2^S + (w 2^S) mh), evaluated once per value
            const float ma = __fmul_rn(__fmul_rn(Wk(1), scl), mt.hi);
            const float md = __fmul_rn(__fmul_rn(Wk(5), scl), mt.hi);
            int ksum = 0;
            int* kd = &KR(s, 1, y, kc);
            static_for<1, 9>([&](auto K) {
                constexpr int k = decltype(K)::value;
                const int kv = __float2int_rn(__fmaf_rn(Stor<T>::lds(dd, (k - 1) * WW), scl, k < 5 ? ma : md));
                kd[(k - 1) * RING * KX] = kv;
                ksum += kv;
            });
            // m~ minus everything the node sends, so that phi = this + (everything it receives)
            const ff basev = ff_add(mt, fixed_to_ff(-ksum, s == 0 ? isc_phi : isc_psi));
            MT(s, y, kc) = make_float2(basev.hi, basev.lo);
        }
    };

    // stage K from the TMA stage holding rows [r0, r0 + RB) (the first NROW are converted);
    // at the periodic seam the window columns outside [0, nx) come from the side buffer
    auto stageK_t = [&](auto nrow_c, int r0) {
        constexpr int NROW = decltype(nrow_c)::value;
        const int items = NROW * KX * nsets;
        for (int it = tid; it < items; it += NTHREADS) {
            const int kc = it % KX;
            const int rest = it / KX;
            const int rr = rest % NROW;
            const int s = rest / NROW;
            const int y = r0 + rr;
            if (y < 0 || y >= ny) continue;
            const int wcol = kc + (WOFF - 3);
            // main box, or side column (left seam: window columns 0..WOFF-1; right seam:
            // WW-WOFF..WW-1)
            const bool side = seam < 0 ? wcol < WOFF : (seam > 0 && wcol >= WW - WOFF);
            const int col = side ? rr * WOFF + (seam < 0 ? wcol : wcol - (WW - WOFF)) : rr * WW + wcol;
            const int pst = side ? RB * WOFF : RB * WW;
            const float2 mv = ((const float2*)(sTma + (side ? (s == 0 ? TS::O_SMOM0 : TS::O_SMOM1)
                                                          : (s == 0 ? TS::O_MOM0 : TS::O_MOM1))))[col];
            ff mt = {mv.x, mv.y};
            if (s == 0) {
                if (P.linear) {
                    mt = ff_add(mt, clin);
                } else if (qcoef != 0.0f) {
                    const float php = ((const float*)(sTma + (side ? TS::O_SPHP : TS::O_PHPK)))[col];
                    mt = ff_add_f(mt, __fmul_rn(qcoef, hprime(php, P)));
                }
            } else {
                mt = ff_add(mt, cuni);
            }
            const T* dd = (const T*)(sTma + (side ? (s == 0 ? TS::O_SDEV0 : TS::O_SDEV1) : (s == 0 ? TS::O_DEV0 : TS::O_DEV1))) + col;
            const float scl = s == 0 ? sc_phi : sc_psi;
            const float ma = __fmul_rn(__fmul_rn(Wk(1), scl), mt.hi);
            const float md = __fmul_rn(__fmul_rn(Wk(5), scl), mt.hi);
            int ksum = 0;
            int* kd = &KR(s, 1, y, kc);
            static_for<1, 9>([&](auto K) {
                constexpr int k = decltype(K)::value;
                const int kv = __float2int_rn(__fmaf_rn(Stor<T>::lds(dd, (k - 1) * pst), scl, k < 5 ? ma : md));
                kd[(k - 1) * RING * KX] = kv;
                ksum += kv;
            });
            const ff basev = ff_add(mt, fixed_to_ff(-ksum, s == 0 ? isc_phi : isc_psi));
            MT(s, y, kc) = make_float2(basev.hi, basev.lo);
        }
    };

    auto stagePhi = [&](auto nrow_c, int r0) {
        constexpr int nrow = decltype(nrow_c)::value;
        const int items = nrow * PX * 2;
        for (int it = tid; it < items; it += NTHREADS) {
            const int pc = it % PX;
            const int rest = it / PX;
            const int rr = rest % nrow;
            const int s = rest / nrow;
            const int y = r0 + rr;
            if (y < 0 || y >= ny) continue;
            if (s == 1 && !P.psi_on) { SH(y, pc) = 0.0f; SL(y, pc) = 0.0f; continue; }
            const int kc = pc + 1;
            const float2 mv = MT(s, y, kc);
            const ff mt = {mv.x, mv.y};
            int ks = 0;
            if (y > 0 && y < ny - 1) {
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    ks += KR(s, k, y - CYk(k), kc - CXk(k));
                });
            } else {
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    ks += k_in(sK, s, k, y, kc, ny);
                });
            }
            const ff v = ff_add(mt, fixed_to_ff(ks, s == 0 ? isc_phi : isc_psi));
            if (s == 0) { PH(y, pc) = v.hi; PL(y, pc) = v.lo; }
            else { SH(y, pc) = v.hi; SL(y, pc) = v.lo; }
        }
    };

    auto stageMu = [&](auto nrow_c, int r0) {
        constexpr int nrow = decltype(nrow_c)::value;
        const int items = nrow * MX;
        for (int it = tid; it < items; it += NTHREADS) {
            const int mc = it % MX;
            const int y = r0 + it / MX;
            if (y < 0 || y >= ny) continue;
            const int pc = mc + 1;
            const float phi = PH(y, pc), psi = SH(y, pc);
            float lp = 0.0f, ls = 0.0f;
            if (y > 0 && y < ny - 1) {
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    lp += Wk(k) * PH(y + CYk(k), pc + CXk(k));
                    ls += Wk(k) * SH(y + CYk(k), pc + CXk(k));
                });
            } else {
                // ghost row beyond the wall: Eq. boundary, three columns
                const int w = y == 0 ? 0 : 1;
                const int side = y == 0 ? -1 : 1;
                float gph[3], gps[3];
#pragma unroll
                for (int j = 0; j < 3; ++j) wall_ghost(PH(y, pc - 1 + j), SH(y, pc - 1 + j), w, P, gph[j], gps[j]);
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    const bool out = (CYk(k) == side) || (y + CYk(k) < 0) || (y + CYk(k) >= ny);
                    const float vphi = out ? gph[CXk(k) + 1] : PH(y + CYk(k), pc + CXk(k));
                    const float vpsi = out ? gps[CXk(k) + 1] : SH(y + CYk(k), pc + CXk(k));
                    lp += Wk(k) * vphi;
                    ls += Wk(k) * vpsi;
                });
            }
            const float lapG_phi = 6.0f * (lp - (1.0f - Wk(0)) * phi);
            const float lapG_psi = 6.0f * (ls - (1.0f - Wk(0)) * psi);
            MU(y, mc) = 4.0f * P.beta * (1.0f - psi) * (phi * phi * phi - phi) - P.kappa * lapG_phi + P.W * psi * phi;
            if (P.psi_on) {
                const float psc = fminf(fmaxf(psi, P.psi_clamp), 1.0f - P.psi_clamp);
                const float om = 1.0f - phi * phi;
                MP(y, mc) = P.kT * (__logf(psc) - __logf(1.0f - psc)) - P.lambda_s * lapG_psi - P.beta * om * om +
                            0.5f * P.W * phi * phi;
            } else {
                MP(y, mc) = 0.0f;
            }
        }
    };

    auto stageCollide = [&](int r0, int r1) {
        const int cc = tid % TX;
        const int y = r0 + tid / TX;
        const int gx = x0 + cc;
        if (y >= r1 || gx >= nx) return;
        const long long c = (long long)y * nx + gx;
        const int pc = cc + 2, mc = cc + 1, kc = cc + 3;
        const ff phff = {PH(y, pc), PL(y, pc)};
        const ff psff = {SH(y, pc), SL(y, pc)};
        const float phi = phff.hi, psi = psff.hi;
        const bool wall_row = (y == 0 || y == ny - 1);

        // flow pull first (longest latency): halfway bounce-back with the moving-wall term
        float f[9];
        const int rr = tid / TX;   // row within the iteration (TMA stage row)
        const float php_self = __ldg(php_in + c);
        // the source-term history of the previous step, loaded here so that its latency
        // overlaps the flow part (after the f stores the loads could not move up)
        T* hi_ = hist + c;
        float Rp_phi = 0.f, Rp_psi = 0.f, hphux = 0.f, hphuy = 0.f, hpsux = 0.f, hpsuy = 0.f;
        if (!DIAG && !first) {
            Rp_phi = Stor<T>::ld(hi_, 0);
            hphux = Stor<T>::ld(hi_, 2 * N);
            hphuy = Stor<T>::ld(hi_, 3 * N);
            if (P.psi_on) {
                Rp_psi = Stor<T>::ld(hi_, N);
                hpsux = Stor<T>::ld(hi_, 4 * N);
                hpsuy = Stor<T>::ld(hi_, 5 * N);
            }
        }
        {
            const int xm = gx == 0 ? nx - 1 : gx - 1, xp = gx == nx - 1 ? 0 : gx + 1;
            const T* fin = f_in;
            const long long rm = c - gx + (long long)(y > 0 ? -nx : 0);      // row y - 1 (clamped)
            const long long r0c = c - gx;
            const long long rp1 = c - gx + (long long)(y < ny - 1 ? nx : 0);  // row y + 1 (clamped)
            if (TMA) {
                // plane k holds rows shifted by -c_ky: local row rr is the pull source row
                const T* fs = (const T*)(sTma + (fbuf ? TS::O_F1 : TS::O_F0)) + rr * WW + WOFF + cc;
                static_for<0, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    f[k] = Stor<T>::lds(fs, k * RB * WW - CXk(k));
                });
                // the strip's edge column at the periodic seam: the source column outside
                // [0, nx) is in the side buffer
                if (seam != 0 && cc == (seam < 0 ? 0 : TX - 1)) {
                    const T* sf = (const T*)(sTma + (fbuf ? TS::O_SF1 : TS::O_SF0)) + rr * WOFF;
                    static_for<1, 9>([&](auto K) {
                        constexpr int k = decltype(K)::value;
                        if (CXk(k) == (seam < 0 ? 1 : -1)) f[k] = Stor<T>::lds(sf, k * RB * WOFF + (seam < 0 ? WOFF - 1 : 0));
                    });
                }
            } else {
                static_for<0, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    constexpr int cx = CXk(k), cy = CYk(k);
                    const int sx = cx == 0 ? gx : (cx > 0 ? xm : xp);
                    const long long rowb = cy == 0 ? r0c : (cy > 0 ? rm : rp1);
                    f[k] = Stor<T>::ld(fin + (k * (unsigned)N), rowb + sx);
                });
            }
            if (wall_row) {
                const float rho_w = VARRHO ? P.rho_g + (P.rho_l - P.rho_g) * liquid_fraction(php_self, P) : P.rho_l;
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    constexpr int o = OPPk(k);
                    const int sy = y - CYk(k);
                    if (sy < 0 || sy >= ny)
                        f[k] = addc(Stor<T>::ld(fin, (long long)o * N + c), -CXk(o),
                                    6.0f * Wk(o) * rho_w * P.uw[sy < 0 ? 0 : 1]);
                });
            }
        }

        // gradients (mirror ghosts for mu and rho), Neumann Laplacian of psi, wall flux
        float gmx = 0.f, gmy = 0.f, gpx = 0.f, gpy = 0.f, grx = 0.f, gry = 0.f;
        float lns = 0.f, wf_phi = 0.f, wf_psi = 0.f;
        float gfx = 0.f, gfy = 0.f, gsx = 0.f, gsy = 0.f;   // grad phi, grad psi (diagnostic pass)
        if (!wall_row) {
            static_for<1, 9>([&](auto K) {
                constexpr int k = decltype(K)::value;
                constexpr int cx = CXk(k), cy = CYk(k);
                constexpr float w3 = 3.0f * Wk(k);
                const float mu = w3 * MU(y + cy, mc + cx);
                const float mp = w3 * MP(y + cy, mc + cx);
                gmx = addc(gmx, cx, mu); gmy = addc(gmy, cy, mu);
                gpx = addc(gpx, cx, mp); gpy = addc(gpy, cy, mp);
                if (VARRHO) {
                    const float vchi = w3 * liquid_fraction(PH(y + cy, pc + cx), P);
                    grx = addc(grx, cx, vchi); gry = addc(gry, cy, vchi);
                }
                lns += Wk(k) * SH(y + cy, pc + cx);
                if (DIAG) {
                    const float vf = w3 * PH(y + cy, pc + cx), vs = w3 * SH(y + cy, pc + cx);
                    gfx = addc(gfx, cx, vf); gfy = addc(gfy, cy, vf);
                    gsx = addc(gsx, cx, vs); gsy = addc(gsy, cy, vs);
                }
            });
        } else {
            const int w = y == 0 ? 0 : 1;
            static_for<1, 9>([&](auto K) {
                constexpr int k = decltype(K)::value;
                constexpr int cx = CXk(k), cy = CYk(k);
                constexpr float w3 = 3.0f * Wk(k);
                const bool out = (y + cy < 0) || (y + cy >= ny);
                const int ym = out ? y : y + cy;   // mirror: same row
                const float mu = w3 * MU(ym, mc + cx);
                const float mp = w3 * MP(ym, mc + cx);
                gmx = addc(gmx, cx, mu); gmy = addc(gmy, cy, mu);
                gpx = addc(gpx, cx, mp); gpy = addc(gpy, cy, mp);
                const float vphi = PH(ym, pc + cx);
                const float vpsi = SH(ym, pc + cx);
                if (VARRHO) {
                    const float vchi = w3 * liquid_fraction(vphi, P);
                    grx = addc(grx, cx, vchi); gry = addc(gry, cy, vchi);
                }
                lns += Wk(k) * vpsi;
                float eph = vphi, eps_ = vpsi;
                if (out) {
                    float gph, gps;
                    wall_ghost(vphi, vpsi, w, P, gph, gps);
                    wf_phi += Wk(k) * (gph - vphi);
                    wf_psi += Wk(k) * (gps - vpsi);
                    eph = gph;
                    eps_ = gps;
                }
                if (DIAG) {   // gradients with the wetting ghosts of Eq. boundary
                    gfx = addc(gfx, cx, w3 * eph); gfy = addc(gfy, cy, w3 * eph);
                    gsx = addc(gsx, cx, w3 * eps_); gsy = addc(gsy, cy, w3 * eps_);
                }
            });
        }
        const float lapN_psi = 6.0f * (lns - (1.0f - Wk(0)) * psi);
        wf_phi *= 6.0f; wf_psi *= 6.0f;
        const float Fx = MMS ? 0.0f : -phi * gmx - psi * gpx + P.Gx;
        const float Fy = MMS ? 0.0f : -phi * gmy - psi * gpy + P.Gy;
        float mms_sphi = 0.0f, mms_spsi = 0.0f;
        if (MMS && !DIAG) mms_source(P, A.level, gx, y, mms_sphi, mms_spsi);
        float chi = 0.f, rho = P.rho_l, inv_rho = inv_rho_l;
        if (VARRHO) {
            // grad rho = (rho_l - rho_g) grad chi over the clipped neighbour values
            const float drho = P.rho_l - P.rho_g;
            grx *= drho; gry *= drho;
            chi = liquid_fraction(phi, P);
            rho = P.rho_g + (P.rho_l - P.rho_g) * chi;
            inv_rho = __frcp_rn(rho);
        }

        float jx = 0.f, jy = 0.f, fsum = 0.f;
        static_for<0, 9>([&](auto K) {
            constexpr int k = decltype(K)::value;
            jx = addc(jx, CXk(k), f[k]);
            jy = addc(jy, CYk(k), f[k]);
            if (k) fsum += f[k];
        });
        const float ux = (jx + 0.5f * Fx) * inv_rho;
        const float uy = (jy + 0.5f * Fy) * inv_rho;
        const float usq = ux * ux + uy * uy;
        const float ugr = VARRHO ? ux * grx + uy * gry : 0.0f;
        const float pres = (1.0f / 3.0f) / (1.0f - Wk(0)) * (fsum + 0.5f * ugr - rho * Wk(0) * usq * 1.5f);

        // integrals the multipliers need (Eq. eq15, Eq. AC_psi); the diagnostic pass also
        // reduces the reported totals and checks for divergence
        const float hp = hprime(phi, P);
        s1acc += hp * MU(y, mc);
        s2acc += hp * hp;
        if (DIAG || (P.target && !P.linear)) {
            const float u = phi * P.inv_phi_b;
            acc[P_Q] = ff_add_f(acc[P_Q], 1.5f * u - 0.5f * u * u * u);
        }
        if (DIAG || (P.target && P.linear)) acc[P_PHI] = ff_add(acc[P_PHI], phff);
        if (DIAG) {
            if (P.psi_on) clamps += (psi < P.psi_clamp || psi > 1.0f - P.psi_clamp) ? 1.0f : 0.0f;
            kinacc += 0.5f * rho * usq;
            acc[P_PSI] = ff_add(acc[P_PSI], psff);
            range |= !(fabsf(ux) < 1.0f && fabsf(uy) < 1.0f && fabsf(phi) < 2.0f && fabsf(pres) < 1e3f);
            // discrete free energy of Eq. eq1 (bulk densities with the gradient terms of the
            // isotropic stencil, plus the wall energy f_w of Eq. eq8 on the wall rows)
            const float om = 1.0f - phi * phi;
            float e = P.beta * om * om + 0.5f * P.kappa * (gfx * gfx + gfy * gfy);
            if (P.psi_on) {
                const float psc = fminf(fmaxf(psi, P.psi_clamp), 1.0f - P.psi_clamp);
                e += P.kT * (psc * logf(psc) + (1.0f - psc) * log1pf(-psc)) + 0.5f * P.lambda_s * (gsx * gsx + gsy * gsy) -
                     P.beta * psi * om * om + 0.5f * P.W * psi * phi * phi;
            }
            if (y == 0) e += wall_energy(phi, psi, 0, P);
            if (y == ny - 1) e += wall_energy(phi, psi, 1, P);
            acc[P_EF] = ff_add_f(acc[P_EF], e);
            // one-step change of phi against the previous time level kept for the source terms
            const float dph = (phff.hi - php_self) + phff.lo;
            acc[P_DPHI2] = ff_add_f(acc[P_DPHI2], dph * dph);
            acc[P_PHI2] = ff_add_f(acc[P_PHI2], phi * phi);
        }

        // free reaction term of the surfactant (R_psi without mubar), rounded to storage:
        // M_psi (-k_B T ln(psi/(1-psi)) + beta (1-phi^2)^2 - (W/2) phi^2 + lambda_s (Lap_G - Lap_N) psi)
        // - M_0 Lap_N psi, written with the mu_psi of stage MU at this node (which holds the
        // same logarithm and adsorption terms with -lambda_s Lap_G psi):
        // -M_psi mu_psi - (M_psi lambda_s + M_0) Lap_N psi
        // free reaction term of phi (R_phi without the lambda^n term, which is deferred), with
        // the kappa-weighted wall flux of the ghost-row closure, rounded to storage
        const float Rf_phi = Stor<T>::rnd(P.M_phi * (-4.0f * P.beta * (1.0f - psi) * (phi * phi * phi - phi) -
                                                     P.W * psi * phi + P.kappa * wf_phi) + mms_sphi);
        if (P.linear) acc[P_SR] = ff_add_f(acc[P_SR], Rf_phi);
        float Rf_psi = 0.0f;
        if (P.psi_on) {
            Rf_psi = Stor<T>::rnd(-P.M_psi * MP(y, mc) - (P.M_psi * P.lambda_s + P.M_0) * lapN_psi + mms_spsi);
            acc[P_S3] = ff_add_f(acc[P_S3], Rf_psi);
        }

        if (DIAG) {
            // each output may be absent on its own
            if (A.o_phi) A.o_phi[c] = ff_to_d(phff);
            if (A.o_psi) A.o_psi[c] = ff_to_d(psff);
            if (A.o_ux) A.o_ux[c] = (double)ux;
            if (A.o_uy) A.o_uy[c] = (double)uy;
            if (A.o_p) A.o_p[c] = (double)pres;
            return;
        }

        // ---- flow collision (Sec. 3): f^eq, source F_{i,1}
        {
            float s2 = P.sf[2];
            if (VARRHO) {
                const float nu = P.nu_g + (P.nu_l - P.nu_g) * chi;
                s2 = __frcp_rn(3.0f * nu + 0.5f);
            }
            const float p3 = 3.0f * pres - 1.5f * rho * usq;
            T* fo = f_out + c;
            const unsigned Nu = (unsigned)N;
            if (P.mrt_f) {
                float feq[9], src[9], sv[9];
                static_for<0, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    const float cu = cdot(k, ux, uy);
                    feq[k] = Wk(k) * (p3 + rho * (3.0f * cu + 4.5f * cu * cu)) - (k == 0 ? 3.0f * pres : 0.0f);
                    float sk = 3.0f * cdot(k, Fx, Fy);
                    if (VARRHO) sk += ugr + 3.0f * (cu * cdot(k, grx, gry) - (1.0f / 3.0f) * ugr);
                    src[k] = Wk(k) * sk;
                });
                sv[0] = P.sf[0] > 0.f ? P.sf[0] : s2;
                sv[1] = sv[2] = P.sf[1] > 0.f ? P.sf[1] : s2;
                sv[3] = sv[4] = sv[5] = s2;
                sv[6] = sv[7] = P.sf[3] > 0.f ? P.sf[3] : s2;
                sv[8] = P.sf[4] > 0.f ? P.sf[4] : s2;
                mrt_collide(f, feq, src, sv);
                static_for<0, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    Stor<T>::st(fo, (long long)(k * Nu), f[k]);
                });
            } else {
                const float a = 1.0f - 0.5f * s2;
                static_for<0, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    const float cu = cdot(k, ux, uy);
                    const float feq = Wk(k) * (p3 + rho * (3.0f * cu + 4.5f * cu * cu)) - (k == 0 ? 3.0f * pres : 0.0f);
                    float sk = 3.0f * cdot(k, Fx, Fy);
                    if (VARRHO) sk += ugr + 3.0f * (cu * cdot(k, grx, gry) - (1.0f / 3.0f) * ugr);
                    Stor<T>::st(fo, (long long)(k * Nu), f[k] + s2 * (feq - f[k]) + a * Wk(k) * sk);
                });
            }
        }

        // ---- history of the source terms (Sec. 3, backward differences)
        const float phux = phi * ux, phuy = phi * uy, psux = psi * ux, psuy = psi * uy;
        float dphux = 0.f, dphuy = 0.f, dpsux = 0.f, dpsuy = 0.f;
        if (!first) {
            dphux = phux - hphux;
            dphuy = phuy - hphuy;
            if (P.psi_on) {
                dpsux = psux - hpsux;
                dpsuy = psuy - hpsuy;
            }
        }

        // ---- the two scalar sets share one code path, unrolled so that the independent
        // phi and psi collisions interleave (more instruction-level parallelism)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s >= nsets) break;
            const float cval = s == 0 ? phi : psi;
            const ff cff = s == 0 ? phff : psff;
            float Rf;
            ff dR;
            Rf = s == 0 ? Rf_phi : Rf_psi;
            // dR = R + (R - R_prev)/2 minus the multiplier part of R_prev; exact in float-float
            // for the surfactant (its total is conserved to round-off), plain float for phi
            if (first) {
                dR = {Rf, 0.0f};
            } else if (s == 0 && !P.linear) {
                dR = {1.5f * Rf - 0.5f * Rp_phi - lam_half * hprime(php_self, P), 0.0f};
            } else {
                // exact in float-float where the total is conserved: the surfactant, and phi
                // under the linear constraint
                const ff t = two_sum(Rf, -(s == 0 ? Rp_phi : Rp_psi));
                dR = ff_add(ff_add_f(ff_scale_pow2(t, 0.5f), Rf), s == 0 ? lin_half : mub_half);
            }
            const ff mstar = ff_add(cff, dR);
            const float isc = s == 0 ? isc_phi : isc_psi;
            float g[9];
            float gs = 0.f;
            if (wall_row) {
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    g[k] = (float)k_in(sK, s, k, y, kc, ny) * isc;
                    gs += g[k];
                });
            } else {
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    g[k] = (float)KR(s, k, y - CYk(k), kc - CXk(k)) * isc;
                    gs += g[k];
                });
            }
            g[0] = cval - gs;
            const float eta = s == 0 ? P.eta_phi : P.eta_psi;
            const float ax = 3.0f * (s == 0 ? dphux : dpsux), ay = 3.0f * (s == 0 ? dphuy : dpsuy);
            const float cux = 3.0f * (s == 0 ? phux : psux), cuy = 3.0f * (s == 0 ? phuy : psuy);
            const float* sr = s == 0 ? P.sg : P.sh;
            const int mrt = s == 0 ? P.mrt_g : P.mrt_h;
            const float s1 = sr[1];
            // the zeroth moment is carried exactly by m*; the deviations are g*_k - w_k hi(m*)
            // with the local source w_k dR folded in:  g*_k + w_k (dR - hi(m*))
            const float shift = (dR.hi + dR.lo) - mstar.hi;
            T* dout = (s == 0 ? gd_out : hd_out) + c;
            if (mrt) {
                float geq[9], src[9], sv[9];
                static_for<0, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    geq[k] = Wk(k) * (eta * cval + cdot(k, cux, cuy)) + (k == 0 ? (1.0f - eta) * cval : 0.0f);
                    src[k] = Wk(k) * cdot(k, ax, ay);
                });
                sv[0] = sr[0] > 0.f ? sr[0] : s1;
                sv[1] = sv[2] = s1;
                sv[3] = sv[4] = sv[5] = sr[2] > 0.f ? sr[2] : s1;
                sv[6] = sv[7] = sr[3] > 0.f ? sr[3] : s1;
                sv[8] = sr[4] > 0.f ? sr[4] : s1;
                mrt_collide(g, geq, src, sv);
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    Stor<T>::st(dout, (long long)((k - 1) * (unsigned)N), g[k] + Wk(k) * shift);
                });
            } else {
                const float a = 1.0f - 0.5f * s1;
                const float ec = eta * cval;
                static_for<1, 9>([&](auto K) {
                    constexpr int k = decltype(K)::value;
                    const float geq = Wk(k) * (ec + cdot(k, cux, cuy));
                    const float gk = g[k] + s1 * (geq - g[k]) + a * Wk(k) * cdot(k, ax, ay);
                    Stor<T>::st(dout, (long long)((k - 1) * (unsigned)N), gk + Wk(k) * shift);
                });
            }
            float2 mo;
            mo.x = mstar.hi;
            mo.y = mstar.lo;
            (s == 0 ? gm_out : hm_out)[c] = mo;
            Stor<T>::st(hi_, (long long)s * N, Rf);
            Stor<T>::st(hi_, (long long)(2 + 2 * s) * N, s == 0 ? phux : psux);
            Stor<T>::st(hi_, (long long)(3 + 2 * s) * N, s == 0 ? phuy : psuy);
        }
        php_out[c] = phi;
    };

    // --------------------------------------------------------------- pipeline
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    // ---- TMA staging (single domain): issue, bounded waits, periodic-seam side loads
    const int warp = tid >> 5, lane = tid & 31;
    auto tma_fail = [&](uint64_t* bar, uint32_t par) {
        if (A.err) atomicOr(A.err, ERR_TMA_WAIT);
        mbar_wait_bounded(bar, par);   // let copies still in flight land before going on
    };
    // stage-K boxes of rows [r0, r0 + RB): lane 0 of warps 0..4 issue one box each, warp 0
    // also the expected byte count (a complete_tx may come first: the count goes negative
    // until then, and the phase cannot complete before warp 0's arrive)
    auto issue_K = [&](int r0) {
        if (lane == 0 && warp < 5) {
            uint64_t* bar = &s_bar[0];
            const int xw = x0 - WOFF;
            if (warp == 0) {
                mbar_expect_tx(bar, (uint32_t)(nsets == 2 ? TS::K_BYTES : TS::K_BYTES - TS::DEV - TS::MOM));
                tma_load_3d(sTma + TS::O_DEV0, &M.dev[0], xw, r0, 0, bar);
            } else if (warp == 1) {
                tma_load_2d(sTma + TS::O_MOM0, &M.mom[0], 2 * xw, r0, bar);
            } else if (warp == 2) {
                tma_load_2d(sTma + TS::O_PHPK, &M.php, xw, r0, bar);
            } else if (nsets == 2) {
                if (warp == 3) tma_load_3d(sTma + TS::O_DEV1, &M.dev[1], xw, r0, 0, bar);
                else tma_load_2d(sTma + TS::O_MOM1, &M.mom[1], 2 * xw, r0, bar);
            }
        }
        if (seam != 0) {
            // the WOFF periodic-image columns: 16-byte cp.async chunks, one per thread
            constexpr int CD = WOFF * (int)sizeof(T) / 16, CM = WOFF * 8 / 16, CP = WOFF * 4 / 16;
            const int xs = seam < 0 ? nx - WOFF : 0;
            int q = tid;
            const int nd = 2 * 8 * RB * CD, nm = 2 * RB * CM, np = RB * CP;
            if (q < nd) {
                const int ch = q % CD, rest = q / CD, rr = rest % RB, pl = rest / RB;   // pl 0..15
                const int y = r0 + rr;
                if (y >= 0 && y < ny && (pl < 8 || nsets == 2)) {
                    const T* src = (pl < 8 ? gd_in : hd_in) + (long long)(pl & 7) * N + (long long)y * nx + xs + ch * (16 / (int)sizeof(T));
                    cp_async16(sTma + (pl < 8 ? TS::O_SDEV0 : TS::O_SDEV1) + (((pl & 7) * RB + rr) * WOFF) * sizeof(T) + ch * 16, src);
                }
            } else if ((q -= nd) < nm) {
                const int ch = q % CM, rest = q / CM, rr = rest % RB, st = rest / RB;
                const int y = r0 + rr;
                if (y >= 0 && y < ny && (st == 0 || nsets == 2)) {
                    const float2* src = (st == 0 ? gm_in : hm_in) + (long long)y * nx + xs + ch * 2;
                    cp_async16(sTma + (st == 0 ? TS::O_SMOM0 : TS::O_SMOM1) + (rr * WOFF) * sizeof(float2) + ch * 16, src);
                }
            } else if ((q -= nm) < np) {
                const int ch = q % CP, rr = q / CP;
                const int y = r0 + rr;
                if (y >= 0 && y < ny)
                    cp_async16(sTma + TS::O_SPHP + (rr * WOFF) * sizeof(float) + ch * 16, php_in + (long long)y * nx + xs + ch * 4);
            }
            cp_async_commit();
        }
    };
    // flow boxes of collide rows [r0, r0 + RB) into buffer fb: plane k by lane 0 of warp k % 8
    auto issue_F = [&](int r0, int fb) {
        uint64_t* bar = &s_bar[1 + fb];
        unsigned char* dst = sTma + (fb ? TS::O_F1 : TS::O_F0);
        if (lane == 0) {
            if (warp == 0) mbar_expect_tx(bar, (uint32_t)TS::F_BYTES);
            for (int k = warp; k < 9; k += NTHREADS / 32)
                tma_load_3d(dst + k * TS::FPL, &M.f, x0 - WOFF, r0 - (k == 2 || k == 5 || k == 6 ? 1 : (k == 4 || k == 7 || k == 8 ? -1 : 0)), k, bar);
        }
        if (seam != 0) {
            constexpr int CD = WOFF * (int)sizeof(T) / 16;
            const int xs = seam < 0 ? nx - WOFF : 0;
            const int q = tid;
            if (q < 9 * RB * CD) {
                const int ch = q % CD, rest = q / CD, rr = rest % RB, k = rest / RB;
                const int ysrc = r0 + rr - CYk_rt(k);
                if (ysrc >= 0 && ysrc < ny)
                    cp_async16(sTma + (fb ? TS::O_SF1 : TS::O_SF0) + ((k * RB + rr) * WOFF) * sizeof(T) + ch * 16,
                               f_in + (long long)k * N + (long long)ysrc * nx + xs + ch * (16 / (int)sizeof(T)));
            }
            cp_async_commit();
        }
    };
    auto wait_K = [&]() {
        if (!mbar_wait_bounded(&s_bar[0], phK)) tma_fail(&s_bar[0], phK);
        phK ^= 1u;
    };
    auto wait_F = [&](int fb) {
        uint32_t& ph = fb ? phF1 : phF0;
        if (!mbar_wait_bounded(&s_bar[1 + fb], ph)) tma_fail(&s_bar[1 + fb], ph);
        ph ^= 1u;
    };

    auto march_tma = [&](int strip, int y0, int y1) {
        ys = y0;
        ye = y1;
        x0 = strip * TX;
        seam = x0 - WOFF < 0 ? -1 : (x0 - WOFF + WW > nx ? 1 : 0);
        __syncthreads();   // the previous piece's last collide read the rings and stages
        issue_K(ys - 3);
        wait_K();
        if (seam) { cp_async_wait_all(); __syncthreads(); }
        stageK_t(I4{}, ys - 3);
        __syncthreads();
        issue_K(ys + 1);
        wait_K();
        if (seam) { cp_async_wait_all(); __syncthreads(); }
        stageK_t(I2{}, ys + 1);
        __syncthreads();
        issue_K(ys + 3);
        fbuf = 0;
        issue_F(ys, 0);
        stagePhi(I4{}, ys - 2);
        __syncthreads();
        stageMu(I2{}, ys - 1);
        if (seam) cp_async_wait_all();
        __syncthreads();
        for (int r = ys; r < ye; r += RB) {
            // the flow boxes of the next iteration go out a whole iteration ahead (their
            // buffer was last read by the collide before the previous barrier)
            if (r + RB < ye) issue_F(r + RB, fbuf ^ 1);
            wait_K();
            stageK_t(I4{}, r + 3);
            __syncthreads();
            if (r + RB < ye) issue_K(r + RB + 3);
            stagePhi(I4{}, r + 2);
            __syncthreads();
            stageMu(I4{}, r + 1);
            if (seam) cp_async_wait_all();   // side columns of the next K and flow boxes
            __syncthreads();
            wait_F(fbuf);
            stageCollide(r, min(r + RB, ye));
            __syncthreads();
            fbuf ^= 1;
        }
    };

    auto march = [&](int strip, int y0, int y1) {
        if constexpr (TMA) {
            march_tma(strip, y0, y1);
            return;
        }
        ys = y0;
        ye = y1;
        x0 = strip * TX;
        vec = (nx % VEC == 0) && (nx >= WW);   // seam strips wrap chunk by chunk
        if (vec) prep_chunks();
        __syncthreads();   // the previous piece's last collide read the rings
        issue(0, ys - 3, 4);
        cp_async_wait_all();
        __syncthreads();
        stageK(I4{}, 0, ys - 3);
        __syncthreads();
        issue(0, ys + 1, 2);
        cp_async_wait_all();
        __syncthreads();
        stageK(I2{}, 0, ys + 1);
        __syncthreads();
        issue(1, ys + 3, RB);
        stagePhi(I4{}, ys - 2);
        __syncthreads();
        stageMu(I2{}, ys - 1);
        cp_async_wait_all();   // the first iteration's rows
        __syncthreads();
        int b = 1;
        for (int r = ys; r < ye; r += RB) {
            if (r + RB < ye) issue(b ^ 1, r + RB + 3, RB);   // next iteration's rows, overlapped
            stageK(I4{}, b, r + 3);
            __syncthreads();
            stagePhi(I4{}, r + 2);
            __syncthreads();
            stageMu(I4{}, r + 1);
            __syncthreads();
            stageCollide(r, min(r + RB, ye));
            // one barrier both publishes the next iteration's staged rows and frees the
            // rings this collide read
            cp_async_wait_all();
            __syncthreads();
            b ^= 1;
        }
    };

    if (!BATCH) {
        // one domain: the strips x rows, strip-major, cut into gridDim.x equal ranges
        const long long total = A.total;
        long long lo = total * blockIdx.x / gridDim.x;
        const long long hi = total * (blockIdx.x + 1) / gridDim.x;
        while (lo < hi) {
            const int strip = (int)(lo / ny);
            const int y0 = (int)(lo - (long long)strip * ny);
            const int y1 = (int)min((long long)ny, (long long)y0 + (hi - lo));
            lo += y1 - y0;
            march(strip, y0, y1);
        }
        pack_acc();
        finish_reduction<T>(acc, A, DIAG);
        return;
    }

    // batch: persistent CTAs take pieces from the tile queue; every piece is reduced on
    // its own into its instance's slot, and the instance's last piece resolves its record
    __shared__ int s_piece;
    __shared__ bool s_last;
    __shared__ double s_blk[NPART], s_tot[NPART];
    const long long G = *B.G;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_piece = (int)atomicAdd(B.queue, 1u);
        __syncthreads();
        const int pi = s_piece;
        if (pi >= B.npieces) break;
        const Piece pc = B.pieces[pi];
        const InstDesc* I = B.inst + pc.inst;
        {
            const int* src = (const int*)&I->P;
            int* dst = (int*)&sP;
            for (int w = tid; w < (int)(sizeof(Phys) / 4); w += NTHREADS) dst[w] = src[w];
        }
        nx = I->nx;
        ny = I->ny;
        N = I->N;
        const long long n = G - I->G0;
        first = n == 0;
        const int ci = (int)(n & 1), co = ci ^ 1;
        f_in = (const T*)I->f[ci]; gd_in = (const T*)I->gd[ci]; hd_in = (const T*)I->hd[ci];
        gm_in = I->gm[ci]; hm_in = I->hm[ci]; php_in = I->php[ci];
        f_out = (T*)I->f[co]; gd_out = (T*)I->gd[co]; hd_out = (T*)I->hd[co];
        gm_out = (float2*)I->gm[co]; hm_out = (float2*)I->hm[co]; php_out = (float*)I->php[co];
        hist = (T*)I->hist;
        rec_prev = n == 0 ? I->recs + 3 : I->recs + ((n - 1) & 1);
        __syncthreads();   // sP visible
        set_level();
        reset_acc();
        march(pc.strip, pc.y0, pc.y1);
        pack_acc();
        block_sum(acc, s_blk);
        if (tid < NPART) I->partials[(long long)pc.slot * NPART + tid] = s_blk[tid];
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = (atomicAdd(I->counter, 1u) == (unsigned)(I->npieces - 1));
        __syncthreads();
        if (s_last) {
            __threadfence();
            ordered_sum(I->partials, I->npieces, s_tot);
            if (tid == 0) {
                I->recs[n & 1] = resolve_rec(P, first, rec_prev, s_tot, false);
                *I->counter = 0u;
                __threadfence();
            }
        }
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(B.done, 1u) == gridDim.x - 1) {
            *B.queue = 0u;
            *B.done = 0u;
            *B.G = G + 1;
            __threadfence();
        }
    }
}

#undef KR
#undef MT
#undef PH
#undef PL
#undef SH
#undef SL
#undef MU
#undef MP

}  // namespace slbm
