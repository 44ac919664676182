// Three-dimensional extension of the coupled step (include/surflbm3d.h): the scheme of
// Sec. 3 on D3Q19 for the flow f, phase field g and surfactant h, single relaxation time,
// x and z periodic, walls below y = 0 and above y = ny - 1 with the closure of the
// two-dimensional solver (ghost planes of Eq. boundary, halfway bounce-back with the
// moving-wall term for f, specular reflection for g and h, the wall flux in R).
//
// State (FP32, SoA planes of N = nx ny nz cells, ping-pong): f* (19 planes), g*_k and h*_k
// for the 18 moving directions, the zeroth moments m* of g and h minus the fixed-point
// values each node sends (m~, float-float; the rest population is m* minus the moving
// ones), and the history R^{n-1}, (phi u)^{n-1},
// (psi u)^{n-1} (8 planes).  One step is three launches:
//   moments3d     phi, psi = m~ + (received), m~ = m* - (sent) stored by the collide: every
//                 streamed population is converted to 32-bit fixed point by one
//                 deterministic rule, at the sender (into m~) and at the receiver, so the
//                 two integers agree and the exchange telescopes exactly (sum psi, and sum
//                 phi under the linear constraint, conserved to float-float rounding);
//   potentials3d  mu_phi, mu_psi (Eqs. eq_muphi, eq_mupsi) with the isotropic D3Q19
//                 Laplacian and the ghost planes, the free reaction terms, and the FP64
//                 integrals; the last block resolves lambda_phi (Eq. eq15) and mubar_psi
//                 (Eq. AC_psi) of this step, so the collide uses them directly;
//   collide3d     force (Eq. eq_Fs0), u, p, equilibria, sources and the BGK collision of
//                 the three sets, with the pull of f.
#include "surflbm3d.h"
#include "surflbm_internal.cuh"

#include <cmath>
#include <cstring>
#include <new>
#include <string>

using namespace slbm;

namespace {

constexpr int Q3 = 19;
constexpr int T3 = NTHREADS;   // threads per block (the reduction helpers assume NTHREADS)

__host__ __device__ constexpr int cx3(int k) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0, 0, 0, 0};
    return t[k];
}
__host__ __device__ constexpr int cy3(int k) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, -1, 1};
    return t[k];
}
__host__ __device__ constexpr int cz3(int k) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[k];
}
__host__ __device__ constexpr float w3(int k) { return k == 0 ? 1.0f / 3.0f : (k < 7 ? 1.0f / 18.0f : 1.0f / 36.0f); }
__host__ __device__ constexpr double w3d(int k) { return k == 0 ? 1.0 / 3.0 : (k < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
__host__ __device__ constexpr int find3(int a, int b, int c) {
    for (int k = 0; k < 19; ++k)
        if (cx3(k) == a && cy3(k) == b && cz3(k) == c) return k;
    return -1;
}
__host__ __device__ constexpr int opp3(int k) { return find3(-cx3(k), -cy3(k), -cz3(k)); }
__host__ __device__ constexpr int miry3(int k) { return find3(cx3(k), -cy3(k), cz3(k)); }

// c_k . (ax, ay, az) with the zero components folded away at compile time
template <int K>
__device__ __forceinline__ float cdot3(float ax, float ay, float az) {
    float r = 0.0f;
    if constexpr (cx3(K) != 0) r = cx3(K) > 0 ? ax : -ax;
    if constexpr (cy3(K) != 0) r = cy3(K) > 0 ? r + ay : r - ay;
    if constexpr (cz3(K) != 0) r = cz3(K) > 0 ? r + az : r - az;
    return r;
}

struct Grid3 {
    int nx, ny, nz;
    long long N;
    __device__ __forceinline__ long long idx(int x, int y, int z) const { return ((long long)z * ny + y) * nx + x; }
    __device__ __forceinline__ int wx(int x) const { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }
    __device__ __forceinline__ int wz(int z) const { return z < 0 ? z + nz : (z >= nz ? z - nz : z); }
};

// The neighbours of one cell as offsets from its index, set once per cell: x and z wrap
// periodically, y stays in the own row where x + c leaves [0, ny) (the caller decides what a
// wall link means there: mirror, ghost, bounce-back or specular partner).
struct Nbr {
    long long c;
    int ox[3], oz[3], oym, oyp;
    bool ylo, yhi;
    __device__ __forceinline__ Nbr(const Grid3& G, long long c_, int x, int y, int z) : c(c_) {
        const int pl = G.nx * G.ny;
        ox[0] = x == 0 ? G.nx - 1 : -1;
        ox[1] = 0;
        ox[2] = x == G.nx - 1 ? 1 - G.nx : 1;
        oz[0] = z == 0 ? (G.nz - 1) * pl : -pl;
        oz[1] = 0;
        oz[2] = z == G.nz - 1 ? (1 - G.nz) * pl : pl;
        ylo = y == 0;
        yhi = y == G.ny - 1;
        oym = ylo ? 0 : -G.nx;
        oyp = yhi ? 0 : G.nx;
    }
    // index of the node at (x + DX, y + DY, z + DZ), y kept where it would leave the channel
    template <int DX, int DY, int DZ>
    __device__ __forceinline__ long long at() const {
        int o = ox[DX + 1] + oz[DZ + 1];
        if constexpr (DY < 0) o += oym;
        if constexpr (DY > 0) o += oyp;
        return c + o;
    }
    // does y + DY leave [0, ny)?
    template <int DY>
    __device__ __forceinline__ bool out() const { return (DY < 0 && ylo) || (DY > 0 && yhi); }
};

struct Args3 {
    Grid3 g;
    const float* f_in; const float* g_in; const float2* gm_in; const float* h_in; const float2* hm_in;
    float* f_out; float* g_out; float2* gm_out; float* h_out; float2* hm_out;
    float* hist;              // R_phi, R_psi free terms (R_phi full for the nonlinear constraint),
                              // (phi u)_xyz, (psi u)_xyz of the previous step
    float2* phi; float2* psi; // moments of this step (float-float)
    float* mu_phi; float* mu_psi; float* rf_phi; float* rf_psi;
    double* partials;
    unsigned int* counter;
    const Rec* rec_prev;      // level n-1 (zeros before the first step)
    Rec* rec;                 // level n
    int first;
    double* o[6];             // diagnostic outputs (phi, psi, ux, uy, uz, p), may be null
    Phys P;
};

// The population node (x, y, z) receives in direction k: the one sent by x - c_k, or, for
// a link whose source lies beyond a y-wall, the specular partner sent by
// (x - c_kx, y, z - c_kz) in the direction with the y component reversed.
// IN (compile time): the node's row is off both walls, no link leaves the channel
template <int K, bool IN = false>
__device__ __forceinline__ long long recv_index(const Grid3& G, const Nbr& nb) {
    if (!IN && nb.out<-cy3(K)>()) return (long long)(miry3(K) - 1) * G.N + nb.at<-cx3(K), 0, -cz3(K)>();
    return (long long)(K - 1) * G.N + nb.at<-cx3(K), -cy3(K), -cz3(K)>();
}

template <int I, int E, class F>
__device__ __forceinline__ void sfor(F&& f) {
    if constexpr (I < E) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, E>(static_cast<F&&>(f));
    }
}

// exact float-float value of an int64 fixed-point number K * isc (|K| < 2^43, isc a power
// of two): the high part (|K >> 24| < 2^19) and the low 24 bits are each exact in FP32
__device__ __forceinline__ ff fixed64_to_ff(long long K, float isc) {
    const long long kh = K >> 24;
    const float hi = __fmul_rn((float)kh, __fmul_rn(16777216.0f, isc));
    const float lo = __fmul_rn((float)(K - (kh << 24)), isc);
    return two_sum(hi, lo);
}

// Every cell once: the row segments (a segment is up to T3 consecutive x of one row
// (y, z); segment-major order) are dealt round-robin, item blockIdx.x + j gridDim.x to
// block blockIdx.x, so that at any moment the blocks work on consecutive rows: the
// neighbours a cell gathers in the planes z - 1 and z + 1 (ny rows away) are read within
// a few hundred rows of each other, while they are still in L2 (a contiguous range per
// block put them a block's range apart in time, and the links along z were fetched from
// DRAM twice).  The block steps through its items incrementing y and z, so no integer
// division is done per cell.
template <class F>
__device__ __forceinline__ void for_cells(const Grid3& G, F&& body) {
    const int nseg = (G.nx + T3 - 1) / T3;
    const int rows = G.ny * G.nz;
    const long long items = (long long)rows * nseg;
    const long long g = gridDim.x;
    const long long lo = blockIdx.x;
    if (lo >= items) return;
    int seg = (int)(lo / rows), row = (int)(lo - (long long)seg * rows);
    int y = row % G.ny, z = row / G.ny;
    const int dseg = (int)(g / rows), drow = (int)(g - (long long)dseg * rows);
    const int dy = drow % G.ny, dz = drow / G.ny;
    for (long long it = lo; it < items; it += g) {
        const int x = seg * T3 + (int)threadIdx.x;
        if (x < G.nx) body((long long)row * G.nx + x, x, y, z);
        seg += dseg;
        row += drow;
        y += dy;
        z += dz;
        if (y >= G.ny) {
            y -= G.ny;
            ++z;
        }
        if (row >= rows) {
            row -= rows;
            z -= G.nz;
            ++seg;
        }
    }
}

// ------------------------------------------------------------------ moments3d
__global__ void __launch_bounds__(T3) moments3d(const Args3 A) {
    const Grid3 G = A.g;
    const float scl[2] = {(float)(1u << SFIX_PHI), 2147483648.0f};
    const float isc[2] = {1.0f / scl[0], 1.0f / scl[1]};
    const int nsets = A.P.psi_on ? 2 : 1;
    // rows off the walls take a variant without the wall tests of the links
    auto cell = [&](auto in_c, long long c, int x, int y, int z) {
        constexpr bool IN = decltype(in_c)::value;
        const Nbr nb(G, c, x, y, z);
        for (int s = 0; s < 2; ++s) {
            float2* out = s == 0 ? A.phi : A.psi;
            if (s >= nsets) {
                out[c] = make_float2(0.f, 0.f);
                continue;
            }
            const float* pop = s == 0 ? A.g_in : A.h_in;
            // the stored moment is m~ = m* minus everything the node sent (the collide, or
            // the initialisation, subtracted it), so phi = m~ + (everything received)
            const float2 m = (s == 0 ? A.gm_in : A.hm_in)[c];
            long long kr = 0;
            sfor<1, Q3>([&](auto KI) {
                constexpr int k = decltype(KI)::value;
                kr += (long long)__float2int_rn(__fmul_rn(__ldg(pop + recv_index<k, IN>(G, nb)), scl[s]));
            });
            const ff v = ff_add({m.x, m.y}, fixed64_to_ff(kr, isc[s]));
            out[c] = make_float2(v.hi, v.lo);
        }
    };
    for_cells(G, [&](long long c, int x, int y, int z) {
        if (y > 0 && y < G.ny - 1) cell(std::true_type{}, c, x, y, z);
        else cell(std::false_type{}, c, x, y, z);
    });
}

// ------------------------------------------------------------------ potentials3d
// value of a moment field at the neighbour x + c_k, with the ghost value of Eq. boundary
// (G) or the mirror value (N) beyond a wall
template <int K>
__device__ __forceinline__ void nb_vals(const Args3& A, const Nbr& nb, float& ph, float& ps) {
    const long long i = nb.at<cx3(K), cy3(K), cz3(K)>();
    ph = A.phi[i].x;
    ps = A.psi[i].x;
}

__global__ void __launch_bounds__(T3) potentials3d(const Args3 A, int diag) {
    const Grid3 G = A.g;
    const Phys& P = A.P;
    ff acc[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) acc[q] = {0.f, 0.f};
    float clamps = 0.f;
    // rows off the walls take a variant without the ghost-plane tests of the links
    auto cell = [&](auto in_c, long long c, int x, int y, int z) {
        constexpr bool IN = decltype(in_c)::value;
        const float2 pc = A.phi[c], sc = A.psi[c];
        const float phi = pc.x, psi = sc.x;
        float lgp = 0.f, lgs = 0.f, lnp = 0.f, lns = 0.f;
        const bool wall = !IN && (y == 0 || y == G.ny - 1);
        const Nbr nb(G, c, x, y, z);
        sfor<1, Q3>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            float ph, ps;
            nb_vals<k>(A, nb, ph, ps);
            lnp += w3(k) * ph;
            lns += w3(k) * ps;
            if (wall && nb.out<cy3(k)>()) {
                // beyond a wall: the mirror value for the Neumann Laplacian, the ghost value of
                // Eq. boundary (from the wall-row values at x + c) for the wetting one
                float gph, gps;
                wall_ghost(ph, ps, cy3(k) < 0 ? 0 : 1, A.P, gph, gps);
                ph = gph;
                ps = gps;
            }
            lgp += w3(k) * ph;
            lgs += w3(k) * ps;
        });
        const float LGp = 6.0f * (lgp - (1.0f - w3(0)) * phi), LNp = 6.0f * (lnp - (1.0f - w3(0)) * phi);
        const float LGs = 6.0f * (lgs - (1.0f - w3(0)) * psi), LNs = 6.0f * (lns - (1.0f - w3(0)) * psi);
        const float mu = 4.0f * P.beta * (1.0f - psi) * (phi * phi * phi - phi) - P.kappa * LGp + P.W * psi * phi;
        float mp = 0.f, rfs = 0.f;
        if (P.psi_on) {
            const float psc = fminf(fmaxf(psi, P.psi_clamp), 1.0f - P.psi_clamp);
            clamps += (psc != psi) ? 1.0f : 0.0f;
            const float om = 1.0f - phi * phi;
            mp = P.kT * (__logf(psc) - __logf(1.0f - psc)) - P.lambda_s * LGs - P.beta * om * om + 0.5f * P.W * phi * phi;
            // R_psi without mubar: M_psi (-k_B T ln + beta (1-phi^2)^2 - W/2 phi^2 + lambda_s (L_G - L_N) psi)
            // - M_0 L_N psi, written with mu_psi
            rfs = -P.M_psi * mp - (P.M_psi * P.lambda_s + P.M_0) * LNs;
        }
        const float rfp = P.M_phi * (-4.0f * P.beta * (1.0f - psi) * (phi * phi * phi - phi) - P.W * psi * phi +
                                     P.kappa * (LGp - LNp));
        A.mu_phi[c] = mu;
        A.mu_psi[c] = mp;
        A.rf_phi[c] = rfp;
        A.rf_psi[c] = rfs;
        const float hp = hprime(phi, P);
        acc[P_S1] = ff_add_f(acc[P_S1], hp * mu);
        acc[P_S2] = ff_add_f(acc[P_S2], hp * hp);
        acc[P_S3] = ff_add_f(acc[P_S3], rfs);
        acc[P_SR] = ff_add_f(acc[P_SR], rfp);
        const float u = phi * P.inv_phi_b;
        acc[P_Q] = ff_add_f(acc[P_Q], 1.5f * u - 0.5f * u * u * u);
        acc[P_PHI] = ff_add(acc[P_PHI], {pc.x, pc.y});
        acc[P_PSI] = ff_add(acc[P_PSI], {sc.x, sc.y});
    };
    for_cells(G, [&](long long c, int x, int y, int z) {
        if (y > 0 && y < G.ny - 1) cell(std::true_type{}, c, x, y, z);
        else cell(std::false_type{}, c, x, y, z);
    });
    acc[P_CLAMP] = {clamps, 0.f};
    __shared__ double s_blk[NPART], s_tot[NPART];
    __shared__ bool s_last;
    block_sum(acc, s_blk);
    if (threadIdx.x < NPART) A.partials[(long long)blockIdx.x * NPART + threadIdx.x] = s_blk[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(A.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ordered_sum(A.partials, gridDim.x, s_tot);
    if (threadIdx.x == 0) {
        *A.rec = resolve_rec(P, A.first, A.rec_prev, s_tot, diag != 0);
        *A.counter = 0u;
        __threadfence();
    }
}

// ------------------------------------------------------------------ collide3d
// uniform part of R as float-float: 1.5 c^n - 0.5 c^{n-1} (or c^n on the first step)
__device__ __forceinline__ ff uniform_part(double cn, double cp, int first) {
    const double u = first ? cn : 1.5 * cn - 0.5 * cp;
    const float hi = (float)u;
    return {hi, (float)(u - (double)hi)};
}

template <bool DIAG>
__global__ void __launch_bounds__(T3, 2) collide3d(const Args3 A) {
    const Grid3 G = A.g;
    const Phys& P = A.P;
    const long long N = G.N;
    const Rec rn = *A.rec, rp = *A.rec_prev;
    const float rho = P.rho_l;
    const float s_f = P.sf[2], s_g = P.sg[1], s_h = P.sh[1];
    const float lamM = (float)(P.M_phi_d * rn.lam);
    // uniform parts of R^n, R^{n-1}: M_psi mubar (psi), M_phi lambda (phi, linear constraint)
    const ff upsi = uniform_part(rn.mpsi_mubar, rp.mpsi_mubar, A.first);
    const ff uphi = uniform_part(P.M_phi_d * rn.lam, P.M_phi_d * rp.lam, A.first);
    float kin = 0.f;
    int range = 0;
    // the common case takes a compile-time variant: the row off both walls (no wall tests
    // of the links), and FAST: the surfactant on, the paper's multiplier, not the first step
    auto cell = [&](auto in_c, auto fast_c, long long c, int x, int y, int z) {
        constexpr bool IN = decltype(in_c)::value;
        constexpr bool FAST = decltype(fast_c)::value;
        const float2 pcf = A.phi[c], scf = A.psi[c];
        const float phi = pcf.x, psi = scf.x;
        // flow pull with halfway bounce-back (moving wall along x)
        const Nbr nb(G, c, x, y, z);
        float f[Q3];
        sfor<0, Q3>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            if (!IN && nb.out<-cy3(k)>()) {
                constexpr int o = opp3(k);
                const float uw = P.uw[cy3(k) > 0 ? 0 : 1];
                f[k] = __ldg(A.f_in + (long long)o * N + c) - 6.0f * w3(o) * rho * (float)cx3(o) * uw;
            } else {
                f[k] = __ldg(A.f_in + (long long)k * N + nb.at<-cx3(k), -cy3(k), -cz3(k)>());
            }
        });
        // gradients of the potentials (mirror values beyond a wall)
        float gmx = 0.f, gmy = 0.f, gmz = 0.f, gpx = 0.f, gpy = 0.f, gpz = 0.f;
        sfor<1, Q3>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            const long long i = nb.at<cx3(k), cy3(k), cz3(k)>();   // mirror value beyond a wall
            const float mu = 3.0f * w3(k) * __ldg(A.mu_phi + i), mp = 3.0f * w3(k) * __ldg(A.mu_psi + i);
            if constexpr (cx3(k) != 0) { gmx += cx3(k) * mu; gpx += cx3(k) * mp; }
            if constexpr (cy3(k) != 0) { gmy += cy3(k) * mu; gpy += cy3(k) * mp; }
            if constexpr (cz3(k) != 0) { gmz += cz3(k) * mu; gpz += cz3(k) * mp; }
        });
        const float Fx = -phi * gmx - psi * gpx + P.Gx;
        const float Fy = -phi * gmy - psi * gpy + P.Gy;
        const float Fz = -phi * gmz - psi * gpz;
        float jx = 0.f, jy = 0.f, jz = 0.f, fsum = 0.f;
        sfor<0, Q3>([&](auto KI) {
            constexpr int k = decltype(KI)::value;
            if constexpr (cx3(k) != 0) jx += cx3(k) * f[k];
            if constexpr (cy3(k) != 0) jy += cy3(k) * f[k];
            if constexpr (cz3(k) != 0) jz += cz3(k) * f[k];
            if constexpr (k != 0) fsum += f[k];
        });
        const float inv_rho = 1.0f / rho;
        const float ux = (jx + 0.5f * Fx) * inv_rho, uy = (jy + 0.5f * Fy) * inv_rho, uz = (jz + 0.5f * Fz) * inv_rho;
        const float usq = ux * ux + uy * uy + uz * uz;
        const float pres = (1.0f / 3.0f) / (1.0f - w3(0)) * (fsum - rho * w3(0) * usq * 1.5f);
        if (DIAG) {
            kin += 0.5f * rho * usq;
            range |= !(fabsf(ux) < 1.0f && fabsf(uy) < 1.0f && fabsf(uz) < 1.0f && fabsf(phi) < 2.0f &&
                       fabsf(pres) < 1e3f);
            if (A.o[0]) A.o[0][c] = (double)pcf.x + (double)pcf.y;
            if (A.o[1]) A.o[1][c] = (double)scf.x + (double)scf.y;
            if (A.o[2]) A.o[2][c] = ux;
            if (A.o[3]) A.o[3][c] = uy;
            if (A.o[4]) A.o[4][c] = uz;
            if (A.o[5]) A.o[5][c] = pres;
            return;
        }
        // flow BGK collision with F_{i,1} (uniform density: w_i c_i . F / c_s^2)
        {
            const float p3 = 3.0f * pres - 1.5f * rho * usq;
            const float a = 1.0f - 0.5f * s_f;
            sfor<0, Q3>([&](auto KI) {
                constexpr int k = decltype(KI)::value;
                const float cu = cdot3<k>(ux, uy, uz);
                const float feq = w3(k) * (p3 + rho * (3.0f * cu + 4.5f * cu * cu)) - (k == 0 ? 3.0f * pres : 0.0f);
                A.f_out[(long long)k * N + c] = f[k] + s_f * (feq - f[k]) + a * w3(k) * 3.0f * cdot3<k>(Fx, Fy, Fz);
            });
        }
        // history and the time derivatives of the source terms (Sec. 3)
        float* hs = A.hist + c;
        const float phux = phi * ux, phuy = phi * uy, phuz = phi * uz;
        const float psux = psi * ux, psuy = psi * uy, psuz = psi * uz;
        float Rp_phi = 0.f, Rp_psi = 0.f, d[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (FAST || !A.first) {
            Rp_phi = hs[0];
            Rp_psi = hs[N];
            d[0] = phux - hs[2 * N]; d[1] = phuy - hs[3 * N]; d[2] = phuz - hs[4 * N];
            d[3] = psux - hs[5 * N]; d[4] = psuy - hs[6 * N]; d[5] = psuz - hs[7 * N];
        }
        const float rfp = A.rf_phi[c], rfs = A.rf_psi[c];
        for (int s = 0; s < 2; ++s) {
            if (!FAST && s == 1 && !P.psi_on) {
                break;
            }
            const ff cff = s == 0 ? ff{pcf.x, pcf.y} : ff{scf.x, scf.y};
            ff dR;
            float Rstore;
            if (s == 0 && (FAST || !P.linear)) {
                // R_phi = free part + M_phi lambda^n h'(phi), both in float (sum phi is not a
                // conserved quantity of the nonlinear constraint)
                const float R = rfp + lamM * hprime(phi, P);
                dR = {(!FAST && A.first) ? R : 1.5f * R - 0.5f * Rp_phi, 0.f};
                Rstore = R;
            } else {
                // free part exactly in float-float plus the uniform part, so that the sum
                // over the grid cancels: 1.5 R^n - 0.5 R^{n-1}
                const float Rf = s == 0 ? rfp : rfs;
                const ff un = s == 0 ? uphi : upsi;
                if (!FAST && A.first) {
                    dR = ff_add(ff{Rf, 0.f}, un);
                } else {
                    const ff t = two_sum(Rf, -(s == 0 ? Rp_phi : Rp_psi));
                    dR = ff_add(ff_add_f(ff_scale_pow2(t, 0.5f), Rf), un);
                }
                Rstore = Rf;
            }
            const float* pop = s == 0 ? A.g_in : A.h_in;
            float* pout = s == 0 ? A.g_out : A.h_out;
            const float sr = s == 0 ? s_g : s_h;
            const float eta = s == 0 ? P.eta_phi : P.eta_psi;
            const float cval = s == 0 ? phi : psi;
            const float cux = 3.0f * (s == 0 ? phux : psux), cuy = 3.0f * (s == 0 ? phuy : psuy),
                        cuz = 3.0f * (s == 0 ? phuz : psuz);
            const float ax = 3.0f * d[3 * s], ay = 3.0f * d[3 * s + 1], az = 3.0f * d[3 * s + 2];
            const float a = 1.0f - 0.5f * sr;
            const float dRf = dR.hi + dR.lo;
            const float scl = s == 0 ? (float)(1u << SFIX_PHI) : 2147483648.0f;
            long long ks = 0;   // the fixed-point values this node sends (the rule of moments3d)
            sfor<1, Q3>([&](auto KI) {
                constexpr int k = decltype(KI)::value;
                const float gk = __ldg(pop + recv_index<k, IN>(G, nb));
                const float geq = w3(k) * (eta * cval + cdot3<k>(cux, cuy, cuz));
                const float v = gk + sr * (geq - gk) + a * w3(k) * cdot3<k>(ax, ay, az) + w3(k) * dRf;
                pout[(long long)(k - 1) * N + c] = v;
                ks += (long long)__float2int_rn(__fmul_rn(v, scl));
            });
            // stored: m~ = m* minus everything sent, so the next moments pass adds only what
            // each node receives and the exchange still telescopes exactly
            const ff ms = ff_add(ff_add(cff, dR), fixed64_to_ff(-ks, 1.0f / scl));
            (s == 0 ? A.gm_out : A.hm_out)[c] = make_float2(ms.hi, ms.lo);
            hs[(long long)s * N] = Rstore;
            hs[(long long)(2 + 3 * s) * N] = s == 0 ? phux : psux;
            hs[(long long)(3 + 3 * s) * N] = s == 0 ? phuy : psuy;
            hs[(long long)(4 + 3 * s) * N] = s == 0 ? phuz : psuz;
        }
    };
    const bool fast = P.psi_on && !P.linear && !A.first;
    for_cells(G, [&](long long c, int x, int y, int z) {
        if (y > 0 && y < G.ny - 1) {
            if (fast) cell(std::true_type{}, std::true_type{}, c, x, y, z);
            else cell(std::true_type{}, std::false_type{}, c, x, y, z);
        } else {
            cell(std::false_type{}, std::false_type{}, c, x, y, z);
        }
    });
    if constexpr (DIAG) {
        // kinetic energy and the range flag of the diagnostic level into its record
        ff acc[NPART];
    #pragma unroll
        for (int q = 0; q < NPART; ++q) acc[q] = {0.f, 0.f};
        acc[P_KIN] = {kin, 0.f};
        acc[P_RANGE] = {(float)range, 0.f};
        __shared__ double s_blk[NPART], s_tot[NPART];
        __shared__ bool s_last;
        block_sum(acc, s_blk);
        if (threadIdx.x < NPART) A.partials[(long long)blockIdx.x * NPART + threadIdx.x] = s_blk[threadIdx.x];
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(A.counter, 1u) == gridDim.x - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        ordered_sum(A.partials, gridDim.x, s_tot);
        if (threadIdx.x == 0) {
            A.rec->kin = s_tot[P_KIN];
            A.rec->range = s_tot[P_RANGE];
            *A.counter = 0u;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------ initial state
// Post-collision populations whose first pull gives the equilibria at rest of the
// initial fields: g*_k(x) = w_k eta phi0(target), target x + c_k (or its specular partner
// (x + c_kx, y, z + c_kz) for a link through a wall); the zeroth moment is their sum; the
// flow populations are 0 except on moving-wall links (the inverse of the wall term).
__global__ void init3d(Grid3 G, const double* phi0, const double* psi0, int psi_on, double eta_phi, double eta_psi,
                       double rho, double uw0, double uw1, float* f, float* g, float2* gm, float* h, float2* hm,
                       float* hist) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.N) return;
    const int x = (int)(c % G.nx);
    const long long r = c / G.nx;
    const int y = (int)(r % G.ny), z = (int)(r / G.ny);
    for (int s = 0; s < 2; ++s) {
        const double* F = s == 0 ? phi0 : psi0;
        const bool on = s == 0 || psi_on;
        const double eta = s == 0 ? eta_phi : eta_psi;
        float* pop = s == 0 ? g : h;
        double msum = on ? (1.0 - (1.0 - w3d(0)) * eta) * F[c] : 0.0;
        const float scl = s == 0 ? (float)(1u << SFIX_PHI) : 2147483648.0f;
        long long ks = 0;
        for (int k = 1; k < Q3; ++k) {
            int ty = y + cy3(k);
            if (ty < 0 || ty >= G.ny) ty = y;
            const long long t = G.idx(G.wx(x + cx3(k)), ty, G.wz(z + cz3(k)));
            const double v = on ? w3d(k) * eta * F[t] : 0.0;
            pop[(long long)(k - 1) * G.N + c] = (float)v;
            // the exact value: every initial value is sent exactly once, so the grid total
            // of the zeroth moments (and of phi, psi after the first pull) is that of F
            msum += v;
            ks += (long long)__float2int_rn(__fmul_rn((float)v, scl));
        }
        // the rest population w_0 eta F plus (1 - eta) F is part of the zeroth moment; stored
        // minus the fixed-point values the node sends (m~, as the collide stores it)
        const double mt = msum - (double)ks / (double)scl;
        const float hi = (float)mt;
        (s == 0 ? gm : hm)[c] = make_float2(hi, (float)(mt - (double)hi));
    }
    for (int k = 0; k < Q3; ++k) {
        const int ty = y + cy3(k);
        double v = 0.0;
        if (ty < 0 || ty >= G.ny) v = 6.0 * w3d(k) * rho * cx3(k) * (ty < 0 ? uw0 : uw1);
        f[(long long)k * G.N + c] = (float)v;
    }
    for (int q = 0; q < 8; ++q) hist[(long long)q * G.N + c] = 0.f;
}

std::string g_err3 = "no error";

}  // namespace

struct slbm3d_domain {
    slbm_domain core;           // parameters, derived constants, walls (no 2D state allocated)
    int nz = 1;
    Grid3 G{};
    int cur = 0;
    long long n = 0;
    bool initialised = false;
    int grid[3] = {1, 1, 1};    // moments3d, potentials3d, collide3d: resident blocks (persistent)
    float* f[2] = {nullptr, nullptr};
    float* g[2] = {nullptr, nullptr};
    float* h[2] = {nullptr, nullptr};
    float2* gm[2] = {nullptr, nullptr};
    float2* hm[2] = {nullptr, nullptr};
    float* hist = nullptr;
    float2* mom = nullptr;      // phi, psi of the current step (2 N float2)
    float* pot = nullptr;       // mu_phi, mu_psi, R_phi free, R_psi free (4 N)
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    Rec* recs = nullptr;        // [0], [1] by step parity, [2] diagnostic, [3] zeros
    double* out = nullptr;      // 6 N doubles (diagnostic read-back), on first use
    size_t bytes = 0;
    std::string err = "no error";
};

namespace {

slbm_status fail3(slbm3d_domain* d, slbm_status s, const std::string& m) {
    if (d) d->err = m; else g_err3 = m;
    return s;
}

slbm_status cuda_fail3(slbm3d_domain* d, cudaError_t e, const char* what) {
    cudaGetLastError();
    return fail3(d, SLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class P>
cudaError_t alloc3(slbm3d_domain* d, P** ptr, size_t bytes) {
    cudaError_t e = slbm_device_malloc((void**)ptr, bytes);
    if (e == cudaSuccess) d->bytes += bytes;
    else *ptr = nullptr;
    return e;
}

Args3 make_args3(slbm3d_domain* d, bool diag) {
    Args3 a;
    std::memset(&a, 0, sizeof(a));
    const int i = d->cur, o = d->cur ^ 1;
    a.g = d->G;
    a.f_in = d->f[i]; a.g_in = d->g[i]; a.gm_in = d->gm[i]; a.h_in = d->h[i]; a.hm_in = d->hm[i];
    a.f_out = d->f[o]; a.g_out = d->g[o]; a.gm_out = d->gm[o]; a.h_out = d->h[o]; a.hm_out = d->hm[o];
    a.hist = d->hist;
    const long long N = d->G.N;
    a.phi = d->mom; a.psi = d->mom + N;
    a.mu_phi = d->pot; a.mu_psi = d->pot + N; a.rf_phi = d->pot + 2 * N; a.rf_psi = d->pot + 3 * N;
    a.partials = d->partials;
    a.counter = d->counter;
    a.rec_prev = d->n == 0 ? d->recs + 3 : d->recs + ((d->n - 1) & 1);
    a.rec = diag ? d->recs + 2 : d->recs + (d->n & 1);
    a.first = d->n == 0;
    a.P = d->core.phys;
    return a;
}

cudaError_t launch_level(slbm3d_domain* d, bool diag) {
    Args3 a = make_args3(d, diag);
    cudaStream_t st = d->core.stream;
    moments3d<<<d->grid[0], T3, 0, st>>>(a);
    potentials3d<<<d->grid[1], T3, 0, st>>>(a, diag ? 1 : 0);
    if (diag) {
        if (d->out) {
            for (int q = 0; q < 6; ++q) a.o[q] = d->out + (long long)q * d->G.N;
        }
        collide3d<true><<<d->grid[1], T3, 0, st>>>(a);
    } else {
        collide3d<false><<<d->grid[2], T3, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

slbm_status slbm3d_create_domain(const slbm_params* p, int nz, void* stream, slbm3d_domain** out) {
    if (!out) return fail3(nullptr, SLBM_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why = slbm_validate_params(p);
    if (why.empty()) {
        if (nz < 1) why = "nz must be >= 1";
        else if ((long long)p->nx * p->ny * nz > (1LL << 27)) why = "grid larger than 2^27 cells";
        else if (p->precision != SLBM_FP32) why = "the 3D extension stores FP32";
        else if (p->rho_l != p->rho_g || (p->tau_f_gas > 0 && p->tau_f_gas != p->tau_f))
            why = "the 3D extension has uniform density and viscosity";
        else if (p->multiplier != SLBM_MULT_PAPER && p->multiplier != SLBM_MULT_TARGET)
            why = "the 3D extension has the PAPER and TARGET multipliers";
        else
            for (int i = 0; i < 4; ++i)
                if (p->mrt_f[i] != 0 || p->mrt_g[i] != 0 || p->mrt_h[i] != 0) why = "the 3D extension collides with one relaxation time";
    }
    if (!why.empty()) return fail3(nullptr, SLBM_EINVAL, why);
    slbm3d_domain* d = new (std::nothrow) slbm3d_domain();
    if (!d) return fail3(nullptr, SLBM_ENOMEM, "host allocation failed");
    d->core.p = *p;
    d->core.stream = (cudaStream_t)stream;
    d->nz = nz;
    d->G = Grid3{p->nx, p->ny, nz, (long long)p->nx * p->ny * nz};
    d->core.N = d->G.N;
    slbm_derive_phys(&d->core);
    d->core.phys.Nd = (double)d->G.N;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // persistent grids: the resident blocks of each kernel, at most one block per row segment
    const long long segs = (long long)((p->nx + T3 - 1) / T3) * p->ny * nz;
    const void* fns[3] = {(const void*)moments3d, (const void*)potentials3d, (const void*)collide3d<false>};
    int maxgrid = 1;
    for (int k = 0; k < 3; ++k) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fns[k], T3, 0) != cudaSuccess || per < 1) per = 1;
        const long long g = (long long)per * sms;
        d->grid[k] = (int)(g < segs ? g : segs);
        if (d->grid[k] > maxgrid) maxgrid = d->grid[k];
    }
    cudaGetLastError();
    const size_t N = (size_t)d->G.N;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = alloc3(d, &d->f[b], Q3 * N * 4);
        if (e == cudaSuccess) e = alloc3(d, &d->g[b], (Q3 - 1) * N * 4);
        if (e == cudaSuccess) e = alloc3(d, &d->h[b], (Q3 - 1) * N * 4);
        if (e == cudaSuccess) e = alloc3(d, &d->gm[b], N * sizeof(float2));
        if (e == cudaSuccess) e = alloc3(d, &d->hm[b], N * sizeof(float2));
    }
    if (e == cudaSuccess) e = alloc3(d, &d->hist, 8 * N * 4);
    if (e == cudaSuccess) e = alloc3(d, &d->mom, 2 * N * sizeof(float2));
    if (e == cudaSuccess) e = alloc3(d, &d->pot, 4 * N * 4);
    if (e == cudaSuccess) e = alloc3(d, &d->partials, (size_t)maxgrid * NPART * sizeof(double));
    if (e == cudaSuccess) e = alloc3(d, &d->counter, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = alloc3(d, &d->recs, 4 * sizeof(Rec));
    if (e == cudaSuccess) e = cudaMemsetAsync(d->counter, 0, 2 * sizeof(unsigned int), d->core.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->recs, 0, 4 * sizeof(Rec), d->core.stream);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        slbm3d_destroy(d);
        return fail3(nullptr, oom ? SLBM_ENOMEM : SLBM_ECUDA, std::string("device state: ") + cudaGetErrorString(e));
    }
    *out = d;
    return SLBM_OK;
}

slbm_status slbm3d_set_walls(slbm3d_domain* d, int wall, double theta0_deg, double beta_sg, double beta_sl, double u_x) {
    if (!d) return SLBM_EINVAL;
    if (wall < 0 || wall > 1) return fail3(d, SLBM_EINVAL, "wall must be 0 (bottom) or 1 (top)");
    if (!(theta0_deg > 0 && theta0_deg < 180)) return fail3(d, SLBM_EINVAL, "theta0 must lie in (0, 180) degrees");
    if (!(beta_sg >= 0) || !(beta_sl >= 0)) return fail3(d, SLBM_EINVAL, "adsorption elasticities must be >= 0");
    if (!(std::fabs(u_x) < 0.3)) return fail3(d, SLBM_EINVAL, "|u_x| must be below 0.3 (lattice units)");
    d->core.wall_theta[wall] = theta0_deg;
    d->core.wall_bsg[wall] = beta_sg;
    d->core.wall_bsl[wall] = beta_sl;
    d->core.wall_u[wall] = u_x;
    slbm_wall_phys(&d->core, wall);
    return SLBM_OK;
}

slbm_status slbm3d_init_fields(slbm3d_domain* d, const double* phi, const double* psi) {
    if (!d || !phi) return d ? fail3(d, SLBM_EINVAL, "phi is NULL") : SLBM_EINVAL;
    if (d->core.p.psi_on && !psi) return fail3(d, SLBM_EINVAL, "psi is NULL while psi_on = 1");
    const size_t bytes = (size_t)d->G.N * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (!d->out) e = alloc3(d, &d->out, 6 * bytes);
    if (e != cudaSuccess) return cuda_fail3(d, e, "field buffer");
    cudaStream_t st = d->core.stream;
    e = cudaMemcpyAsync(d->out, phi, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d->core.p.psi_on) e = cudaMemcpyAsync(d->out + d->G.N, psi, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail3(d, e, "init copy");
    d->cur = 0;
    d->n = 0;
    const unsigned blocks = (unsigned)((d->G.N + 255) / 256);
    init3d<<<blocks, 256, 0, st>>>(d->G, d->out, d->out + d->G.N, d->core.p.psi_on, d->core.p.eta_phi,
                                   d->core.p.eta_psi, d->core.p.rho_l, d->core.wall_u[0], d->core.wall_u[1], d->f[0],
                                   d->g[0], d->gm[0], d->h[0], d->hm[0], d->hist);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(d->recs, 0, 4 * sizeof(Rec), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail3(d, e, "init");
    d->initialised = true;
    return SLBM_OK;
}

slbm_status slbm3d_step(slbm3d_domain* d, long long nsteps) {
    if (!d) return SLBM_EINVAL;
    if (nsteps < 0) return fail3(d, SLBM_EINVAL, "nsteps must be >= 0");
    if (!d->initialised) return fail3(d, SLBM_ESTATE, "fields not initialised");
    for (long long s = 0; s < nsteps; ++s) {
        cudaError_t e = launch_level(d, false);
        if (e != cudaSuccess) return cuda_fail3(d, e, "step launch");
        d->cur ^= 1;
        ++d->n;
    }
    return SLBM_OK;
}

slbm_status slbm3d_read_fields(slbm3d_domain* d, double* phi, double* psi, double* ux, double* uy, double* uz,
                               double* p) {
    if (!d) return SLBM_EINVAL;
    if (!d->initialised) return fail3(d, SLBM_ESTATE, "fields not initialised");
    cudaError_t e = launch_level(d, true);
    if (e != cudaSuccess) return cuda_fail3(d, e, "diagnostic launch");
    double* host[6] = {phi, psi, ux, uy, uz, p};
    const size_t bytes = (size_t)d->G.N * sizeof(double);
    for (int q = 0; q < 6 && e == cudaSuccess; ++q)
        if (host[q]) e = cudaMemcpyAsync(host[q], d->out + (long long)q * d->G.N, bytes, cudaMemcpyDeviceToHost, d->core.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->core.stream);
    if (e != cudaSuccess) return cuda_fail3(d, e, "read_fields");
    return SLBM_OK;
}

slbm_status slbm3d_read_totals(slbm3d_domain* d, slbm_totals* t) {
    if (!d || !t) return d ? fail3(d, SLBM_EINVAL, "totals is NULL") : SLBM_EINVAL;
    if (!d->initialised) return fail3(d, SLBM_ESTATE, "fields not initialised");
    cudaError_t e = launch_level(d, true);
    Rec r;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, d->recs + 2, sizeof(Rec), cudaMemcpyDeviceToHost, d->core.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->core.stream);
    if (e != cudaSuccess) return cuda_fail3(d, e, "read_totals");
    std::memset(t, 0, sizeof(*t));
    t->step = d->n;
    t->Q_phi = r.Q;
    t->H = r.H;
    t->phi_total = r.phi_tot;
    t->psi_total = r.psi_tot;
    t->lambda_phi = r.lam;
    t->mubar_psi = (d->core.p.psi_on && d->core.p.M_psi > 0) ? r.mpsi_mubar / d->core.p.M_psi : 0.0;
    t->kinetic = r.kin;
    t->S1 = r.S1;
    t->S2 = r.S2;
    t->clamp_count = (long long)r.clamps;
    t->range_count = (long long)r.range;
    const double vals[] = {r.Q, r.H, r.phi_tot, r.psi_tot, r.lam, r.kin};
    for (double v : vals)
        if (!std::isfinite(v)) return fail3(d, SLBM_EUNSTABLE, "a reduced total is not finite");
    if (t->range_count > 0) return fail3(d, SLBM_EUNSTABLE, "a velocity, phi or p left its range");
    return SLBM_OK;
}

size_t slbm3d_device_bytes(const slbm3d_domain* d) { return d ? d->bytes : 0; }

void slbm3d_destroy(slbm3d_domain* d) {
    if (!d) return;
    void* bufs[] = {d->f[0], d->f[1], d->g[0], d->g[1], d->h[0], d->h[1], d->gm[0], d->gm[1], d->hm[0], d->hm[1],
                    d->hist, d->mom, d->pot, d->partials, d->counter, d->recs, d->out};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete d;
}

const char* slbm3d_last_error(const slbm3d_domain* d) { return d ? d->err.c_str() : g_err3.c_str(); }

}  // extern "C"
