// C-ABI implementation of include/surflbm.h: parameter derivation, device state,
// initialisation kernel and launches of the fused step kernel.
#include "surflbm.h"
#include "surflbm_step.cuh"

#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>

using namespace slbm;

namespace {

std::string g_create_error = "no error";
constexpr double CS2 = 1.0 / 3.0;

struct InitArgs {
    int nx, ny;
    long long N;
    const double* phi0;
    const double* psi0;
    double eta_phi, eta_psi, rho_l, rho_g, inv_phi_b;
    double uw[2];
    double u0x;          // uniform initial velocity (x), 0 except in the manufactured-solution test
    int psi_on;
};

// Pre-collision populations at time 0 = equilibria at rest of the initial fields.  The
// stored state is post-collision (the kernel pulls), so each population is set to the
// equilibrium of the node it will stream to: g*_k(y) = w_k eta phi0(target(y, k)), with
// the target y + c_k, or the specular partner (y_x + c_kx, y_y) for a wall link; flow
// populations are 0 except on moving-wall links, which carry the inverse of the
// moving-wall term so the first pull yields f = 0.
template <class T>
__global__ void init_kernel(InitArgs a, T* f, T* gd, float2* gm, T* hd, float2* hm, float* php) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.N) return;
    const int x = (int)(c % a.nx), y = (int)(c / a.nx);
    for (int set = 0; set < 2; ++set) {
        const double* F = set == 0 ? a.phi0 : a.psi0;
        const double eta = set == 0 ? a.eta_phi : a.eta_psi;
        T* d = set == 0 ? gd : hd;
        float2* m = set == 0 ? gm : hm;
        double gk[9];
        const double fc = (set == 1 && !a.psi_on) ? 0.0 : F[c];
        gk[0] = (1.0 - (1.0 - WkD(0)) * eta) * fc;
        double msum = gk[0];
        for (int k = 1; k < 9; ++k) {
            int tx = x + CXk(k), ty = y + CYk(k);
            if (ty < 0 || ty >= a.ny) ty = y;
            tx = wrapx(tx, a.nx);
            const double ft = (set == 1 && !a.psi_on) ? 0.0 : F[(long long)ty * a.nx + tx];
            // w_k (eta c + c_k . (c u) / c_s^2) at the target; u = (u0x, 0) keeps it the same
            // for the specular partner of a wall link
            gk[k] = WkD(k) * (eta + 3.0 * CXk(k) * a.u0x) * ft;
            msum += gk[k];
        }
        float2 mv;
        mv.x = (float)msum;
        mv.y = (float)(msum - (double)mv.x);
        m[c] = mv;
        for (int k = 1; k < 9; ++k) Stor<T>::st(d, (long long)(k - 1) * a.N + c, (float)(gk[k] - (double)Wk(k) * mv.x));
    }
    // flow: the equilibrium f^eq_k(rho, u0) (p = 0) of the node the population streams to;
    // a link into a wall stores what the moving-wall bounce-back turns into f^eq of the
    // opposite direction at this node
    auto rho_at = [&](long long i) {
        return a.rho_g + (a.rho_l - a.rho_g) * fmin(fmax(0.5 * (a.phi0[i] * a.inv_phi_b + 1.0), 0.0), 1.0);
    };
    auto feq = [&](int k, double rho) {
        const double cu = CXk(k) * a.u0x;
        return WkD(k) * rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * a.u0x * a.u0x);
    };
    for (int k = 0; k < 9; ++k) {
        double v;
        const int ty = y + CYk(k);
        if (ty < 0 || ty >= a.ny) {
            const double rho = rho_at(c);
            v = feq(OPPk(k), rho) + 6.0 * WkD(k) * rho * CXk(k) * a.uw[ty < 0 ? 0 : 1];
        } else {
            v = feq(k, rho_at((long long)ty * a.nx + wrapx(x + CXk(k), a.nx)));
        }
        Stor<T>::st(f, (long long)k * a.N + c, (float)v);
    }
    php[c] = (float)a.phi0[c];
}

size_t elem_size(int prec) { return prec == SLBM_FP32 ? 4 : 2; }

}  // namespace

#include "surflbm_internal.cuh"

namespace {

slbm_status fail(slbm_domain* d, slbm_status s, const std::string& msg) {
    if (d) d->err = msg; else g_create_error = msg;
    return s;
}

slbm_status cuda_fail(slbm_domain* d, cudaError_t e, const char* what) {
    return fail(d, SLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

std::string validate(const slbm_params* p) {
    if (!p) return "params is NULL";
    if (p->nx < 1 || p->ny < 2) return "need nx >= 1 and ny >= 2";
    if ((long long)p->nx * p->ny > (1LL << 28)) return "grid larger than 2^28 cells";
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5) || !(p->tau_h > 0.5)) return "relaxation times must exceed 0.5";
    if (p->tau_f_gas > 0 && !(p->tau_f_gas > 0.5)) return "tau_f_gas must exceed 0.5";
    for (int i = 0; i < 4; ++i)
        if (p->mrt_f[i] < 0 || p->mrt_f[i] >= 2 || p->mrt_g[i] < 0 || p->mrt_g[i] >= 2 || p->mrt_h[i] < 0 ||
            p->mrt_h[i] >= 2)
            return "MRT rates must lie in [0, 2)";
    if (!(p->eps > 0)) return "eps must be positive";
    if (!(p->sigma >= 0)) return "sigma must be >= 0";
    if (!(p->psi_b >= 0 && p->psi_b < 1)) return "psi_b must lie in [0, 1)";
    if (!(p->M_psi >= 0) || !(p->M_phi >= 0)) return "mobilities must be >= 0";
    if (!(p->eta_phi > 0) || !(p->eta_psi > 0)) return "eta must be positive";
    if (!(p->rho_l > 0) || !(p->rho_g > 0)) return "densities must be positive";
    if (p->constraint != SLBM_CONSTRAINT_NONLINEAR && p->constraint != SLBM_CONSTRAINT_LINEAR) return "bad constraint";
    if (p->multiplier != SLBM_MULT_PAPER && p->multiplier != SLBM_MULT_TARGET && p->multiplier != SLBM_MULT_EXACT)
        return "bad multiplier";
    if (p->precision < SLBM_FP32 || p->precision > SLBM_BF16DEV) return "bad precision";
    if (p->wall_saturation != 0 && p->wall_saturation != 1) return "wall_saturation must be 0 or 1";
    if (p->staging != SLBM_STAGING_CPASYNC && p->staging != SLBM_STAGING_TMA) return "bad staging";
    return "";
}

void set_wall_phys(slbm_domain* d, int w) {
    const double c = std::cos(d->wall_theta[w] * M_PI / 180.0);
    const double sg = d->p.sigma * (16.0 / 15.0 + c) / 2.0;
    const double sl = d->p.sigma * (16.0 / 15.0 - c) / 2.0;
    d->phys.wcos[w] = (float)(d->p.sigma * c);
    d->phys.wSg[w] = (float)(sg * d->wall_bsg[w]);
    d->phys.wSl[w] = (float)(sl * d->wall_bsl[w]);
    d->phys.wS0g[w] = (float)sg;
    d->phys.wS0l[w] = (float)sl;
    const bool sat = d->p.wall_saturation != 0;
    d->phys.wLg[w] = (sat && d->wall_bsg[w] > 0.0) ? (float)(-0.5 / d->wall_bsg[w]) : -1e30f;
    d->phys.wLl[w] = (sat && d->wall_bsl[w] > 0.0) ? (float)(-0.5 / d->wall_bsl[w]) : -1e30f;
    d->phys.uw[w] = (float)d->wall_u[w];
}

void derive(slbm_domain* d) {
    const slbm_params& p = d->p;
    d->beta = 3.0 * p.sigma / (4.0 * p.eps);
    d->kappa = 3.0 * p.eps * p.sigma / 8.0;
    d->lambda_s = p.lambda_s < 0 ? d->kappa / 2.0 : p.lambda_s;
    d->W = p.Ex > 0 ? 4.0 * d->beta / p.Ex : 0.0;
    d->kT = 4.0 * d->beta * p.Pi;
    if (p.phi_b > 0) d->phi_b = p.phi_b;
    else if (d->beta > 0 && p.psi_b > 0) d->phi_b = std::sqrt(1.0 - d->W * p.psi_b / (4.0 * d->beta * (1.0 - p.psi_b)));
    else d->phi_b = 1.0;
    d->M_phi = d->kappa > 0 ? p.eta_phi * CS2 * (p.tau_g - 0.5) / d->kappa : p.M_phi;
    d->M_0 = p.eta_psi * CS2 * (p.tau_h - 0.5) - p.M_psi * d->lambda_s;
    Phys& P = d->phys;
    std::memset(&P, 0, sizeof(P));
    P.beta = (float)d->beta; P.kappa = (float)d->kappa; P.lambda_s = (float)d->lambda_s; P.W = (float)d->W;
    P.kT = (float)d->kT; P.phi_b = (float)d->phi_b; P.inv_phi_b = (float)(1.0 / d->phi_b);
    P.M_phi = (float)d->M_phi; P.M_psi = (float)p.M_psi; P.M_0 = (float)d->M_0;
    P.eta_phi = (float)p.eta_phi; P.eta_psi = (float)p.eta_psi;
    P.rho_l = (float)p.rho_l; P.rho_g = (float)p.rho_g;
    const double nu_l = CS2 * (p.tau_f - 0.5);
    const double nu_g = CS2 * ((p.tau_f_gas > 0 ? p.tau_f_gas : p.tau_f) - 0.5);
    P.nu_l = (float)nu_l; P.nu_g = (float)nu_g; P.var_nu = nu_l != nu_g;
    P.Gx = (float)p.Gx; P.Gy = (float)p.Gy;
    // rates: (s0, s1, s2, s3, s4); 0 means "equal to the main rate"
    P.sf[0] = (float)p.mrt_f[0]; P.sf[1] = (float)p.mrt_f[1]; P.sf[2] = (float)(1.0 / p.tau_f);
    P.sf[3] = (float)p.mrt_f[2]; P.sf[4] = (float)p.mrt_f[3];
    P.sg[0] = (float)p.mrt_g[0]; P.sg[1] = (float)(1.0 / p.tau_g); P.sg[2] = (float)p.mrt_g[1];
    P.sg[3] = (float)p.mrt_g[2]; P.sg[4] = (float)p.mrt_g[3];
    P.sh[0] = (float)p.mrt_h[0]; P.sh[1] = (float)(1.0 / p.tau_h); P.sh[2] = (float)p.mrt_h[1];
    P.sh[3] = (float)p.mrt_h[2]; P.sh[4] = (float)p.mrt_h[3];
    P.mrt_f = p.mrt_f[0] != 0 || p.mrt_f[1] != 0 || p.mrt_f[2] != 0 || p.mrt_f[3] != 0;
    P.mrt_g = p.mrt_g[0] != 0 || p.mrt_g[1] != 0 || p.mrt_g[2] != 0 || p.mrt_g[3] != 0;
    P.mrt_h = p.mrt_h[0] != 0 || p.mrt_h[1] != 0 || p.mrt_h[2] != 0 || p.mrt_h[3] != 0;
    P.psi_clamp = 1e-12f;
    P.psi_on = p.psi_on != 0;
    P.linear = p.constraint == SLBM_CONSTRAINT_LINEAR;
    // the exact root is sought from the target estimate, which also makes the step
    // kernel reduce H (and so H0 on the first step)
    P.target = p.multiplier == SLBM_MULT_TARGET || p.multiplier == SLBM_MULT_EXACT;
    P.Nd = (double)p.nx * (double)p.ny;
    P.M_phi_d = d->M_phi;
    P.M_psi_d = p.M_psi;
    for (int w = 0; w < 2; ++w) set_wall_phys(d, w);
}

template <class T>
StepArgs<T> make_args(slbm_domain* d, bool diag) {
    StepArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    const int i = d->cur, o = d->cur ^ 1;
    a.nx = d->p.nx; a.ny = d->p.ny; a.N = d->N; a.total = d->total; a.band_h = d->band_h;
    a.f_in = (const T*)d->f[i]; a.gd_in = (const T*)d->gd[i]; a.gm_in = d->gm[i];
    a.hd_in = (const T*)d->hd[i]; a.hm_in = d->hm[i]; a.php_in = d->php[i];
    a.f_out = (T*)d->f[o]; a.gd_out = (T*)d->gd[o]; a.gm_out = d->gm[o];
    a.hd_out = (T*)d->hd[o]; a.hm_out = d->hm[o]; a.php_out = d->php[o];
    a.hist = (T*)d->hist;
    a.partials = d->partials;
    a.counter = d->counter;
    a.err = d->counter + 1;
    a.rec_prev = d->n == 0 ? d->recs + 3 : d->recs + ((d->n - 1) & 1);
    a.rec_out = diag ? d->recs + 2 : d->recs + (d->n & 1);
    a.first = d->n == 0;
    a.level = d->n;
    if (diag && d->fields) {
        a.o_phi = d->fields; a.o_psi = d->fields + d->N; a.o_ux = d->fields + 2 * d->N;
        a.o_uy = d->fields + 3 * d->N; a.o_p = d->fields + 4 * d->N;
    }
    a.P = d->phys;
    return a;
}

template <class T>
cudaError_t prepare_kernels() {
    static PerDeviceOnce once;
    return once([] {
        const int sm = (int)smem_bytes<T>(), st = (int)smem_bytes_tma<T>();
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(step_kernel<T, false, false, false>, attr, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, true, false, false>, attr, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, false, true, false>, attr, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, true, true, false>, attr, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, false, false, false, true>, attr, st);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, true, false, false, true>, attr, st);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, false, true, false, true>, attr, st);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, true, true, false, true>, attr, st);
        if constexpr (std::is_same<T, float>::value) {
            if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, false, false, false, false, true>, attr, sm);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, true, false, false, false, true>, attr, sm);
        }
        return e;
    });
}

// one launch of the step (or of its diagnostic pass) with the arguments a
template <class T>
cudaError_t launch_with(slbm_domain* d, const StepArgs<T>& a, bool diag) {
    cudaError_t e = prepare_kernels<T>();
    if (e != cudaSuccess) return e;
    // uniform density and viscosity (the common case) drop every density-gradient term
    const bool var = a.P.var_nu || a.P.rho_l != a.P.rho_g;
    const BatchArgs nb{};
    if constexpr (std::is_same<T, float>::value) {
        if (d->mms) {
            static const TmaMaps none{};
            const size_t sm = smem_bytes<T>();
            if (diag) step_kernel<T, true, false, false, false, true><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, none);
            else step_kernel<T, false, false, false, false, true><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, none);
            return cudaGetLastError();
        }
    }
    if (d->tma) {
        const size_t sm = smem_bytes_tma<T>();
        const TmaMaps& m = d->maps[d->cur];
        if (diag) {
            if (var) step_kernel<T, true, true, false, true><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, m);
            else step_kernel<T, true, false, false, true><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, m);
        } else {
            if (var) step_kernel<T, false, true, false, true><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, m);
            else step_kernel<T, false, false, false, true><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, m);
        }
    } else {
        const size_t sm = smem_bytes<T>();
        static const TmaMaps none{};
        if (diag) {
            if (var) step_kernel<T, true, true, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, none);
            else step_kernel<T, true, false, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, none);
        } else {
            if (var) step_kernel<T, false, true, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, none);
            else step_kernel<T, false, false, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, nb, none);
        }
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_step(slbm_domain* d, bool diag) {
    return launch_with<T>(d, make_args<T>(d, diag), diag);
}

template <class T>
int resident_ctas_per_sm(bool tma) {
    int n = 0;
    if (prepare_kernels<T>() != cudaSuccess) return 1;
    const cudaError_t e = tma ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<T, false, false, false, true>,
                                                                           NTHREADS, smem_bytes_tma<T>())
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<T, false, false, false>,
                                                                           NTHREADS, smem_bytes<T>());
    if (e != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// Persistent grid: one CTA per resident slot, unless the grid is so small that a CTA
// would get fewer than 16 strip rows (the 6-row prologue is paid per piece).
int choose_ctas(slbm_domain* d, int ctas_per_sm) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long slots = (long long)sms * ctas_per_sm;
    long long n = (d->total + 15) / 16;
    if (n > slots) n = slots;
    if (n < 1) n = 1;
    return (int)n;
}

// Band-major split.  The strip-major ranges of choose_ctas balance the rows to within one,
// but the CTAs of neighbouring strips march different rows at any moment, so the halo
// columns a strip stages (whole DRAM bursts that the neighbouring strip also reads) are
// fetched from DRAM twice.  Pieces (band of H rows, strip) taken round-robin, band by band,
// put the CTAs of neighbouring strips on the same rows at the same time, and the second
// read of a halo burst hits L2 (measured at 4096 x 2048: 1.25 instead of 1.97 GB read per
// step).  Chosen when its cost, in rows per CTA plus a prologue per piece, is within
// BAND_SLACK of the strip-major cost; H at least 16 rows.
constexpr double BAND_SLACK = 1.05;
constexpr int PROLOGUE_ROWS = 2;
void choose_bands(slbm_domain* d, int ctas_per_sm) {
    d->band_h = 0;
    const int ny = d->p.ny;
    const int strips = (int)(d->total / ny);
    if (strips < 2 || ny < 32) return;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long slots = (long long)sms * ctas_per_sm;
    const long long g0 = d->grid.x;
    // strip-major: a CTA marches ceil(total / grid) rows in at most two pieces
    const double cost_s = (double)((d->total + g0 - 1) / g0) + 2 * PROLOGUE_ROWS;
    double best = 0.0;
    int best_h = 0;
    long long best_g = 0;
    for (int nb = 2; nb <= ny / 16; ++nb) {
        const int H = (ny + nb - 1) / nb;
        const long long pieces = (long long)((ny + H - 1) / H) * strips;
        const long long g = pieces < slots ? pieces : slots;
        const long long rounds = (pieces + g - 1) / g;
        const double cost = (double)rounds * (H + PROLOGUE_ROWS);
        if (best_h == 0 || cost < best) {
            best = cost;
            best_h = H;
            best_g = g;
        }
    }
    if (best_h > 0 && best <= BAND_SLACK * cost_s) {
        d->band_h = best_h;
        d->grid = dim3((unsigned)best_g);
    }
}

// ---- tensor maps of the TMA staging (driver entry point looked up once, no libcuda link)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// a map of rank 2 or 3 over `base` (element bytes es), dims/box innermost first
bool encode_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                const cuuint32_t* box, int es) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    return fn(m, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// TMA staging: whole strips (nx a multiple of TX, so that only the two seam strips have
// window columns outside [0, nx), exactly WOFF of them) and at least two strips
bool tma_eligible(const slbm_params& p) { return p.staging == SLBM_STAGING_TMA && p.nx % TX == 0 && p.nx >= 2 * TX; }

bool build_maps(slbm_domain* d) {
    const int es = (int)elem_size(d->p.precision);
    const cuuint64_t nx = (cuuint64_t)d->p.nx, ny = (cuuint64_t)d->p.ny, N = (cuuint64_t)d->N;
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        TmaMaps& m = d->maps[b];
        std::memset(&m, 0, sizeof(m));
        {
            const cuuint64_t dims[3] = {nx, ny, 8}, str[2] = {nx * es, N * es};
            const cuuint32_t box[3] = {(cuuint32_t)WW, (cuuint32_t)RB, 8};
            ok = ok && encode_map(&m.dev[0], d->gd[b], 3, dims, str, box, es);
            ok = ok && encode_map(&m.dev[1], d->hd[b], 3, dims, str, box, es);
        }
        {
            const cuuint64_t dims[2] = {2 * nx, ny}, str[1] = {2 * nx * 4};
            const cuuint32_t box[2] = {(cuuint32_t)(2 * WW), (cuuint32_t)RB};
            ok = ok && encode_map(&m.mom[0], d->gm[b], 2, dims, str, box, 4);
            ok = ok && encode_map(&m.mom[1], d->hm[b], 2, dims, str, box, 4);
        }
        {
            const cuuint64_t dims[2] = {nx, ny}, str[1] = {nx * 4};
            const cuuint32_t box[2] = {(cuuint32_t)WW, (cuuint32_t)RB};
            ok = ok && encode_map(&m.php, d->php[b], 2, dims, str, box, 4);
        }
        {
            const cuuint64_t dims[3] = {nx, ny, 9}, str[2] = {nx * es, N * es};
            const cuuint32_t box[3] = {(cuuint32_t)WW, (cuuint32_t)RB, 1};
            ok = ok && encode_map(&m.f, d->f[b], 3, dims, str, box, es);
        }
    }
    return ok;
}

cudaError_t launch(slbm_domain* d, bool diag) {
    switch (d->p.precision) {
        case SLBM_FP16DEV: return launch_step<__half>(d, diag);
        case SLBM_BF16DEV: return launch_step<__nv_bfloat16>(d, diag);
        default: return launch_step<float>(d, diag);
    }
}

template <class T>
cudaError_t launch_init(slbm_domain* d, const double* phi0, const double* psi0) {
    InitArgs a;
    a.nx = d->p.nx; a.ny = d->p.ny; a.N = d->N;
    a.phi0 = phi0; a.psi0 = psi0;
    a.eta_phi = d->p.eta_phi; a.eta_psi = d->p.eta_psi;
    a.rho_l = d->p.rho_l; a.rho_g = d->p.rho_g; a.inv_phi_b = 1.0 / d->phi_b;
    a.uw[0] = d->wall_u[0]; a.uw[1] = d->wall_u[1];
    a.u0x = d->mms ? d->mms_u0x : 0.0;
    a.psi_on = d->p.psi_on != 0;
    const int c = d->cur;
    const unsigned blocks = (unsigned)((d->N + 255) / 256);
    init_kernel<T><<<blocks, 256, 0, d->stream>>>(a, (T*)d->f[c], (T*)d->gd[c], d->gm[c], (T*)d->hd[c], d->hm[c],
                                                  d->php[c]);
    return cudaGetLastError();
}

template <class P>
slbm_status dalloc(slbm_domain* d, P** ptr, size_t bytes) {
    if (d->ext) {
        // carve from the caller's workspace (ws == nullptr: count only, for slbm_workspace_bytes)
        const size_t off = (d->ws_off + 255) & ~(size_t)255;
        if (off + bytes > d->ws_size) {
            *ptr = nullptr;
            return fail(d, SLBM_ENOMEM, "workspace too small: need " + std::to_string(off + bytes) + " bytes, have " +
                                            std::to_string(d->ws_size));
        }
        *ptr = d->ws ? (P*)(d->ws + off) : nullptr;
        d->ws_off = off + bytes;
        d->bytes += bytes;
        return SLBM_OK;
    }
    cudaError_t e = slbm_device_malloc((void**)ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(d, SLBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    d->bytes += bytes;
    return SLBM_OK;
}

// Grid of the step kernel and the sizes that depend on it (current device).
void plan_domain(slbm_domain* d) {
    const slbm_params* p = &d->p;
    int per_sm = 1;
    const bool tma = tma_eligible(*p) && encode_fn() != nullptr;
    switch (p->precision) {
        case SLBM_FP16DEV: per_sm = resident_ctas_per_sm<__half>(tma); break;
        case SLBM_BF16DEV: per_sm = resident_ctas_per_sm<__nv_bfloat16>(tma); break;
        default: per_sm = resident_ctas_per_sm<float>(tma); break;
    }
    d->total = (long long)((p->nx + TX - 1) / TX) * p->ny;
    d->grid = dim3((unsigned)choose_ctas(d, per_sm));
    choose_bands(d, per_sm);
    if (p->multiplier == SLBM_MULT_EXACT) d->exact_blocks = exact_multiplier_blocks(p->precision, d->N);
}

// Every device buffer of a domain, in a fixed order (the workspace layout of
// slbm_create_domain_ext); the 5 N-double field buffer only when with_fields.
slbm_status alloc_state(slbm_domain* d, bool with_fields) {
    const size_t es = elem_size(d->p.precision);
    const size_t N = (size_t)d->N;
    slbm_status s = SLBM_OK;
    for (int b = 0; b < 2 && s == SLBM_OK; ++b) {
        if ((s = dalloc(d, &d->f[b], 9 * N * es))) break;
        if ((s = dalloc(d, &d->gd[b], 8 * N * es))) break;
        if ((s = dalloc(d, &d->hd[b], 8 * N * es))) break;
        if ((s = dalloc(d, &d->gm[b], N * sizeof(float2)))) break;
        if ((s = dalloc(d, &d->hm[b], N * sizeof(float2)))) break;
        if ((s = dalloc(d, &d->php[b], N * sizeof(float)))) break;
    }
    size_t nblocks = (size_t)d->grid.x * d->grid.y;
    if ((size_t)d->exact_blocks > nblocks) nblocks = (size_t)d->exact_blocks;
    if (s == SLBM_OK) s = dalloc(d, &d->hist, 6 * N * es);
    if (s == SLBM_OK) s = dalloc(d, &d->partials, nblocks * NPART * sizeof(double));
    if (s == SLBM_OK) s = dalloc(d, &d->counter, 2 * sizeof(unsigned int));
    if (s == SLBM_OK) s = dalloc(d, &d->recs, 4 * sizeof(Rec));
    if (s == SLBM_OK && with_fields) s = dalloc(d, &d->fields, 5 * N * sizeof(double));
    return s;
}

// ---- scratch of slbm_read_fields_noalloc: static device memory, no allocation
static_assert(sizeof(Rec) <= 256, "record must fit the scratch tail");
static_assert(NPART == SLBM_NOALLOC_PARTS, "partial slots of the static scratch");
static __device__ __align__(256) unsigned char g_noalloc_scratch[SLBM_NOALLOC_SCRATCH_BYTES];

// device address of g_noalloc_scratch, looked up once per device with that device current
cudaError_t noalloc_scratch(unsigned char** out) {
    static std::mutex mtx;
    static unsigned char* addr[128] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mtx);
    if (!addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = (unsigned char*)ptr;
    }
    *out = addr[dev];
    return cudaSuccess;
}

template <class T>
cudaError_t launch_diag_noalloc(slbm_domain* d, unsigned char* scratch, double* o[5]) {
    StepArgs<T> a = make_args<T>(d, true);
    a.partials = (double*)scratch;
    a.counter = (unsigned int*)(scratch + SLBM_NOALLOC_MAX_CTAS * NPART * 8);
    a.err = a.counter + 1;
    a.rec_out = (Rec*)(scratch + SLBM_NOALLOC_MAX_CTAS * NPART * 8 + 256);
    a.o_phi = o[0]; a.o_psi = o[1]; a.o_ux = o[2]; a.o_uy = o[3]; a.o_p = o[4];
    return launch_with<T>(d, a, true);
}

// the step's error bits (a bounded TMA wait that ran out); call after a stream sync
slbm_status check_err_word(slbm_domain* d, const unsigned int* word) {
    unsigned int bits = 0;
    cudaError_t e = cudaMemcpyAsync(&bits, word, sizeof(bits), cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return cuda_fail(d, e, "error word");
    if (bits & ERR_TMA_WAIT) return fail(d, SLBM_ECUDA, "a TMA staging wait of the step ran past its bound");
    return SLBM_OK;
}

void fill_totals(const slbm_domain* d, const Rec& r, slbm_totals* t) {
    t->step = d->n;
    t->Q_phi = r.Q;
    t->H = r.H;
    t->phi_total = r.phi_tot;
    t->psi_total = r.psi_tot;
    t->lambda_phi = r.lam;
    t->mubar_psi = (d->p.psi_on && d->p.M_psi > 0) ? r.mpsi_mubar / d->p.M_psi : 0.0;
    t->kinetic = r.kin;
    t->S1 = r.S1;
    t->S2 = r.S2;
    t->clamp_count = (long long)r.clamps;
    t->range_count = (long long)r.range;
    t->free_energy = r.ef;
    t->residual = r.phi2 > 0.0 ? std::sqrt(r.dphi2 / r.phi2) : 0.0;
}

}  // namespace

std::atomic<unsigned long long> g_device_allocs{0};

cudaError_t slbm_device_malloc(void** ptr, size_t bytes) {
    const cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) g_device_allocs.fetch_add(1, std::memory_order_relaxed);
    return e;
}

// parameter checks and derivation shared with the three-dimensional domain
std::string slbm_validate_params(const slbm_params* p) { return validate(p); }
void slbm_derive_phys(slbm_domain* d) { derive(d); }
void slbm_wall_phys(slbm_domain* d, int w) { set_wall_phys(d, w); }

extern "C" {

void slbm_default_params(slbm_params* p, int nx, int ny) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nx = nx; p->ny = ny;
    p->tau_f = 0.8; p->tau_f_gas = -1.0; p->tau_g = 0.8; p->tau_h = 0.8;
    p->sigma = 0.01; p->eps = 4.0; p->Ex = 1.0; p->Pi = 0.18407;
    p->M_phi = 0.0; p->M_psi = 0.5; p->eta_phi = 1.0; p->eta_psi = 1.0;
    p->lambda_s = -1.0; p->psi_b = 0.0; p->phi_b = -1.0;
    p->rho_l = 1.0; p->rho_g = 1.0;
    p->constraint = SLBM_CONSTRAINT_NONLINEAR; p->multiplier = SLBM_MULT_PAPER;
    p->precision = SLBM_FP32; p->psi_on = 1;
    p->wall_saturation = 1;
}

}  // extern "C"

namespace {
// ws_bytes == 0 and ws == nullptr: the library allocates; otherwise the caller's workspace
slbm_status create_common(const slbm_params* p, void* stream, void* ws, size_t ws_bytes, bool ext, slbm_domain** out) {
    if (!out) return fail(nullptr, SLBM_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why = validate(p);
    if (!why.empty()) return fail(nullptr, SLBM_EINVAL, why);
    if (ext && !ws) return fail(nullptr, SLBM_EINVAL, "workspace is NULL");
    if (ext && ((uintptr_t)ws & 255)) return fail(nullptr, SLBM_EINVAL, "workspace must be 256-byte aligned");
    slbm_domain* d = new (std::nothrow) slbm_domain();
    if (!d) return fail(nullptr, SLBM_ENOMEM, "host allocation failed");
    d->p = *p;
    d->stream = (cudaStream_t)stream;
    d->N = (long long)p->nx * p->ny;
    d->ext = ext;
    d->ws = (unsigned char*)ws;
    d->ws_size = ws_bytes;
    derive(d);
    plan_domain(d);
    slbm_status s = alloc_state(d, ext);
    if (s != SLBM_OK) {
        g_create_error = d->err;
        slbm_destroy(d);
        return s;
    }
    d->tma = tma_eligible(d->p) && build_maps(d);
    cudaError_t e = cudaMemsetAsync(d->counter, 0, 2 * sizeof(unsigned int), d->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->recs, 0, 4 * sizeof(Rec), d->stream);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "cudaMemsetAsync");
        slbm_destroy(d);
        return SLBM_ECUDA;
    }
    *out = d;
    return SLBM_OK;
}
}  // namespace

extern "C" {

slbm_status slbm_create_domain(const slbm_params* p, void* stream, slbm_domain** out) {
    return create_common(p, stream, nullptr, 0, false, out);
}

size_t slbm_workspace_bytes(const slbm_params* p) {
    if (!validate(p).empty()) return 0;
    slbm_domain d;
    d.p = *p;
    d.N = (long long)p->nx * p->ny;
    d.ext = true;              // count only: ws stays NULL
    d.ws_size = ~(size_t)0;
    plan_domain(&d);
    if (alloc_state(&d, true) != SLBM_OK) return 0;
    return (d.ws_off + 255) & ~(size_t)255;
}

slbm_status slbm_create_domain_ext(const slbm_params* p, void* workspace, size_t bytes, void* stream,
                                   slbm_domain** out) {
    return create_common(p, stream, workspace, bytes, true, out);
}

slbm_status slbm_set_walls(slbm_domain* d, int wall, double theta0_deg, double beta_sg, double beta_sl, double u_x) {
    if (!d) return SLBM_EINVAL;
    if (wall < 0 || wall > 1) return fail(d, SLBM_EINVAL, "wall must be 0 (bottom) or 1 (top)");
    if (!(theta0_deg > 0 && theta0_deg < 180)) return fail(d, SLBM_EINVAL, "theta0 must lie in (0, 180) degrees");
    if (!(beta_sg >= 0) || !(beta_sl >= 0)) return fail(d, SLBM_EINVAL, "adsorption elasticities must be >= 0");
    if (!(std::fabs(u_x) < 0.3)) return fail(d, SLBM_EINVAL, "|u_x| must be below 0.3 (lattice units)");
    d->wall_theta[wall] = theta0_deg;
    d->wall_bsg[wall] = beta_sg;
    d->wall_bsl[wall] = beta_sl;
    d->wall_u[wall] = u_x;
    set_wall_phys(d, wall);
    return SLBM_OK;
}

namespace {
slbm_status init_fields_from(slbm_domain* d, const double* phi, const double* psi, cudaMemcpyKind kind) {
    if (!d || !phi) return d ? fail(d, SLBM_EINVAL, "phi is NULL") : SLBM_EINVAL;
    if (d->p.psi_on && !psi) return fail(d, SLBM_EINVAL, "psi is NULL while psi_on = 1");
    const size_t bytes = (size_t)d->N * sizeof(double);
    if (!d->fields) {
        slbm_status s = dalloc(d, &d->fields, 5 * bytes);
        if (s) return s;
    }
    cudaError_t e = cudaSuccess;
    if (phi != d->fields) e = cudaMemcpyAsync(d->fields, phi, bytes, kind, d->stream);
    if (e == cudaSuccess && d->p.psi_on && psi != d->fields + d->N)
        e = cudaMemcpyAsync(d->fields + d->N, psi, bytes, kind, d->stream);
    if (e != cudaSuccess) return cuda_fail(d, e, "cudaMemcpyAsync (init)");
    d->cur = 0;
    d->n = 0;
    switch (d->p.precision) {
        case SLBM_FP16DEV: e = launch_init<__half>(d, d->fields, d->fields + d->N); break;
        case SLBM_BF16DEV: e = launch_init<__nv_bfloat16>(d, d->fields, d->fields + d->N); break;
        default: e = launch_init<float>(d, d->fields, d->fields + d->N); break;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d->recs, 0, 4 * sizeof(Rec), d->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->counter, 0, 2 * sizeof(unsigned int), d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);   // host arrays may be freed on return
    if (e != cudaSuccess) return cuda_fail(d, e, "init");
    d->initialised = true;
    return SLBM_OK;
}
}  // namespace

slbm_status slbm_init_fields(slbm_domain* d, const double* phi, const double* psi) {
    return init_fields_from(d, phi, psi, cudaMemcpyHostToDevice);
}

slbm_status slbm_init_fields_device(slbm_domain* d, const double* phi, const double* psi) {
    return init_fields_from(d, phi, psi, cudaMemcpyDeviceToDevice);
}

slbm_status slbm_step(slbm_domain* d, long long nsteps) {
    if (!d) return SLBM_EINVAL;
    if (nsteps < 0) return fail(d, SLBM_EINVAL, "nsteps must be >= 0");
    if (!d->initialised) return fail(d, SLBM_ESTATE, "fields not initialised");
    const bool exact = d->p.multiplier == SLBM_MULT_EXACT;
    for (long long s = 0; s < nsteps; ++s) {
        cudaError_t e = launch(d, false);
        if (e == cudaSuccess && exact) e = launch_exact_multiplier(d);
        if (e != cudaSuccess) return cuda_fail(d, e, "step launch");
        d->cur ^= 1;
        d->n += 1;
    }
    return SLBM_OK;
}

slbm_status slbm_read_fields(slbm_domain* d, double* phi, double* psi, double* ux, double* uy, double* p) {
    if (!d) return SLBM_EINVAL;
    if (!d->initialised) return fail(d, SLBM_ESTATE, "fields not initialised");
    const size_t bytes = (size_t)d->N * sizeof(double);
    if (!d->fields) {
        slbm_status s = dalloc(d, &d->fields, 5 * bytes);
        if (s) return s;
    }
    cudaError_t e = launch(d, true);
    double* dst[5] = {phi, psi, ux, uy, p};
    for (int i = 0; i < 5 && e == cudaSuccess; ++i)
        if (dst[i]) e = cudaMemcpyAsync(dst[i], d->fields + i * d->N, bytes, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return cuda_fail(d, e, "read_fields");
    return SLBM_OK;
}

slbm_status slbm_read_totals(slbm_domain* d, slbm_totals* t) {
    if (!d || !t) return d ? fail(d, SLBM_EINVAL, "totals is NULL") : SLBM_EINVAL;
    if (!d->initialised) return fail(d, SLBM_ESTATE, "fields not initialised");
    const size_t bytes = (size_t)d->N * sizeof(double);
    if (!d->fields) {
        slbm_status s = dalloc(d, &d->fields, 5 * bytes);
        if (s) return s;
    }
    cudaError_t e = launch(d, true);
    Rec r;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, d->recs + 2, sizeof(Rec), cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return cuda_fail(d, e, "read_totals");
    if (slbm_status es = check_err_word(d, d->counter + 1)) return es;
    if (e == cudaSuccess && d->p.multiplier == SLBM_MULT_EXACT && d->n > 0) {
        Rec last;
        e = cudaMemcpyAsync(&last, d->recs + ((d->n - 1) & 1), sizeof(Rec), cudaMemcpyDeviceToHost, d->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) return cuda_fail(d, e, "read_totals");
        r.lam = last.lam;
        if (last.pad[1] < 0.0) {
            fill_totals(d, r, t);
            return fail(d, SLBM_EUNSTABLE, "exact multiplier: Newton's method found no root in the last step");
        }
    }
    fill_totals(d, r, t);
    const bool finite = std::isfinite(r.Q) && std::isfinite(r.psi_tot) && std::isfinite(r.lam) && std::isfinite(r.kin);
    if (t->range_count > 0 || !finite) return fail(d, SLBM_EUNSTABLE, "the run has diverged (non-finite or out-of-range values)");
    return SLBM_OK;
}

slbm_status slbm_read_fields_noalloc(slbm_domain* d, double* phi, double* psi, double* ux, double* uy,
                                     double* p, slbm_totals* t) {
    if (!d) return SLBM_EINVAL;
    if (!d->initialised) return fail(d, SLBM_ESTATE, "fields not initialised");
    if (d->grid.x * d->grid.y > SLBM_NOALLOC_MAX_CTAS)
        return fail(d, SLBM_EINVAL, "grid larger than the static scratch of slbm_read_fields_noalloc (" +
                                        std::to_string(SLBM_NOALLOC_MAX_CTAS) + " CTAs)");
    unsigned char* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return cuda_fail(d, e, "cudaGetSymbolAddress (noalloc scratch)");
    // the completion counter must start at zero
    e = cudaMemsetAsync(scratch + SLBM_NOALLOC_MAX_CTAS * NPART * 8, 0, 2 * sizeof(unsigned int), d->stream);
    double* o[5] = {phi, psi, ux, uy, p};
    if (e == cudaSuccess) {
        switch (d->p.precision) {
            case SLBM_FP16DEV: e = launch_diag_noalloc<__half>(d, scratch, o); break;
            case SLBM_BF16DEV: e = launch_diag_noalloc<__nv_bfloat16>(d, scratch, o); break;
            default: e = launch_diag_noalloc<float>(d, scratch, o); break;
        }
    }
    if (e != cudaSuccess) return cuda_fail(d, e, "read_fields_noalloc");
    if (!t) return SLBM_OK;
    Rec r;
    e = cudaMemcpyAsync(&r, scratch + SLBM_NOALLOC_MAX_CTAS * NPART * 8 + 256, sizeof(Rec), cudaMemcpyDeviceToHost,
                        d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return cuda_fail(d, e, "read_fields_noalloc");
    if (slbm_status es = check_err_word(d, (const unsigned int*)(scratch + SLBM_NOALLOC_MAX_CTAS * NPART * 8) + 1)) return es;
    if (slbm_status es = check_err_word(d, d->counter + 1)) return es;
    if (e == cudaSuccess && d->p.multiplier == SLBM_MULT_EXACT && d->n > 0) {
        Rec last;
        e = cudaMemcpyAsync(&last, d->recs + ((d->n - 1) & 1), sizeof(Rec), cudaMemcpyDeviceToHost, d->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) return cuda_fail(d, e, "read_totals");
        r.lam = last.lam;
        if (last.pad[1] < 0.0) {
            fill_totals(d, r, t);
            return fail(d, SLBM_EUNSTABLE, "exact multiplier: Newton's method found no root in the last step");
        }
    }
    fill_totals(d, r, t);
    const bool finite = std::isfinite(r.Q) && std::isfinite(r.psi_tot) && std::isfinite(r.lam) && std::isfinite(r.kin);
    if (t->range_count > 0 || !finite) return fail(d, SLBM_EUNSTABLE, "the run has diverged (non-finite or out-of-range values)");
    return SLBM_OK;
}

// ---- checkpoints: a fixed header, then the current state buffers in a fixed order
}  // extern "C"

namespace {
struct CkptHeader {
    char magic[8];            // "SLBMCKP1"
    uint32_t version, header_bytes;
    slbm_params p;
    double walls[2][4];       // theta0, beta_sg, beta_sl, u_x per wall
    long long n;
    unsigned long long N, payload_bytes;
    uint32_t elem, rec_bytes;
};

// the device buffers of the current time level, in file order
int state_planes(slbm_domain* d, void** ptr, size_t* bytes) {
    const size_t es = elem_size(d->p.precision), N = (size_t)d->N;
    const int c = d->cur;
    void* pp[] = {d->f[c], d->gd[c], d->hd[c], d->gm[c], d->hm[c], d->php[c], d->hist, d->recs};
    const size_t bb[] = {9 * N * es, 8 * N * es, 8 * N * es, N * sizeof(float2), N * sizeof(float2), N * sizeof(float),
                         6 * N * es, 4 * sizeof(Rec)};
    for (int i = 0; i < 8; ++i) { ptr[i] = pp[i]; bytes[i] = bb[i]; }
    return 8;
}

bool same_params(const slbm_params& a, const slbm_params& b) {
    const double da[] = {a.tau_f, a.tau_f_gas, a.tau_g, a.tau_h, a.sigma, a.eps, a.Ex, a.Pi, a.M_phi, a.M_psi,
                         a.eta_phi, a.eta_psi, a.lambda_s, a.psi_b, a.phi_b, a.rho_l, a.rho_g, a.Gx, a.Gy};
    const double db[] = {b.tau_f, b.tau_f_gas, b.tau_g, b.tau_h, b.sigma, b.eps, b.Ex, b.Pi, b.M_phi, b.M_psi,
                         b.eta_phi, b.eta_psi, b.lambda_s, b.psi_b, b.phi_b, b.rho_l, b.rho_g, b.Gx, b.Gy};
    for (size_t i = 0; i < sizeof(da) / sizeof(da[0]); ++i)
        if (std::memcmp(&da[i], &db[i], sizeof(double))) return false;
    for (int i = 0; i < 4; ++i)
        if (a.mrt_f[i] != b.mrt_f[i] || a.mrt_g[i] != b.mrt_g[i] || a.mrt_h[i] != b.mrt_h[i]) return false;
    return a.nx == b.nx && a.ny == b.ny && a.constraint == b.constraint && a.multiplier == b.multiplier &&
           a.precision == b.precision && a.psi_on == b.psi_on && a.wall_saturation == b.wall_saturation;
}
}  // namespace

extern "C" {

slbm_status slbm_save(slbm_domain* d, const char* path) {
    if (!d) return SLBM_EINVAL;
    if (!path) return fail(d, SLBM_EINVAL, "path is NULL");
    if (!d->initialised) return fail(d, SLBM_ESTATE, "fields not initialised");
    void* ptr[8];
    size_t bytes[8];
    const int np = state_planes(d, ptr, bytes);
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "SLBMCKP1", 8);
    h.version = 1;
    h.header_bytes = sizeof(CkptHeader);
    h.p = d->p;
    for (int w = 0; w < 2; ++w) {
        h.walls[w][0] = d->wall_theta[w]; h.walls[w][1] = d->wall_bsg[w];
        h.walls[w][2] = d->wall_bsl[w]; h.walls[w][3] = d->wall_u[w];
    }
    h.n = d->n;
    h.N = (unsigned long long)d->N;
    h.elem = (uint32_t)elem_size(d->p.precision);
    h.rec_bytes = sizeof(Rec);
    for (int i = 0; i < np; ++i) h.payload_bytes += bytes[i];
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(d, SLBM_EINVAL, std::string("cannot open ") + path + " for writing");
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1;
    std::string buf;
    for (int i = 0; i < np && ok; ++i) {
        buf.resize(bytes[i]);
        cudaError_t e = cudaMemcpyAsync(&buf[0], ptr[i], bytes[i], cudaMemcpyDeviceToHost, d->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) {
            std::fclose(fp);
            return cuda_fail(d, e, "save");
        }
        ok = std::fwrite(buf.data(), 1, bytes[i], fp) == bytes[i];
    }
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(d, SLBM_EINVAL, std::string("write to ") + path + " failed");
    return SLBM_OK;
}

slbm_status slbm_load(slbm_domain* d, const char* path) {
    if (!d) return SLBM_EINVAL;
    if (!path) return fail(d, SLBM_EINVAL, "path is NULL");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(d, SLBM_EINVAL, std::string("cannot open ") + path);
    CkptHeader h;
    if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, "SLBMCKP1", 8) != 0 || h.version != 1 ||
        h.header_bytes != sizeof(CkptHeader)) {
        std::fclose(fp);
        return fail(d, SLBM_EINVAL, std::string(path) + " is not a checkpoint of this library version");
    }
    if (!same_params(h.p, d->p) || h.N != (unsigned long long)d->N || h.elem != elem_size(d->p.precision) ||
        h.rec_bytes != sizeof(Rec)) {
        std::fclose(fp);
        return fail(d, SLBM_EINVAL, "checkpoint parameters differ from the domain's");
    }
    d->cur = 0;
    void* ptr[8];
    size_t bytes[8];
    const int np = state_planes(d, ptr, bytes);
    size_t total = 0;
    for (int i = 0; i < np; ++i) total += bytes[i];
    if (total != h.payload_bytes) {
        std::fclose(fp);
        return fail(d, SLBM_EINVAL, "checkpoint payload size mismatch");
    }
    std::string buf;
    for (int i = 0; i < np; ++i) {
        buf.resize(bytes[i]);
        if (std::fread(&buf[0], 1, bytes[i], fp) != bytes[i]) {
            std::fclose(fp);
            return fail(d, SLBM_EINVAL, std::string(path) + " is truncated");
        }
        cudaError_t e = cudaMemcpyAsync(ptr[i], buf.data(), bytes[i], cudaMemcpyHostToDevice, d->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);   // buf is reused
        if (e != cudaSuccess) {
            std::fclose(fp);
            return cuda_fail(d, e, "load");
        }
    }
    std::fclose(fp);
    for (int w = 0; w < 2; ++w) {
        d->wall_theta[w] = h.walls[w][0]; d->wall_bsg[w] = h.walls[w][1];
        d->wall_bsl[w] = h.walls[w][2]; d->wall_u[w] = h.walls[w][3];
        set_wall_phys(d, w);
    }
    d->n = h.n;
    cudaError_t e = cudaMemsetAsync(d->counter, 0, 2 * sizeof(unsigned int), d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return cuda_fail(d, e, "load");
    d->initialised = true;
    return SLBM_OK;
}

slbm_status slbm_set_mms(slbm_domain* d, const slbm_mms* m) {
    if (!d) return SLBM_EINVAL;
    if (!m) {
        d->mms = false;
        d->mms_u0x = 0.0;
        return SLBM_OK;
    }
    if (d->p.precision != SLBM_FP32) return fail(d, SLBM_EINVAL, "the manufactured-solution test runs in FP32 storage");
    if (d->phys.var_nu || d->p.rho_l != d->p.rho_g) return fail(d, SLBM_EINVAL, "the test needs uniform density and viscosity");
    if (!(m->dx > 0) || !(m->dt > 0)) return fail(d, SLBM_EINVAL, "dx and dt must be positive");
    d->mms = true;
    d->mms_u0x = m->u * m->dt / m->dx;
    Phys& P = d->phys;
    P.mms_a = (float)m->amplitude; P.mms_u = (float)m->u; P.mms_M = (float)m->M; P.mms_beta = (float)m->beta;
    P.mms_kappa = (float)m->kappa; P.mms_kT = (float)m->kT; P.mms_W = (float)m->W;
    P.mms_dx = (float)m->dx; P.mms_dt = (float)m->dt;
    return SLBM_OK;
}

size_t slbm_device_bytes(const slbm_domain* d) { return d ? d->bytes : 0; }

unsigned long long slbm_device_allocations(void) { return g_device_allocs.load(std::memory_order_relaxed); }

}  // extern "C"

// Library-internal: the diagnostic pass of the current level written into the domain's own
// field buffer, reduced with its own partials (no shared scratch); queued on its stream.
slbm_status diag_into_fields(slbm_domain* d) {
    if (!d->initialised || !d->fields) return fail(d, SLBM_ESTATE, "fields not initialised");
    cudaError_t e = launch(d, true);
    return e == cudaSuccess ? SLBM_OK : cuda_fail(d, e, "diagnostic pass");
}

extern "C" {

void slbm_destroy(slbm_domain* d) {
    if (!d) return;
    if (d->ext) {   // the workspace belongs to the caller
        delete d;
        return;
    }
    for (int b = 0; b < 2; ++b) {
        cudaFree(d->f[b]); cudaFree(d->gd[b]); cudaFree(d->hd[b]);
        cudaFree(d->gm[b]); cudaFree(d->hm[b]); cudaFree(d->php[b]);
    }
    cudaFree(d->hist); cudaFree(d->partials); cudaFree(d->counter); cudaFree(d->recs); cudaFree(d->fields);
    delete d;
}

const char* slbm_last_error(const slbm_domain* d) { return d ? d->err.c_str() : g_create_error.c_str(); }

const char* slbm_version(void) { return "surflbm 0.1 (sm_103a)"; }

}  // extern "C"
