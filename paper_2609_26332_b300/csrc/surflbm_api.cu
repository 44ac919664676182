// C-ABI implementation of include/surflbm.h: parameter derivation, device state,
// initialisation kernel and launches of the fused step kernel.
#include "surflbm.h"
#include "surflbm_step.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

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
            gk[k] = WkD(k) * eta * ft;
            msum += gk[k];
        }
        float2 mv;
        mv.x = (float)msum;
        mv.y = (float)(msum - (double)mv.x);
        m[c] = mv;
        for (int k = 1; k < 9; ++k) Stor<T>::st(d, (long long)(k - 1) * a.N + c, (float)(gk[k] - (double)Wk(k) * mv.x));
    }
    const double rho = a.rho_g + (a.rho_l - a.rho_g) * 0.5 * (a.phi0[c] * a.inv_phi_b + 1.0);
    for (int k = 0; k < 9; ++k) {
        double v = 0.0;
        const int ty = y + CYk(k);
        if (ty < 0 || ty >= a.ny) v = 6.0 * WkD(k) * rho * CXk(k) * a.uw[ty < 0 ? 0 : 1];
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
    a.nx = d->p.nx; a.ny = d->p.ny; a.N = d->N; a.total = d->total;
    a.f_in = (const T*)d->f[i]; a.gd_in = (const T*)d->gd[i]; a.gm_in = d->gm[i];
    a.hd_in = (const T*)d->hd[i]; a.hm_in = d->hm[i]; a.php_in = d->php[i];
    a.f_out = (T*)d->f[o]; a.gd_out = (T*)d->gd[o]; a.gm_out = d->gm[o];
    a.hd_out = (T*)d->hd[o]; a.hm_out = d->hm[o]; a.php_out = d->php[o];
    a.hist = (T*)d->hist;
    a.partials = d->partials;
    a.counter = d->counter;
    a.rec_prev = d->n == 0 ? d->recs + 3 : d->recs + ((d->n - 1) & 1);
    a.rec_out = diag ? d->recs + 2 : d->recs + (d->n & 1);
    a.first = d->n == 0;
    if (diag && d->fields) {
        a.o_phi = d->fields; a.o_psi = d->fields + d->N; a.o_ux = d->fields + 2 * d->N;
        a.o_uy = d->fields + 3 * d->N; a.o_p = d->fields + 4 * d->N;
    }
    a.P = d->phys;
    return a;
}

template <class T>
cudaError_t prepare_kernels() {
    static cudaError_t done = cudaErrorNotReady;
    if (done == cudaErrorNotReady) {
        const int sm = (int)smem_bytes<T>();
        done = cudaFuncSetAttribute(step_kernel<T, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (done == cudaSuccess)
            done = cudaFuncSetAttribute(step_kernel<T, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (done == cudaSuccess)
            done = cudaFuncSetAttribute(step_kernel<T, false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (done == cudaSuccess)
            done = cudaFuncSetAttribute(step_kernel<T, true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    }
    return done;
}

template <class T>
cudaError_t launch_step(slbm_domain* d, bool diag) {
    cudaError_t e = prepare_kernels<T>();
    if (e != cudaSuccess) return e;
    StepArgs<T> a = make_args<T>(d, diag);
    // uniform density and viscosity (the common case) drop every density-gradient term
    const bool var = a.P.var_nu || a.P.rho_l != a.P.rho_g;
    const size_t sm = smem_bytes<T>();
    if (diag) {
        if (var) step_kernel<T, true, true, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, BatchArgs{});
        else step_kernel<T, true, false, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, BatchArgs{});
    } else {
        if (var) step_kernel<T, false, true, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, BatchArgs{});
        else step_kernel<T, false, false, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, BatchArgs{});
    }
    return cudaGetLastError();
}

template <class T>
int resident_ctas_per_sm() {
    int n = 0;
    if (prepare_kernels<T>() != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<T, false, false, false>, NTHREADS, smem_bytes<T>()) != cudaSuccess)
        return 1;
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
    a.psi_on = d->p.psi_on != 0;
    const int c = d->cur;
    const unsigned blocks = (unsigned)((d->N + 255) / 256);
    init_kernel<T><<<blocks, 256, 0, d->stream>>>(a, (T*)d->f[c], (T*)d->gd[c], d->gm[c], (T*)d->hd[c], d->hm[c],
                                                  d->php[c]);
    return cudaGetLastError();
}

template <class P>
slbm_status dalloc(slbm_domain* d, P** ptr, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(d, SLBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    d->bytes += bytes;
    return SLBM_OK;
}

// ---- scratch of slbm_read_fields_noalloc: static device memory, no allocation
static_assert(sizeof(Rec) <= 128, "record must fit the scratch tail");
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
    cudaError_t e = prepare_kernels<T>();
    if (e != cudaSuccess) return e;
    StepArgs<T> a = make_args<T>(d, true);
    a.partials = (double*)scratch;
    a.counter = (unsigned int*)(scratch + SLBM_NOALLOC_MAX_CTAS * 9 * 8);
    a.rec_out = (Rec*)(scratch + SLBM_NOALLOC_MAX_CTAS * 9 * 8 + 256);
    a.o_phi = o[0]; a.o_psi = o[1]; a.o_ux = o[2]; a.o_uy = o[3]; a.o_p = o[4];
    const bool var = a.P.var_nu || a.P.rho_l != a.P.rho_g;
    const size_t sm = smem_bytes<T>();
    if (var) step_kernel<T, true, true, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, BatchArgs{});
    else step_kernel<T, true, false, false><<<d->grid, NTHREADS, sm, d->stream>>>(a, BatchArgs{});
    return cudaGetLastError();
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
}

}  // namespace

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

slbm_status slbm_create_domain(const slbm_params* p, void* stream, slbm_domain** out) {
    if (!out) return fail(nullptr, SLBM_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why = validate(p);
    if (!why.empty()) return fail(nullptr, SLBM_EINVAL, why);
    slbm_domain* d = new (std::nothrow) slbm_domain();
    if (!d) return fail(nullptr, SLBM_ENOMEM, "host allocation failed");
    d->p = *p;
    d->stream = (cudaStream_t)stream;
    d->N = (long long)p->nx * p->ny;
    derive(d);
    {
        int per_sm = 1;
        switch (p->precision) {
            case SLBM_FP16DEV: per_sm = resident_ctas_per_sm<__half>(); break;
            case SLBM_BF16DEV: per_sm = resident_ctas_per_sm<__nv_bfloat16>(); break;
            default: per_sm = resident_ctas_per_sm<float>(); break;
        }
        d->total = (long long)((p->nx + TX - 1) / TX) * p->ny;
        d->grid = dim3((unsigned)choose_ctas(d, per_sm));
    }
    const size_t es = elem_size(p->precision);
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
    if (p->multiplier == SLBM_MULT_EXACT) {
        d->exact_blocks = exact_multiplier_blocks(p->precision, d->N);
        if ((size_t)d->exact_blocks > nblocks) nblocks = (size_t)d->exact_blocks;
    }
    if (s == SLBM_OK) s = dalloc(d, &d->hist, 6 * N * es);
    if (s == SLBM_OK) s = dalloc(d, &d->partials, nblocks * NPART * sizeof(double));
    if (s == SLBM_OK) s = dalloc(d, &d->counter, sizeof(unsigned int));
    if (s == SLBM_OK) s = dalloc(d, &d->recs, 4 * sizeof(Rec));
    if (s != SLBM_OK) {
        g_create_error = d->err;
        slbm_destroy(d);
        return s;
    }
    cudaError_t e = cudaMemsetAsync(d->counter, 0, sizeof(unsigned int), d->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->recs, 0, 4 * sizeof(Rec), d->stream);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "cudaMemsetAsync");
        slbm_destroy(d);
        return SLBM_ECUDA;
    }
    *out = d;
    return SLBM_OK;
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
    if (e == cudaSuccess) e = cudaMemsetAsync(d->counter, 0, sizeof(unsigned int), d->stream);
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
    e = cudaMemsetAsync(scratch + SLBM_NOALLOC_MAX_CTAS * 9 * 8, 0, sizeof(unsigned int), d->stream);
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
    e = cudaMemcpyAsync(&r, scratch + SLBM_NOALLOC_MAX_CTAS * 9 * 8 + 256, sizeof(Rec), cudaMemcpyDeviceToHost,
                        d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return cuda_fail(d, e, "read_fields_noalloc");
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

size_t slbm_device_bytes(const slbm_domain* d) { return d ? d->bytes : 0; }

void slbm_destroy(slbm_domain* d) {
    if (!d) return;
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
