// Batches: many independent domains (instances of uneven sizes and parameters) stepped
// together, one launch of the persistent tile-queue kernel per time step, K steps
// replayed from a captured CUDA graph, converged instances retired between graph
// replays, and the tiling (strip width x band height, i.e. the cells each thread marches
// per piece, x resident CTAs per SM) chosen by a timing autotuner whose choices are cached
// in a JSON file.
#include "surflbm_internal.cuh"

// the step kernel with 32-column strips (128 threads per CTA) and with 128-column strips
// (512 threads, one CTA per SM), the batch's other tile shapes
namespace slbm {
namespace w32 {
#define SLBM_TILE_TX 32
#include "surflbm_step_tile.inc"
#undef SLBM_TILE_TX
}  // namespace w32
namespace w128 {
#define SLBM_TILE_TX 128
#include "surflbm_step_tile.inc"
#undef SLBM_TILE_TX
}  // namespace w128
}  // namespace slbm

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

using namespace slbm;

namespace {

std::string g_batch_create_error = "no error";

// residual of one instance over K steps: sums of (x - x_snap)^2 and x^2 for
// phi (previous-step phi) and psi (post-collision zeroth moment), then the snapshot update
struct ResidualArgs {
    const float* php;      // current phi of the instance
    const float2* hm;      // current psi moment
    float* snap;           // 2 N floats: phi, psi snapshots
    double* out;           // 4 doubles: sum dphi^2, sum phi^2, sum dpsi^2, sum psi^2
    long long N;
};

__global__ void residual_kernel(const ResidualArgs* args, const int* blk_inst, const long long* blk_start) {
    const int b = blockIdx.x;
    const ResidualArgs a = args[blk_inst[b]];
    const long long i0 = blk_start[b];
    double s[4] = {0, 0, 0, 0};
    for (long long i = i0 + threadIdx.x; i < min(a.N, i0 + 4096); i += blockDim.x) {
        const float ph = a.php[i], ps = a.hm[i].x;
        const float dph = ph - a.snap[i], dps = ps - a.snap[a.N + i];
        s[0] += (double)dph * dph;
        s[1] += (double)ph * ph;
        s[2] += (double)dps * dps;
        s[3] += (double)ps * ps;
        a.snap[i] = ph;
        a.snap[a.N + i] = ps;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double v = s[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(a.out + q, v);   // convergence check only
    }
}

template <class T>
cudaError_t prepare_batch_kernels() {
    static PerDeviceOnce once;
    return once([] {
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        const int sm = (int)smem_bytes<T>(), sm32 = (int)w32::smem_bytes<T>(), sm128 = (int)w128::smem_bytes<T>();
        cudaError_t e = cudaFuncSetAttribute(step_kernel<T, false, false, true>, attr, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, false, true, true>, attr, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(w32::step_kernel<T, false, false, true>, attr, sm32);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(w32::step_kernel<T, false, true, true>, attr, sm32);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(w128::step_kernel<T, false, false, true>, attr, sm128);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(w128::step_kernel<T, false, true, true>, attr, sm128);
        return e;
    });
}

// resident CTAs per SM the strip width allows at most (shared memory and registers)
int max_ctas_per_sm(int width) { return width == 32 ? 3 : (width == 128 ? 1 : 2); }

}  // namespace


namespace {

slbm_status bfail(slbm_batch* b, slbm_status s, const std::string& msg) {
    if (b) b->err = msg; else g_batch_create_error = msg;
    return s;
}
slbm_status bcuda(slbm_batch* b, cudaError_t e, const char* what) {
    return bfail(b, SLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int pieces_of(const slbm_domain* d, int width, int band_rows, int* bands_out) {
    const int strips = (d->p.nx + width - 1) / width;
    int bands = (d->p.ny + band_rows - 1) / band_rows;
    if (bands < 1) bands = 1;
    if (bands_out) *bands_out = bands;
    return strips * bands;
}

void drop_graph(slbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_len = 0;
}

// Rebuild the instance descriptors and the tile queue for the active instances.
slbm_status build_tables(slbm_batch* b) {
    drop_graph(b);
    std::vector<InstDesc> inst(b->count);
    std::vector<Piece> pieces;
    for (int i = 0; i < b->count; ++i) {
        slbm_domain* d = b->dom[i];
        InstDesc& I = inst[i];
        std::memset(&I, 0, sizeof(I));
        for (int k = 0; k < 2; ++k) {
            I.f[k] = d->f[k]; I.gd[k] = d->gd[k]; I.hd[k] = d->hd[k];
            I.gm[k] = d->gm[k]; I.hm[k] = d->hm[k]; I.php[k] = d->php[k];
        }
        I.hist = d->hist;
        I.recs = d->recs;
        I.partials = b->d_partials + b->part_off[i];
        I.counter = b->d_counters + i;
        I.nx = d->p.nx;
        I.ny = d->p.ny;
        I.N = d->N;
        I.G0 = b->G0[i];
        I.P = d->phys;
        if (!b->active[i]) continue;
        int bands = 1;
        const int np = pieces_of(d, b->strip_width, b->band_rows, &bands);
        I.npieces = np;
        const int strips = (d->p.nx + b->strip_width - 1) / b->strip_width;
        int slot = 0;
        // band-major order inside an instance: neighbouring strips of one band are queued together
        for (int bd = 0; bd < bands; ++bd) {
            const int y0 = (int)((long long)d->p.ny * bd / bands), y1 = (int)((long long)d->p.ny * (bd + 1) / bands);
            for (int s = 0; s < strips; ++s) {
                Piece pc;
                std::memset(&pc, 0, sizeof(pc));
                pc.inst = i; pc.strip = s; pc.y0 = y0; pc.y1 = y1; pc.slot = slot++;
                pieces.push_back(pc);
            }
        }
    }
    // biggest pieces first keeps the queue tail short
    std::stable_sort(pieces.begin(), pieces.end(), [&](const Piece& a, const Piece& c) {
        return (a.y1 - a.y0) > (c.y1 - c.y0);
    });
    cudaFree(b->d_pieces);
    b->d_pieces = nullptr;
    b->npieces = (int)pieces.size();
    cudaError_t e = cudaSuccess;
    if (b->npieces > 0) {
        e = slbm_device_malloc((void**)&b->d_pieces, pieces.size() * sizeof(Piece));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_pieces, pieces.data(), pieces.size() * sizeof(Piece), cudaMemcpyHostToDevice, b->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_inst, inst.data(), inst.size() * sizeof(InstDesc), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch tables");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->nctas = std::max(1, std::min(sms * b->ctas_per_sm, b->npieces));
    b->tables_valid = true;
    return SLBM_OK;
}

template <class T>
cudaError_t launch_batch(slbm_batch* b) {
    cudaError_t e = prepare_batch_kernels<T>();
    if (e != cudaSuccess) return e;
    StepArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    BatchArgs ba;
    ba.inst = b->d_inst;
    ba.pieces = b->d_pieces;
    ba.npieces = b->npieces;
    ba.queue = b->d_queue;
    ba.done = b->d_queue + 1;
    ba.G = b->d_G;
    static const TmaMaps none{};
    if (b->strip_width == 32) {
        const size_t sm = w32::smem_bytes<T>();
        if (b->var) w32::step_kernel<T, false, true, true><<<b->nctas, w32::NTHREADS, sm, b->stream>>>(a, ba, none);
        else w32::step_kernel<T, false, false, true><<<b->nctas, w32::NTHREADS, sm, b->stream>>>(a, ba, none);
    } else if (b->strip_width == 128) {
        const size_t sm = w128::smem_bytes<T>();
        if (b->var) w128::step_kernel<T, false, true, true><<<b->nctas, w128::NTHREADS, sm, b->stream>>>(a, ba, none);
        else w128::step_kernel<T, false, false, true><<<b->nctas, w128::NTHREADS, sm, b->stream>>>(a, ba, none);
    } else {
        const size_t sm = smem_bytes<T>();
        if (b->var) step_kernel<T, false, true, true><<<b->nctas, NTHREADS, sm, b->stream>>>(a, ba, none);
        else step_kernel<T, false, false, true><<<b->nctas, NTHREADS, sm, b->stream>>>(a, ba, none);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_any(slbm_batch* b) {
    switch (b->precision) {
        case SLBM_FP16DEV: return launch_batch<__half>(b);
        case SLBM_BF16DEV: return launch_batch<__nv_bfloat16>(b);
        default: return launch_batch<float>(b);
    }
}

// host bookkeeping after n steps of every active instance
void advance(slbm_batch* b, long long n) {
    b->G += n;
    for (int i = 0; i < b->count; ++i)
        if (b->active[i]) {
            b->dom[i]->n += n;
            b->dom[i]->cur ^= (int)(n & 1);
        }
}

slbm_status run_steps(slbm_batch* b, long long nsteps) {
    if (!b->tables_valid) {
        slbm_status s = build_tables(b);
        if (s) return s;
    }
    if (b->npieces == 0 || nsteps <= 0) return SLBM_OK;
    cudaError_t e = b->precision == SLBM_FP16DEV ? prepare_batch_kernels<__half>()
                  : b->precision == SLBM_BF16DEV ? prepare_batch_kernels<__nv_bfloat16>()
                                                 : prepare_batch_kernels<float>();
    if (e != cudaSuccess) return bcuda(b, e, "batch kernel attributes");
    long long left = nsteps;
    // whole graphs of graph_steps launches, then single launches for the remainder
    if (left >= b->graph_steps) {
        if (!b->graph || b->graph_len != b->graph_steps) {
            drop_graph(b);
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            for (int k = 0; k < b->graph_steps && e == cudaSuccess; ++k) e = launch_batch_any(b);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) return bcuda(b, e, "batch graph capture");
            b->graph_len = b->graph_steps;
        }
        while (left >= b->graph_steps) {
            e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "batch graph launch");
            left -= b->graph_steps;
        }
    }
    for (; left > 0; --left) {
        e = launch_batch_any(b);
        if (e != cudaSuccess) return bcuda(b, e, "batch launch");
    }
    advance(b, nsteps);
    return SLBM_OK;
}

// residual of every active instance (max over phi, psi of
// ||x^n - x^{n-K}|| / (K ||x^n||)); r[i] = +inf for the first call
slbm_status residuals(slbm_batch* b, long long K, std::vector<double>& r) {
    r.assign(b->count, INFINITY);
    std::vector<ResidualArgs> args;
    std::vector<int> blk_inst;
    std::vector<long long> blk_start;
    std::vector<int> which;
    for (int i = 0; i < b->count; ++i) {
        if (!b->active[i]) continue;
        slbm_domain* d = b->dom[i];
        ResidualArgs a;
        a.php = d->php[d->cur];
        a.hm = d->hm[d->cur];
        a.snap = b->d_snap_base + b->snap_off[i];
        a.N = d->N;
        a.out = nullptr;
        const int idx = (int)args.size();
        args.push_back(a);
        which.push_back(i);
        for (long long s = 0; s < d->N; s += 4096) {
            blk_inst.push_back(idx);
            blk_start.push_back(s);
        }
    }
    if (args.empty()) return SLBM_OK;
    // scratch kept by the batch: sized on the first call (every instance active, the most
    // it can need: instances only retire), reused by every later check
    const size_t nb = blk_inst.size();
    const size_t bytes = args.size() * sizeof(ResidualArgs) + nb * (sizeof(int) + sizeof(long long)) +
                         args.size() * 4 * sizeof(double) + 64;
    cudaError_t e = cudaSuccess;
    if (bytes > b->res_bytes) {
        cudaFree(b->d_res);
        b->d_res = nullptr;
        b->res_bytes = 0;
        e = slbm_device_malloc((void**)&b->d_res, bytes);
        if (e != cudaSuccess) return bcuda(b, e, "residual scratch");
        b->res_bytes = bytes;
        b->bytes += bytes;
    }
    char* buf = b->d_res;
    double* d_out = (double*)buf;
    ResidualArgs* d_args = (ResidualArgs*)(buf + args.size() * 4 * sizeof(double));
    long long* d_bs = (long long*)((char*)d_args + args.size() * sizeof(ResidualArgs));
    int* d_bi = (int*)((char*)d_bs + nb * sizeof(long long));
    for (size_t k = 0; k < args.size(); ++k) args[k].out = d_out + 4 * k;
    e = cudaMemsetAsync(d_out, 0, args.size() * 4 * sizeof(double), b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_args, args.data(), args.size() * sizeof(ResidualArgs), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_bs, blk_start.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_bi, blk_inst.data(), nb * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
        residual_kernel<<<(unsigned)nb, 256, 0, b->stream>>>(d_args, d_bi, d_bs);
        e = cudaGetLastError();
    }
    std::vector<double> h(args.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "residual");
    if (b->have_snap) {
        for (size_t k = 0; k < args.size(); ++k) {
            const double rp = std::sqrt(h[4 * k]) / ((double)K * std::sqrt(std::max(h[4 * k + 1], 1e-300)));
            const double rs = std::sqrt(h[4 * k + 2]) / ((double)K * std::sqrt(std::max(h[4 * k + 3], 1e-300)));
            const bool psi_on = b->dom[which[k]]->p.psi_on;
            const bool finite = std::isfinite(h[4 * k]) && std::isfinite(h[4 * k + 1]) &&
                                (!psi_on || (std::isfinite(h[4 * k + 2]) && std::isfinite(h[4 * k + 3])));
            r[which[k]] = !finite ? NAN : psi_on ? std::max(rp, rs) : rp;
        }
    }
    b->have_snap = true;
    return SLBM_OK;
}

std::string signature(const slbm_batch* b) {
    long long cells = 0;
    std::vector<int> sizes;
    for (int i = 0; i < b->count; ++i) {
        cells += b->dom[i]->N;
        sizes.push_back(b->dom[i]->p.nx * 10000 + b->dom[i]->p.ny);
    }
    std::sort(sizes.begin(), sizes.end());
    unsigned long long h = 1469598103934665603ull;   // FNV-1a of the sorted size list
    for (int s : sizes) {
        h ^= (unsigned long long)s;
        h *= 1099511628211ull;
    }
    std::ostringstream o;
    o << "p" << b->precision << "_n" << b->count << "_c" << cells << "_h" << std::hex << h;
    return o.str();
}

}  // namespace

extern "C" {

slbm_status slbm_create_batch(const slbm_params* params, const slbm_wall_spec* walls, int count, void* stream,
                              slbm_batch** out) {
    if (!out) return bfail(nullptr, SLBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || count < 1) return bfail(nullptr, SLBM_EINVAL, "need params for at least one instance");
    for (int i = 1; i < count; ++i)
        if (params[i].precision != params[0].precision)
            return bfail(nullptr, SLBM_EINVAL, "all instances of a batch share one precision");
    for (int i = 0; i < count; ++i)
        if (params[i].multiplier == SLBM_MULT_EXACT)
            return bfail(nullptr, SLBM_EINVAL, "the exact multiplier is available for single domains only");
    slbm_batch* b = new (std::nothrow) slbm_batch();
    if (!b) return bfail(nullptr, SLBM_ENOMEM, "host allocation failed");
    b->count = count;
    b->precision = params[0].precision;
    b->stream = (cudaStream_t)stream;
    if (!b->stream) {
        cudaError_t es = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (es != cudaSuccess) {
            delete b;
            return bfail(nullptr, SLBM_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(es));
        }
        b->own_stream = true;
    }
    stream = b->stream;
    b->dom.assign(count, nullptr);
    b->active.assign(count, 0);
    b->G0.assign(count, 0);
    b->part_off.assign(count, 0);
    b->snap_off.assign(count, 0);
    b->max_pieces.assign(count, 0);
    size_t part_total = 0, snap_total = 0;
    for (int i = 0; i < count; ++i) {
        slbm_status s = slbm_create_domain(&params[i], stream, &b->dom[i]);
        if (s) {
            g_batch_create_error = std::string("instance ") + std::to_string(i) + ": " + slbm_last_error(nullptr);
            slbm_batch_destroy(b);
            return s;
        }
        slbm_domain* d = b->dom[i];
        if (walls) {
            for (int w = 0; w < 2; ++w) {
                const slbm_wall_spec& ws = walls[2 * i + w];
                s = slbm_set_walls(d, w, ws.theta0_deg, ws.beta_sg, ws.beta_sl, ws.u_x);
                if (s) {
                    g_batch_create_error = std::string("instance ") + std::to_string(i) + ": " + d->err;
                    slbm_batch_destroy(b);
                    return s;
                }
            }
        }
        b->var = b->var || d->phys.var_nu || d->phys.rho_l != d->phys.rho_g;
        b->bytes += d->bytes;
        b->max_pieces[i] = pieces_of(d, 32, 8, nullptr);   // the narrowest strips and smallest band the tiling allows
        b->part_off[i] = part_total;
        part_total += (size_t)b->max_pieces[i] * NPART;
        b->snap_off[i] = snap_total;
        snap_total += 2 * (size_t)d->N;
    }
    cudaError_t e = slbm_device_malloc((void**)&b->d_inst, count * sizeof(InstDesc));
    if (e == cudaSuccess) e = slbm_device_malloc((void**)&b->d_partials, part_total * sizeof(double));
    if (e == cudaSuccess) e = slbm_device_malloc((void**)&b->d_counters, count * sizeof(unsigned int));
    if (e == cudaSuccess) e = slbm_device_malloc((void**)&b->d_queue, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = slbm_device_malloc((void**)&b->d_G, sizeof(long long));
    if (e == cudaSuccess) e = slbm_device_malloc((void**)&b->d_snap_base, snap_total * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, count * sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_G, 0, sizeof(long long), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_batch_create_error = std::string("batch allocation: ") + cudaGetErrorString(e);
        slbm_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? SLBM_ENOMEM : SLBM_ECUDA;
    }
    b->bytes += count * sizeof(InstDesc) + part_total * sizeof(double) + snap_total * sizeof(float);
    *out = b;
    return SLBM_OK;
}

slbm_status slbm_batch_init_fields(slbm_batch* b, int idx, const double* phi, const double* psi) {
    if (!b) return SLBM_EINVAL;
    if (idx < 0 || idx >= b->count) return bfail(b, SLBM_EINVAL, "instance index out of range");
    slbm_status s = slbm_init_fields(b->dom[idx], phi, psi);
    if (s) return bfail(b, s, b->dom[idx]->err);
    b->active[idx] = 1;
    b->G0[idx] = b->G;
    b->tables_valid = false;
    b->have_snap = false;
    return SLBM_OK;
}

slbm_status slbm_batch_init_fields_device(slbm_batch* b, int idx, const double* phi, const double* psi) {
    if (!b) return SLBM_EINVAL;
    if (idx < 0 || idx >= b->count) return bfail(b, SLBM_EINVAL, "instance index out of range");
    slbm_status s = slbm_init_fields_device(b->dom[idx], phi, psi);
    if (s) return bfail(b, s, b->dom[idx]->err);
    b->active[idx] = 1;
    b->G0[idx] = b->G;
    b->tables_valid = false;
    b->have_snap = false;
    return SLBM_OK;
}

slbm_status slbm_batch_set_tiling(slbm_batch* b, int band_rows, int ctas_per_sm, int graph_steps) {
    if (!b) return SLBM_EINVAL;
    if (band_rows < 8 || ctas_per_sm < 1 || ctas_per_sm > max_ctas_per_sm(b->strip_width) || graph_steps < 1)
        return bfail(b, SLBM_EINVAL, "need band_rows >= 8, ctas_per_sm in 1 .. 2 (3 for 32-column strips), graph_steps >= 1");
    b->band_rows = band_rows;
    b->ctas_per_sm = ctas_per_sm;
    b->graph_steps = graph_steps;
    b->tables_valid = false;
    return SLBM_OK;
}

slbm_status slbm_batch_set_strip_width(slbm_batch* b, int width) {
    if (!b) return SLBM_EINVAL;
    if (width != 32 && width != 64 && width != 128) return bfail(b, SLBM_EINVAL, "strip width must be 32, 64 or 128");
    b->strip_width = width;
    if (b->ctas_per_sm > max_ctas_per_sm(width)) b->ctas_per_sm = max_ctas_per_sm(width);
    b->tables_valid = false;
    drop_graph(b);
    return SLBM_OK;
}

slbm_status slbm_batch_get_tiling(const slbm_batch* b, int* strip_width, int* band_rows, int* ctas_per_sm) {
    if (!b) return SLBM_EINVAL;
    if (strip_width) *strip_width = b->strip_width;
    if (band_rows) *band_rows = b->band_rows;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    return SLBM_OK;
}

slbm_status slbm_batch_step(slbm_batch* b, long long nsteps) {
    if (!b) return SLBM_EINVAL;
    if (nsteps < 0) return bfail(b, SLBM_EINVAL, "nsteps must be >= 0");
    return run_steps(b, nsteps);
}

slbm_status slbm_batch_run_to_equilibrium(slbm_batch* b, double tol, long long max_steps, int check_every,
                                          long long* steps_out) {
    if (!b || !steps_out) return b ? bfail(b, SLBM_EINVAL, "steps_out is NULL") : SLBM_EINVAL;
    if (check_every < 1 || !(tol > 0)) return bfail(b, SLBM_EINVAL, "need check_every >= 1 and tol > 0");
    for (int i = 0; i < b->count; ++i) steps_out[i] = b->active[i] ? -1 : 0;
    std::vector<double> r;
    slbm_status s = residuals(b, check_every, r);   // first snapshot
    if (s) return s;
    long long done = 0;
    while (done < max_steps) {
        bool any = false;
        for (int i = 0; i < b->count; ++i) any = any || b->active[i];
        if (!any) break;
        const long long chunk = std::min<long long>(check_every, max_steps - done);
        s = run_steps(b, chunk);
        if (s) return s;
        done += chunk;
        s = residuals(b, chunk, r);
        if (s) return s;
        bool changed = false;
        for (int i = 0; i < b->count; ++i) {
            if (!b->active[i]) continue;
            if (r[i] < tol || std::isnan(r[i])) {
                steps_out[i] = std::isnan(r[i]) ? -2 : b->dom[i]->n;   // NaN residual: diverged
                b->active[i] = 0;
                changed = true;
            }
        }
        if (changed) b->tables_valid = false;
    }
    return SLBM_OK;
}

slbm_status slbm_batch_autotune(slbm_batch* b, const char* cache_path, int* band_rows_out, int* ctas_out) {
    if (!b) return SLBM_EINVAL;
    const std::string sig = signature(b);
    auto apply = [&](int width, int br, int cs) {
        slbm_batch_set_strip_width(b, width);
        slbm_batch_set_tiling(b, br, cs, b->graph_steps);
        if (band_rows_out) *band_rows_out = br;
        if (ctas_out) *ctas_out = cs;
    };
    // cached choice?  lines "key": [band_rows, ctas_per_sm, strip_width] (a two-entry line:
    // 64-column strips)
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            int br = 0, cs = 0, width = 64;
            char key[256] = {0};
            const int got = std::sscanf(line.c_str(), " \"%255[^\"]\": [%d, %d, %d]", key, &br, &cs, &width);
            if (got >= 3 && sig == key && (width == 32 || width == 64 || width == 128)) {
                apply(width, br, cs);
                return SLBM_OK;
            }
        }
    }
    // candidates: strip width (the tile's x extent) x band height (its y extent, i.e. the
    // band_rows / 4 cells each thread marches per piece) x resident CTAs per SM
    const int bands[] = {16, 32, 64, 128, 256};
    double best = INFINITY;
    int best_w = b->strip_width, best_br = b->band_rows, best_cs = b->ctas_per_sm;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int width : {64, 32, 128}) {
        slbm_batch_set_strip_width(b, width);
        for (int cs = 1; cs <= max_ctas_per_sm(width); ++cs) {
            for (int br : bands) {
                slbm_batch_set_tiling(b, br, cs, b->graph_steps);
                slbm_status s = run_steps(b, 2);    // build tables, warm up
                if (s) return s;
                cudaEventRecord(e0, b->stream);
                s = run_steps(b, 6);
                if (s) return s;
                cudaEventRecord(e1, b->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_w = width;
                    best_br = br;
                    best_cs = cs;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply(best_w, best_br, best_cs);
    if (cache_path) {
        // append the choice (a JSON object, one key per line)
        std::vector<std::string> lines;
        {
            std::ifstream in(cache_path);
            std::string line;
            while (std::getline(in, line))
                if (line.find("\": [") != std::string::npos) lines.push_back(line);
        }
        for (auto& l : lines)
            if (!l.empty() && l.back() == ',') l.pop_back();
        char buf[320];
        std::snprintf(buf, sizeof(buf), "  \"%s\": [%d, %d, %d]", sig.c_str(), best_br, best_cs, best_w);
        lines.push_back(buf);
        std::ofstream outf(cache_path);
        outf << "{\n";
        for (size_t k = 0; k < lines.size(); ++k) outf << lines[k] << (k + 1 < lines.size() ? ",\n" : "\n");
        outf << "}\n";
    }
    return SLBM_OK;
}

slbm_status slbm_batch_read_fields(slbm_batch* b, int idx, double* phi, double* psi, double* ux, double* uy,
                                   double* p) {
    if (!b) return SLBM_EINVAL;
    if (idx < 0 || idx >= b->count) return bfail(b, SLBM_EINVAL, "instance index out of range");
    slbm_status s = slbm_read_fields(b->dom[idx], phi, psi, ux, uy, p);
    return s ? bfail(b, s, b->dom[idx]->err) : SLBM_OK;
}

slbm_status slbm_batch_read_totals(slbm_batch* b, int idx, slbm_totals* t) {
    if (!b) return SLBM_EINVAL;
    if (idx < 0 || idx >= b->count) return bfail(b, SLBM_EINVAL, "instance index out of range");
    slbm_status s = slbm_read_totals(b->dom[idx], t);
    return s ? bfail(b, s, b->dom[idx]->err) : SLBM_OK;
}

slbm_status slbm_batch_step_instance(slbm_batch* b, int idx, long long nsteps) {
    if (!b) return SLBM_EINVAL;
    if (idx < 0 || idx >= b->count) return bfail(b, SLBM_EINVAL, "instance index out of range");
    slbm_status s = slbm_step(b->dom[idx], nsteps);
    if (s) return bfail(b, s, b->dom[idx]->err);
    b->G0[idx] -= nsteps;        // keep n = G - G0 for the batch kernel
    b->tables_valid = false;
    return SLBM_OK;
}

int slbm_batch_active(const slbm_batch* b, int* flags) {
    if (!b) return 0;
    int n = 0;
    for (int i = 0; i < b->count; ++i) {
        if (flags) flags[i] = b->active[i];
        n += b->active[i];
    }
    return n;
}

size_t slbm_batch_device_bytes(const slbm_batch* b) { return b ? b->bytes : 0; }

const char* slbm_batch_last_error(const slbm_batch* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

void slbm_batch_destroy(slbm_batch* b) {
    if (!b) return;
    drop_graph(b);
    for (slbm_domain* d : b->dom) slbm_destroy(d);
    cudaFree(b->d_inst);
    cudaFree(b->d_pieces);
    cudaFree(b->d_partials);
    cudaFree(b->d_counters);
    cudaFree(b->d_res);
    cudaFree(b->d_queue);
    cudaFree(b->d_G);
    cudaFree(b->d_snap_base);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
