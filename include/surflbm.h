/*
 * surflbm.h - C ABI of the B300 (sm_103a) solver for the coupled phase-field /
 * surfactant / flow lattice Boltzmann model of Huang, Chai, Liu and Huang,
 * "A thermodynamically consistent and conservative phase-field model for surfactant
 * contact line dynamics with solid adsorption".
 *
 * One call of slbm_step advances the three coupled D2Q9 MRT lattice Boltzmann
 * equations of Sec. 3 by one or more time steps on the GPU:
 *   - the conservative Allen-Cahn equation for the phase field phi with the weighted
 *     nonlinear Lagrange multiplier lambda_phi = int h' mu / int h'^2 (Eqs. AC_phi, eq15),
 *   - the Allen-Cahn equation for the surfactant psi with the linear constraint
 *     mubar_psi = mean(mu_psi) (Eq. AC_psi),
 *   - the incompressible Navier-Stokes flow driven by F = -phi grad mu_phi - psi grad mu_psi
 *     (Eqs. eqns, eq_Fs0),
 * with the wetting and solid-adsorption boundary conditions of Eq. boundary.
 *
 * Geometry (lattice units, dx = dt = 1): nx x ny nodes, node (i, j) at x = i,
 * y = j + 1/2; x is periodic; solid walls lie at y = 0 (wall 0, bottom) and y = ny
 * (wall 1, top).  Host arrays are row-major [ny][nx] doubles (index j * nx + i).
 *
 * Conventions: every call returns an slbm_status; nothing throws across the ABI.
 * The library owns all device state of a domain (allocated in slbm_create_domain);
 * the caller owns every host buffer it passes, which the library only reads or writes
 * during the call.  Work is queued on the CUDA stream given at creation (NULL = the
 * legacy default stream); calls that return data synchronise that stream.  A domain
 * must not be used from two threads at once.  After SLBM_ECUDA the domain should be
 * destroyed.  slbm_last_error returns a message owned by the domain (or a static
 * message for a NULL domain) valid until the next call on that domain.
 */
#ifndef SURFLBM_H
#define SURFLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SLBM_OK = 0,
    SLBM_EINVAL = 1,    /* bad argument or parameter                                  */
    SLBM_ENOMEM = 2,    /* device allocation failed                                   */
    SLBM_ECUDA = 3,     /* a CUDA runtime call failed                                 */
    SLBM_EUNSTABLE = 4, /* a reduced quantity became non-finite or a population left  */
                        /* the fixed-point exchange range (the run has diverged)      */
    SLBM_ESTATE = 5     /* call not valid in the current state (e.g. fields not set)  */
} slbm_status;

/* Storage of the moving populations and of the source-term history.
 * FP32: 32-bit floats.  FP16DEV / BF16DEV: 16-bit floats holding deviations from
 * the rest equilibrium w_i m of each scalar set (and the flow populations, whose
 * rest equilibrium at zero reference pressure is 0).  In every mode the conserved
 * zeroth moments are kept in 48-bit float-float, collisions are done in FP32 and
 * global integrals in FP64. */
typedef enum { SLBM_FP32 = 0, SLBM_FP16DEV = 1, SLBM_BF16DEV = 2 } slbm_precision;

/* h_phi of Eq. conservation: nonlinear h = 1/2 + g(phi) (Eq. AC_phi, the paper's
 * model) or linear h = phi (the classical constraint it is compared with). */
typedef enum { SLBM_CONSTRAINT_NONLINEAR = 0, SLBM_CONSTRAINT_LINEAR = 1 } slbm_constraint;

/* lambda_phi: PAPER = Eq. eq15, lambda = S1 / S2.  TARGET = (S1 + (H0 - H) / M_phi) / S2,
 * which feeds back the discrete drift of H = sum h_phi(phi) away from its initial
 * value H0 (the paper's identity holds for the continuous equation only).
 * EXACT = the root, nearest the TARGET value, of H(phi^{n+1}) = H0 for the lattice
 * field itself (the constraint of Sec. 2 in discrete form): phi^{n+1} is affine in
 * lambda^n, so this is a cubic (nonlinear constraint) or linear equation whose four
 * coefficients one extra reduction pass per step sums (44 B per cell of reads with FP32
 * storage, 28 B with 16-bit); H then stays at H0 up to the FP32 rounding of the per-cell
 * terms.  If Newton's method finds no root, the step keeps the TARGET value and
 * slbm_read_totals returns EUNSTABLE.  Single domains only (slbm_create_batch rejects
 * it). */
typedef enum { SLBM_MULT_PAPER = 0, SLBM_MULT_TARGET = 1, SLBM_MULT_EXACT = 2 } slbm_multiplier;

/* Input staging of the step kernel (same results either way; bit-identical fields).
 * CPASYNC (default): every thread stages the rows of the next iteration with 16-byte
 * cp.async copies and the collide loads its flow populations from global memory.
 * TMA: tensor-memory-access tile copies (cp.async.bulk.tensor) issued by the warps' lane 0s
 * complete mbarriers: the stage-K rows (single buffer) and the collide's flow rows (double
 * buffer, one iteration ahead); the periodic-seam columns arrive by cp.async.  Applies to
 * single domains with nx a multiple of 64 and >= 128 (others use CPASYNC).  On the
 * 4096 x 2048 benchmark it is slower (764 vs 691 us per step): the kernel is bounded by
 * DRAM traffic and issue together, and the tile copies of 320-byte rows stall the
 * issuing warps. */
typedef enum { SLBM_STAGING_CPASYNC = 0, SLBM_STAGING_TMA = 1 } slbm_staging;

typedef struct {
    int nx, ny;              /* grid, nx >= 1, ny >= 2                                  */
    double tau_f;            /* flow relaxation time of the liquid, 1/s2^1 (> 0.5)       */
    double tau_f_gas;        /* of the gas; <= 0 means tau_f                            */
    double tau_g, tau_h;     /* phase field 1/s1^2, surfactant 1/s1^3 (> 0.5)           */
    /* remaining MRT rates, (s0, s1, s3, s4) for the flow and (s0, s2, s3, s4) for the
     * scalars; 0 means equal to the field's main rate (all 0: BGK)                   */
    double mrt_f[4], mrt_g[4], mrt_h[4];
    double sigma;            /* clean gas-liquid tension sigma_gl,0 (>= 0)               */
    double eps;              /* interface thickness parameter epsilon (> 0)              */
    double Ex, Pi;           /* W = 4 beta / Ex (Ex <= 0: W = 0), k_B T = 4 beta Pi      */
    double M_phi;            /* used only when kappa = 0; else M_phi kappa = eta c_s^2 (tau_g - 1/2) */
    double M_psi;            /* surfactant mobility; M_0 = eta c_s^2 (tau_h - 1/2) - M_psi lambda_s */
    double eta_phi, eta_psi; /* equilibrium parameters of Sec. 3 (paper leaves them free; 1) */
    double lambda_s;         /* < 0: kappa / 2 (Sec. 2.1)                                */
    double psi_b;            /* reference bulk surfactant for phi_b                     */
    double phi_b;            /* <= 0: sqrt(1 - W psi_b / (4 beta (1 - psi_b))) (Sec. 2.2) */
    double rho_l, rho_g;     /* densities of liquid and gas                             */
    double Gx, Gy;           /* body-force density G                                    */
    int constraint;          /* slbm_constraint                                         */
    int multiplier;          /* slbm_multiplier                                         */
    int precision;           /* slbm_precision                                          */
    int psi_on;              /* 0: surfactant transport disabled (psi == 0)             */
    int wall_saturation;     /* 1: solid tensions capped at half their clean values      */
                             /* (Remark 1; inactive while 1 + beta ln(1 - psi_w) > 1/2)  */
    int staging;             /* slbm_staging: how the step kernel stages its input rows  */
} slbm_params;

/* Quantities reduced in FP64 over the whole grid at one time level. */
typedef struct {
    long long step;          /* number of completed time steps                          */
    double Q_phi;            /* sum of Q(phi) = 2 h_phi(phi) - 1 (Eq. conservation_Q)   */
    double H;                /* sum h_phi(phi): the conserved measure of the constraint */
    double phi_total;        /* sum phi                                                 */
    double psi_total;        /* sum psi (conserved by Eq. AC_psi)                       */
    double lambda_phi;       /* Lagrange multiplier of Eq. eq15 at this time level; in  */
                             /* EXACT mode after >= 1 step: the root the last step used */
    double mubar_psi;        /* mean surfactant chemical potential (Eq. AC_psi)         */
    double kinetic;          /* sum rho |u|^2 / 2                                       */
    double S1, S2;           /* sum h' mu_phi, sum h'^2                                 */
    long long clamp_count;   /* cells whose psi was clamped inside ln(psi / (1 - psi))  */
    long long range_count;   /* non-finite values or fixed-point range violations       */
    double free_energy;      /* discrete E_f of Eq. eq1: cell sums of the bulk densities */
                             /* with kappa/2 |grad phi|^2, lambda_s/2 |grad psi|^2 (the */
                             /* isotropic gradient with the wetting ghosts), plus the   */
                             /* wall energy f_w (Eq. eq8) of both wall rows             */
    double residual;         /* ||phi^n - phi^{n-1}||_2 / ||phi^n||_2 (0 at step 0)      */
} slbm_totals;

typedef struct slbm_domain slbm_domain;

/* Sets every field of *p to the documented defaults for an nx x ny grid
 * (tau = 0.8 everywhere, sigma = 0.01, eps = 4, Ex = 1, Pi = 0.18407, M_psi = 0.5,
 * eta = 1, derived lambda_s and phi_b, unit densities, no body force, nonlinear
 * constraint, paper multiplier, FP32, surfactant on). */
void slbm_default_params(slbm_params* p, int nx, int ny);

/* Validates *p and allocates the device state.  stream: a cudaStream_t or NULL.
 * Errors: EINVAL (bad parameters; message in slbm_last_error(NULL)), ENOMEM, ECUDA.
 * On error *out is set to NULL. */
slbm_status slbm_create_domain(const slbm_params* p, void* stream, slbm_domain** out);

/* Bytes of caller-owned device workspace a domain with parameters *p needs on the
 * current device (all state, scratch and the field read-back buffer), rounded up to
 * 256; 0 if *p is invalid.  The figure depends on the device's SM count (it sizes the
 * per-CTA reduction scratch), so query it with the device that will run the domain. */
size_t slbm_workspace_bytes(const slbm_params* p);

/* As slbm_create_domain, but every device buffer of the domain is carved from
 * `workspace`, `bytes` bytes of device memory the caller owns (e.g. a tensor of a host
 * framework's caching allocator), 256-byte aligned, at least slbm_workspace_bytes(p).
 * The library then never allocates or frees device memory for this domain: slbm_destroy
 * releases only the host-side handle and the workspace stays the caller's (it must
 * outlive the domain and not be used for anything else meanwhile).
 * Errors: EINVAL (bad parameters, NULL or unaligned workspace), ENOMEM (workspace
 * smaller than needed; message states both sizes), ECUDA. */
slbm_status slbm_create_domain_ext(const slbm_params* p, void* workspace, size_t bytes, void* stream,
                                   slbm_domain** out);

/* Sets one wall (0 bottom, 1 top): clean contact angle theta0 in degrees (0, 180),
 * solid adsorption elasticities beta_sg, beta_sl >= 0 of Eq. langmuir, and the
 * tangential wall speed u_x.  sigma_sg0, sigma_sl0 follow from Young's relation and
 * sigma_sg0 + sigma_sl0 = 16 sigma / 15 (Sec. 4.4).  Default: 90 deg, 0, 0, 0.
 * Takes effect from the next step; call before slbm_init_fields for a moving wall so
 * that the initial state is at rest in the wall frame as documented there. */
slbm_status slbm_set_walls(slbm_domain* d, int wall, double theta0_deg,
                           double beta_sg, double beta_sl, double u_x);

/* Copies the initial fields (host, ny*nx doubles each; psi may be NULL when psi_on = 0)
 * and sets the state to the equilibria at rest (u = 0, p = 0) of those fields at
 * step 0, as the pre-collision populations of time 0.  Resets the step counter. */
slbm_status slbm_init_fields(slbm_domain* d, const double* phi, const double* psi);

/* As slbm_init_fields with phi and psi in DEVICE memory of this domain's device
 * (row-major [ny][nx] doubles); used to start from a state computed on the GPU. */
slbm_status slbm_init_fields_device(slbm_domain* d, const double* phi, const double* psi);

/* Queues nsteps >= 0 time steps on the domain's stream (asynchronous): one launch of the
 * fused step kernel per step, plus the exact multiplier's reduction pass after it when
 * multiplier = SLBM_MULT_EXACT.  Returns the status of previously completed work only
 * when it is already known (ECUDA on a launch failure); divergence is reported by
 * slbm_read_totals.  ESTATE if the fields were never initialised. */
slbm_status slbm_step(slbm_domain* d, long long nsteps);

/* Computes phi, psi, u_x, u_y and p at the current time level (the moments of the
 * current populations, Sec. 3) and copies them to the host arrays (ny*nx doubles
 * each; any pointer may be NULL).  Synchronises the stream. */
slbm_status slbm_read_fields(slbm_domain* d, double* phi, double* psi,
                             double* ux, double* uy, double* p);

/* Reduces the totals at the current time level into *t.  Synchronises.
 * Returns EUNSTABLE (with *t filled) when range_count > 0 or a total is non-finite. */
slbm_status slbm_read_totals(slbm_domain* d, slbm_totals* t);

/* Fields and totals at the current time level, written into device memory the
 * caller owns, without allocating anything.  (The paper has no counterpart: this is
 * an interface for callers, not part of the method.)
 *
 * For callers that cannot call cudaMalloc once they are running: host frameworks or
 * memory pools that own and budget all device memory and forbid allocation after
 * set-up, and loops where the device-wide synchronisation an allocation or free can
 * imply would stall other streams.  slbm_read_fields allocates a 5 * nx * ny double
 * buffer on its first call; this variant writes straight into the caller's buffers.
 *
 * phi, psi, ux, uy, p: DEVICE pointers (this domain's device), nx*ny doubles each,
 * row-major [ny][nx]; any may be NULL (then that field is not written).  totals: host
 * pointer or NULL.  With totals != NULL the call synchronises the domain's stream and
 * fills *totals (same meaning and status rules as slbm_read_totals); with NULL it only
 * queues the work on the stream.
 *
 * Scratch: the per-CTA partial sums, the completion counter and the result record live
 * in one file-scope static device array of SLBM_NOALLOC_SCRATCH_BYTES (about 105 KB),
 * held by every GPU that loads this library until the process exits.  The array holds
 * at most SLBM_NOALLOC_MAX_CTAS CTAs of partials; a domain whose grid is larger is
 * rejected with SLBM_EINVAL (grids here are at most 2 CTAs per SM).  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current, so that first call should come before any stream capture.  Every call on a
 * device shares the one array and it keeps the last call's contents (the counter is
 * cleared at the start of each call): calls that overlap on the GPU, from any domain
 * or stream, race and must be serialised by the caller.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 * Errors: EINVAL (NULL domain, grid too large), ESTATE (fields never initialised),
 * ECUDA, EUNSTABLE (as slbm_read_totals). */
#define SLBM_NOALLOC_MAX_CTAS 1024
#define SLBM_NOALLOC_PARTS 13
#define SLBM_NOALLOC_SCRATCH_BYTES (SLBM_NOALLOC_MAX_CTAS * SLBM_NOALLOC_PARTS * 8 + 256 + 256)
slbm_status slbm_read_fields_noalloc(slbm_domain* d, double* phi, double* psi, double* ux, double* uy,
                                     double* p, slbm_totals* totals);

/* ------------------------------------------------------------------------------
 * Batches: many independent domains (instances; grid sizes, parameters and walls may
 * all differ, precision may not) advanced together by one launch of a persistent
 * tile-queue kernel per time step.  Every instance follows exactly the update of
 * slbm_step (Sec. 3; its global multipliers are reduced per instance in a fixed
 * order), so a batch gives the same fields as stepping each instance alone up to the
 * rounding of the reduction order.  Steps are replayed from a captured CUDA graph of
 * graph_steps launches.  Instances are numbered 0 .. count-1.
 * ---------------------------------------------------------------------------- */
typedef struct slbm_batch slbm_batch;

/* One wall of one instance (see slbm_set_walls). */
typedef struct {
    double theta0_deg, beta_sg, beta_sl, u_x;
} slbm_wall_spec;

/* params: count instances; walls: 2 * count entries (bottom, top of each instance), or
 * NULL for neutral walls.  stream: a cudaStream_t, or NULL for a stream the batch
 * creates and owns (graph capture needs a non-default stream).  Allocates the state of
 * every instance.  Errors: EINVAL (message in slbm_batch_last_error(NULL)), ENOMEM, ECUDA. */
slbm_status slbm_create_batch(const slbm_params* params, const slbm_wall_spec* walls, int count, void* stream,
                              slbm_batch** out);

/* Initial fields of instance idx (as slbm_init_fields); the instance becomes active and
 * its time level 0 is the batch's current step. */
slbm_status slbm_batch_init_fields(slbm_batch* b, int idx, const double* phi, const double* psi);
/* As slbm_batch_init_fields with phi, psi in device memory (slbm_init_fields_device). */
slbm_status slbm_batch_init_fields_device(slbm_batch* b, int idx, const double* phi, const double* psi);

/* Tiling of the tile queue: each instance is cut into strips of the strip width (64
 * columns by default, see slbm_batch_set_strip_width) and bands of about band_rows rows
 * (>= 8), so a piece is a tile of width x band_rows cells and each thread of the CTA
 * marching it (4 rows per step of its pipeline) handles band_rows / 4 cells of it;
 * ctas_per_sm resident CTAs per SM (1 or 2 with 64-column strips, 1 to 3 with 32, 1 with
 * 128) take
 * pieces from the queue; graph_steps launches per captured graph. */
slbm_status slbm_batch_set_tiling(slbm_batch* b, int band_rows, int ctas_per_sm, int graph_steps);

/* Strip width of the tile queue: 64 (the step kernel with 256 threads per CTA), 32 (its
 * 32-column instance, 128 threads per CTA, more pieces and smaller shared-memory rings for
 * narrow instances at twice the relative halo) or 128 (512 threads, one CTA per SM, half
 * the relative halo for wide instances).  Same method; fields agree to FP32 rounding
 * (the tiling fixes the order of the per-thread partial sums).  Clamps ctas_per_sm to the
 * width's maximum.  EINVAL for other widths. */
slbm_status slbm_batch_set_strip_width(slbm_batch* b, int width);

/* The current tiling: strip width, band rows, resident CTAs per SM (any may be NULL). */
slbm_status slbm_batch_get_tiling(const slbm_batch* b, int* strip_width, int* band_rows, int* ctas_per_sm);

/* Times the candidate tilings (strip width 64, 32 or 128 x band_rows 16..256 x every allowed
 * CTAs-per-SM count) on this batch and keeps the fastest; the choice is read from /
 * appended to the JSON file cache_path (may be NULL) as [band_rows, ctas_per_sm,
 * strip_width], keyed by precision, instance count, total cells and the size list.  The
 * timed steps are real steps of every active instance (8 per candidate). */
slbm_status slbm_batch_autotune(slbm_batch* b, const char* cache_path, int* band_rows_out, int* ctas_out);

/* nsteps time steps of every active instance (asynchronous on the batch's stream). */
slbm_status slbm_batch_step(slbm_batch* b, long long nsteps);

/* Steps the active instances until each one's residual (max over phi and psi of
 * ||x^n - x^{n-K}||_2 / (K ||x^n||_2), K = check_every) falls below tol, retiring each
 * as it converges, or until max_steps more steps.  steps_out[i] (count entries): the
 * instance's step count at convergence, -1 if it did not converge, -2 if its fields
 * became non-finite (the instance diverged; it is retired at the check that sees it),
 * 0 if it was inactive. */
slbm_status slbm_batch_run_to_equilibrium(slbm_batch* b, double tol, long long max_steps, int check_every,
                                          long long* steps_out);

/* nsteps steps of instance idx alone with its own launches (as slbm_step), keeping the
 * batch's step bookkeeping consistent; the per-instance-launch baseline of the batch. */
slbm_status slbm_batch_step_instance(slbm_batch* b, int idx, long long nsteps);

/* Fields / totals of instance idx at its current time level (as slbm_read_fields /
 * slbm_read_totals; synchronise). */
slbm_status slbm_batch_read_fields(slbm_batch* b, int idx, double* phi, double* psi, double* ux, double* uy,
                                   double* p);
slbm_status slbm_batch_read_totals(slbm_batch* b, int idx, slbm_totals* t);

/* Number of active instances; flags (count ints, may be NULL) receives 1 / 0 each. */
int slbm_batch_active(const slbm_batch* b, int* flags);
size_t slbm_batch_device_bytes(const slbm_batch* b);
const char* slbm_batch_last_error(const slbm_batch* b);
void slbm_batch_destroy(slbm_batch* b);

/* Verification hook: the manufactured-solution accuracy test of Sec. 4.1 on the channel.
 * With m != NULL the domain's steps solve the phi and psi equations driven by the sources
 * that make
 *     phi^e = A e^{-t} sin 2pi(x - u t) cos 2pi y,  psi^e = 1/2 + 0.05 e^{-2t} cos 2pi(x - u t) cos 2pi y
 * exact (physical x, y in [0, 1], node (i, j) at x = i dx, y = (j + 1/2) dx, t = n dt), with
 * mobility M, beta, kappa, k_B T, W (physical units) and the linear multipliers of that
 * test; no force acts on the flow, and the next slbm_init_fields starts the flow at the
 * uniform lattice velocity u dt / dx (set both walls to slide at it).  The caller chooses
 * the lattice parameters so that the lattice equations are those of the test (sigma, eps
 * from beta and kappa / dx^2, Ex = 4 beta / W, Pi = k_B T / (4 beta), tau_g = tau_h = 1,
 * eta_phi = eta_psi = 6 M kappa dt / dx^2, M_psi = M dt, lambda_s = 0, linear constraint).
 * FP32 storage and uniform density only (EINVAL otherwise); m == NULL switches it off. */
typedef struct {
    double amplitude, u, M, beta, kappa, kT, W, dx, dt;
} slbm_mms;
slbm_status slbm_set_mms(slbm_domain* d, const slbm_mms* m);

/* Checkpoint / resume.  slbm_save writes the complete state at the current time level
 * (parameters, walls, step count, populations, zeroth moments, previous phi, source-term
 * history and the multiplier records of the last two levels) to a binary file; the
 * file is specific to this library version.  slbm_load restores such a file into a
 * domain created with the same parameters (every field of slbm_params equal; the walls
 * are taken from the file), after which stepping continues exactly as the saved run
 * would have: N steps, save, load, N steps gives bit-identical fields to 2N steps.
 * Both synchronise the stream.  Errors: EINVAL (NULL path, unreadable or foreign file,
 * parameter mismatch, I/O failure), ESTATE (save before initialisation), ECUDA. */
slbm_status slbm_save(slbm_domain* d, const char* path);
slbm_status slbm_load(slbm_domain* d, const char* path);

/* Bytes of device memory the domain holds. */
size_t slbm_device_bytes(const slbm_domain* d);

/* Number of device allocations (cudaMalloc calls) the library has made in this process,
 * for every domain, batch and network together: a caller that must not allocate once
 * running (domains built with slbm_create_domain_ext, slbm_read_fields_noalloc) can check
 * that the count does not move across its calls.  Thread-safe. */
unsigned long long slbm_device_allocations(void);

/* Releases everything the domain owns (NULL is a no-op). */
void slbm_destroy(slbm_domain* d);

/* Message describing the last error on d (or of the last create when d is NULL). */
const char* slbm_last_error(const slbm_domain* d);

/* Library version string. */
const char* slbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SURFLBM_H */
