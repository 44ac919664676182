/*
 * surflbm3d.h - C ABI of the three-dimensional extension of the coupled phase-field /
 * surfactant / flow lattice Boltzmann solver (B300, sm_103a).
 *
 * Sec. 2.3 of Huang, Chai, Liu and Huang states the model for d = 2 and 3 and Sec. 3
 * writes its lattice Boltzmann scheme for a DdQq lattice; the paper's own runs are
 * two-dimensional and its conclusion names three-dimensional flows as future work.  This
 * is the same scheme (Eqs. AC_phi with the multiplier of Eq. eq15, AC_psi, the flow of
 * Eq. eqns with the force of Eq. eq_Fs0, the walls of Eq. boundary) on the D3Q19 lattice
 * for all three distribution sets, with the single-relaxation-time collision (the MRT of
 * Sec. 3 with all rates of a set equal).
 *
 * Geometry (lattice units): nx x ny x nz nodes, node (i, j, l) at x = i, y = j + 1/2,
 * z = l; x and z periodic; solid walls at y = 0 (wall 0) and y = ny (wall 1).  Host
 * arrays are [nz][ny][nx] doubles (index (l * ny + j) * nx + i).  D3Q19 velocities are
 * ordered: rest; +x, -x, +y, -y, +z, -z; (+1,+1,0), (-1,+1,0), (-1,-1,0), (+1,-1,0);
 * (+1,0,+1), (-1,0,+1), (-1,0,-1), (+1,0,-1); (0,+1,+1), (0,-1,+1), (0,-1,-1), (0,+1,-1).
 *
 * What carries over from the two-dimensional ABI (surflbm.h): the parameter struct
 * slbm_params (its nx, ny are the x and y sizes), the wall model and its closure, the
 * constraint and the PAPER / TARGET multipliers, the status codes, the totals struct and
 * the conventions on ownership, streams and errors.  Restrictions of this extension
 * (EINVAL at creation otherwise): FP32 storage, one relaxation time per set (all mrt_*
 * rates 0), uniform density and viscosity (rho_l == rho_g, tau_f_gas <= 0 or == tau_f),
 * multiplier PAPER or TARGET; the free energy and residual of the totals are not computed
 * (0).  Sum psi, and sum phi under the linear constraint, are conserved to float-float
 * rounding as in two dimensions (fixed-point exchange of every streamed population).
 *
 * A step is three kernel launches on the domain's stream: the moments phi, psi (pull);
 * the chemical potentials, free reaction terms and FP64 integrals, whose last block
 * resolves lambda_phi and mubar_psi of the step; the collision of the three sets with
 * their sources and the pull of the flow set.
 */
#ifndef SURFLBM3D_H
#define SURFLBM3D_H

#include "surflbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slbm3d_domain slbm3d_domain;

/* Validates *p (as slbm_create_domain, plus the restrictions above; nz >= 1,
 * nx * ny * nz <= 2^27) and allocates the device state on the current device.
 * stream: a cudaStream_t or NULL.  Errors: EINVAL (message in slbm3d_last_error(NULL)),
 * ENOMEM, ECUDA.  On error *out is NULL. */
slbm_status slbm3d_create_domain(const slbm_params* p, int nz, void* stream, slbm3d_domain** out);

/* As slbm_set_walls: wall 0 (bottom) or 1 (top), clean contact angle in degrees (0, 180),
 * adsorption elasticities >= 0, tangential wall speed along x (|u_x| < 0.3). */
slbm_status slbm3d_set_walls(slbm3d_domain* d, int wall, double theta0_deg, double beta_sg, double beta_sl,
                             double u_x);

/* Copies the initial fields (host, nz*ny*nx doubles; psi may be NULL when psi_on = 0)
 * and sets the state to the equilibria at rest of those fields at step 0. */
slbm_status slbm3d_init_fields(slbm3d_domain* d, const double* phi, const double* psi);

/* Queues nsteps >= 0 time steps (three launches each) on the stream.  ESTATE before
 * slbm3d_init_fields; ECUDA on a launch failure. */
slbm_status slbm3d_step(slbm3d_domain* d, long long nsteps);

/* phi, psi, u_x, u_y, u_z, p at the current time level into host arrays of nz*ny*nx
 * doubles (any may be NULL).  Synchronises the stream. */
slbm_status slbm3d_read_fields(slbm3d_domain* d, double* phi, double* psi, double* ux, double* uy, double* uz,
                               double* p);

/* Totals at the current time level (sums in FP64; free_energy and residual are 0).
 * Synchronises.  EUNSTABLE (with *t filled) when a total is non-finite or a velocity,
 * phi or p left its range. */
slbm_status slbm3d_read_totals(slbm3d_domain* d, slbm_totals* t);

/* Bytes of device memory the domain holds. */
size_t slbm3d_device_bytes(const slbm3d_domain* d);

/* Releases the domain (NULL is a no-op). */
void slbm3d_destroy(slbm3d_domain* d);

/* Message of the last error on d (or of the last create when d is NULL). */
const char* slbm3d_last_error(const slbm3d_domain* d);

#ifdef __cplusplus
}
#endif

#endif
