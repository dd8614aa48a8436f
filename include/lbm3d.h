/*
 * C ABI of the three-dimensional form of the coupled step: a D3Q19
 * multiple-relaxation-time pseudopotential flow lattice (the paper's Section 2
 * model with the d'Humieres moment basis and the Li forcing) coupled to a D3Q7
 * temperature lattice with the rho c_v-weighted streaming of Eq. 39.  The
 * paper states that the model extends to three dimensions (Section 1) and
 * shows only the two-dimensional form; the three-dimensional choices (moment
 * basis, D3Q7 matrix, the sigma term on the energy moment, the wetting ghost
 * layer with a tangential gradient) are the library's readings and are
 * listed in its design notes.
 *
 * Conventions as in lbm.h (return codes, sticky device errors, ownership,
 * asynchronous steps on the context stream), with:
 *  - fields on the host are double arrays [nz][ny][nx], x fastest, node
 *    (0,0,0) at the bottom corner; gravity points to -z;
 *  - populations are [q][nz][ny][nx] (q = 19 for f in the D3Q19 order rest,
 *    +-x, +-y, +-z, then the edge pairs (+-1,+-1,0), (+-1,-+1,0),
 *    (+-1,0,+-1), (+-1,0,-+1), (0,+-1,+-1), (0,+-1,-+1); q = 7 for g: rest,
 *    +-x, +-y, +-z);
 *  - x and y are periodic; z is periodic or bounded by walls at both ends.
 */
#ifndef LBM3D_GB300_H
#define LBM3D_GB300_H

#include <stddef.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* z boundaries: flow_z = LBM_PERIODIC, or LBM_WALL for halfway bounce-back
 * no-slip walls at z = -1/2 and z = nz - 1/2 with the wetting ghost layer of
 * Section 3.3 (rho_ghost = rho(layer 2) + tan(pi/2 - theta) |tangential
 * difference of rho over two spacings at layer 1|).  therm[0] (bottom) and
 * therm[1] (top): LBM_T_PERIODIC exactly when flow_z is periodic, otherwise
 * LBM_T_DIRICHLET (anti-bounce-back to T_edge) or LBM_T_ADIABATIC. */
typedef struct {
    int flow_z;
    int therm[2];
    double T_edge[2];
    double theta_deg;
} lbm3d_bc;

typedef struct lbm3d_ctx lbm3d_ctx;

/* Device bytes of the state of an nx x ny x nz domain at prec (LBM_FP64 or
 * LBM_FP32): two copies of f (19), g (7) and P, 15 per-node scalars (rho, T,
 * psi, T dp/dT, j, 1/(rho c_v), u, F, |F_m|^2/psi^2), plus the psi of the two
 * wall ghost layers.  0 for invalid arguments. */
size_t lbm3d_state_bytes(int nx, int ny, int nz, int prec);

/* Creates a context; stream as in lbm_create (NULL: a library stream).
 * The same lbm_params as the two-dimensional form; sigma enters the energy
 * moment so that a planar interface sees the two-dimensional pressure tensor.
 * Errors: LBM_EINVAL (sizes < 1, prec not FP64/FP32, bad boundaries or
 * parameters), LBM_ENOMEM, LBM_ECUDA. */
int lbm3d_create(int nx, int ny, int nz, const lbm_params* params, const lbm3d_bc* bc,
                 int prec, void* stream, lbm3d_ctx** out);

/* State at t = 0 from host fields [nz][ny][nx]: f = f^eq(rho, u), g = w^ T,
 * P history cleared.  Clears the sticky error.  Synchronises. */
int lbm3d_init_fields(lbm3d_ctx* ctx, const double* rho, const double* ux, const double* uy,
                      const double* uz, const double* T);

/* Queues n coupled steps (asynchronous; CUDA graph of 32 steps replayed for
 * long runs).  LBM_ESTATE before initialisation; returns a sticky error. */
int lbm3d_step(lbm3d_ctx* ctx, int n);

/* rho, the half-force velocity u = (sum c f + F/2)/rho and T of the current
 * state; any pointer may be NULL.  Synchronises; returns the sticky error. */
int lbm3d_get_fields(lbm3d_ctx* ctx, double* rho, double* ux, double* uy, double* uz,
                     double* T);

/* Populations of the current state as absolute values: f [19][nz][ny][nx],
 * g [7][nz][ny][nx], P [nz][ny][nx]; any pointer may be NULL.  Synchronises. */
int lbm3d_get_populations(lbm3d_ctx* ctx, double* f, double* g, double* P);

/* lbm_diag of the current state, in double on the device: liquid_area is the
 * liquid volume (nodes with rho above (rho_l + rho_g)/2) and the diameters
 * are those of the sphere (hemisphere when sessile) of that volume.
 * Synchronises. */
int lbm3d_diagnostics(lbm3d_ctx* ctx, double rho_l, double rho_g, int sessile, lbm_diag* out);

/* Selects how a step runs; the state and its result are the same either way
 * (same arithmetic per node; sums over nodes in another order).  fused != 0
 * (the default in FP32): one kernel per step marching through the z planes
 * of 16 x 16 node tiles, zseg planes per CTA (0: chosen from the domain and
 * the device), recomputing the fields the stencils need around each tile, so
 * that f, g and P are read and written once per step.  fused == 0 (the
 * default in FP64, where the recomputation costs more than the traffic it
 * saves): kernels over the nodes (force and velocity; collisions with the
 * push of f and g; the next state's fields), which keep per-node fields in
 * device memory between them.
 * The steps of Section 3.2 (Eqs. 5, 9, 11, 20, 24, 39, 49-50) in three
 * dimensions; the paper has no counterpart of the choice.  Takes effect at
 * the next lbm3d_step.  LBM_EINVAL for a NULL context or zseg < 0. */
int lbm3d_set_path(lbm3d_ctx* ctx, int fused, int zseg);
/* The current path and planes per CTA (either pointer may be NULL). */
int lbm3d_get_path(const lbm3d_ctx* ctx, int* fused, int* zseg);

long long lbm3d_step_count(const lbm3d_ctx* ctx);
int lbm3d_sync(lbm3d_ctx* ctx);
void lbm3d_destroy(lbm3d_ctx* ctx);
const char* lbm3d_last_error(const lbm3d_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM3D_GB300_H */
