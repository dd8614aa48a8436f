/*
 * C ABI of the GB300 (sm_103a) implementation of the coupled time step of the
 * thermal lattice Boltzmann model for liquid-vapor phase change of Wang, Huang
 * & He (arXiv 2205.00686): a D2Q9 multiple-relaxation-time pseudopotential
 * flow lattice (Section 2) coupled to the paper's D2Q5 multiple-relaxation-
 * time temperature lattice with the rho c_v-weighted streaming (Section 3.2,
 * Eq. 39), with the wetting, Dirichlet, open, periodic and no-slip boundaries
 * of Sections 3.3 and 4.
 *
 * Conventions shared by every entry point:
 *  - Fields on the host are row-major double arrays [ny][nx], x fastest, node
 *    (0,0) at the south-west corner; gravity points to -y.
 *  - Populations on the host are double arrays [q][ny][nx] (q = 9 for f, the
 *    D2Q9 order of Eq. 2; q = 5 for g, the D2Q5 order of Eq. 26).
 *  - The caller owns every host array; the library copies what it needs and
 *    keeps no host pointer.  The library owns the device memory it allocates.
 *  - Work is queued on the context's CUDA stream; entry points that return
 *    host data synchronise that stream.
 *  - Every function returns LBM_OK (0) or a negative LBM_E* code and never
 *    throws.  A device-side error (negative psi^2, non-finite state) is sticky:
 *    it is reported by the next synchronising call and clears only on
 *    lbm_init_fields, lbm_set_populations or lbm_load.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define LBM_OK 0
#define LBM_EINVAL (-1)      /* bad argument, size or boundary combination     */
#define LBM_ENOMEM (-2)      /* device or host allocation failed               */
#define LBM_ENONFINITE (-3)  /* a NaN / Inf appeared in rho or T               */
#define LBM_EPSI (-4)        /* psi^2 = 2 (rho c_s^2 - p_EOS) < 0 at some node  */
#define LBM_ECUDA (-5)       /* a CUDA runtime call failed                     */
#define LBM_EIO (-6)         /* checkpoint file could not be read or written  */
#define LBM_ESTATE (-7)      /* call out of order (e.g. step before init)     */
#define LBM_ETOOBIG (-8)     /* size beyond a fixed capacity (no-alloc entry)  */
#define LBM_ETIMEOUT (-9)    /* a bounded device wait ran out (staged rows)    */

/* ---- precision of storage and arithmetic ------------------------------- */
typedef enum {
    LBM_FP64 = 0,      /* f, g, P stored and computed in double             */
    LBM_FP32 = 1,      /* f, g, P stored and computed in float              */
    LBM_FP32_G16 = 2   /* as LBM_FP32, but g stored in IEEE half             */
} lbm_prec;

/* ---- boundaries ---------------------------------------------------------- */
enum { LBM_EDGE_W = 0, LBM_EDGE_E = 1, LBM_EDGE_S = 2, LBM_EDGE_N = 3 };
typedef enum { LBM_PERIODIC = 0, LBM_WALL = 1, LBM_OPEN = 2 } lbm_flow_bc;
typedef enum { LBM_T_PERIODIC = 0, LBM_T_DIRICHLET = 1, LBM_T_ADIABATIC = 2 } lbm_therm_bc;

/* Boundary specification (Sections 3.3 and 4).
 *  flow[e]:  LBM_PERIODIC, LBM_WALL (halfway bounce-back no-slip wall with the
 *            Ding-Spelt wetting ghost layer; south/north edges only) or
 *            LBM_OPEN (zero-gradient extrapolation of the unknown populations).
 *  therm[e]: LBM_T_PERIODIC, LBM_T_DIRICHLET (halfway anti-bounce-back to
 *            T_edge[e]) or LBM_T_ADIABATIC (halfway bounce-back).
 *  Each lattice is periodic along an axis on both of its edges or on neither.
 *  A periodic thermal axis needs a periodic flow axis; a periodic flow axis
 *  may carry Dirichlet or adiabatic thermal edges (Section 4.1: the droplet
 *  in open space streams f periodically and holds T = T_g at the edges).
 *  theta_deg: equilibrium contact angle of walls (Section 3.3).
 *  heater_x0..heater_x1-1: south-edge nodes held at T_heater instead of
 *  T_edge[S] (Section 4.3). */
typedef struct {
    int flow[4];
    int therm[4];
    double T_edge[4];
    double theta_deg;
    int heater_x0, heater_x1;
    double T_heater;
} lbm_bc;

/* ---- physical and numerical parameters (all double) -------------------- *
 * a, b, R, omega: Peng-Robinson EOS (Section 2, Eq. 10), T_c = 0.0778 a /
 *   (0.45724 b R).
 * G, sigma: interaction strength of Eq. 9 and the tunable sigma of Eq. 8.
 * nu: kinematic viscosity, s_p = 1/(3 nu + 1/2).  s0, s_e, s_eps, s_j, s_q: the
 *   other diagonal entries of S (Section 2).
 * lambda: thermal conductivity; varsigma_1 = varsigma_2 = 1/(lambda/c_s^2 +
 *   1/2) with c_s^2 = w_dot/2 (Section 3.2.2).  cv: specific heat.  w_dot: the
 *   D2Q5 rest-weight parameter (w_0 = 1 - w_dot, w_1..4 = w_dot/4).  vs0, vs3,
 *   vs4: the other entries of Lambda.
 * gravity: g of the body force (rho - rho_ave)(0, -g) (Section 4.3).
 * rho_ref, T_ref: storage references; populations are stored as deviations
 *   f_i - w_i rho_ref and g_i - w^_i T_ref.  rho_ref <= 0 means "the mean of
 *   the initial density"; T_ref <= 0 means "the mean of the initial T".
 * frozen_flow (test hook): u = 0 and rho fixed; only g advances.
 * frozen_thermal (isothermal hook): g fixed; only f advances. */
typedef struct {
    double a, b, R, omega;
    double G, sigma;
    double nu, s0, s_e, s_eps, s_j, s_q;
    double lambda, cv, w_dot, vs0, vs3, vs4;
    double gravity;
    double rho_ref, T_ref;
    int frozen_flow, frozen_thermal;
} lbm_params;

/* Diagnostics (Sections 3.3 and 4), accumulated in double on the device:
 * mass = sum rho, energy = sum rho c_v T, liquid_* over nodes with rho above
 * the interface level (rho_l + rho_g)/2, liquid_area_smooth = sum of
 * clamp((rho - rho_g)/(rho_l - rho_g), 0, 1), diameters of the equivalent
 * disc (or half disc when sessile), max_u = max |u|. */
typedef struct {
    double mass, energy, liquid_mass, liquid_area, liquid_area_smooth;
    double diameter, diameter_smooth, max_u;
    long long step;
    int nonfinite;
} lbm_diag;

typedef struct lbm_ctx lbm_ctx;
typedef struct lbm_batch lbm_batch;

/* Fills *p with the paper's constants and the library's readings:
 * a = 3/49, b = 2/21, R = 1, omega = 0.344, G = -1, sigma = 1.25, nu = 0.1,
 * cv = 5, lambda = 1/3, w_dot = 2/3, every other rate 1.0, gravity 0. */
int lbm_default_params(lbm_params* p);

/* Device bytes lbm_create needs for an nx x ny domain at precision prec
 * (both ping-pong copies of f, g and P).  Returns 0 for invalid sizes. */
size_t lbm_state_bytes(int nx, int ny, int prec);

/* Creates a simulation context: one nx x ny domain of the coupled problem of
 * Section 2 (D2Q9 flow lattice, Peng-Robinson EOS, Eqs. 1-11) and Section 3.2
 * (D2Q5 temperature lattice, Eqs. 39-40), with the boundaries of Sections
 * 3.3 and 4 (periodic, halfway bounce-back walls with the wetting ghost
 * layer, open edges, Dirichlet / adiabatic / heater temperatures) given in
 * lbm_bc, the model constants of Section 4 in lbm_params.
 *  stream: a cudaStream_t (as void*) to queue work on, or NULL for a stream
 *          the library creates and owns.  The legacy default stream cannot be
 *          captured into CUDA graphs; pass a created stream.
 *  device_mem / device_bytes: optional caller-owned device buffer of at least
 *          lbm_state_bytes(nx, ny, prec) bytes, 256-byte aligned, to hold the
 *          state (e.g. from a PyTorch allocation); NULL to let the library
 *          allocate.  The caller keeps it alive until lbm_destroy.
 * Errors: LBM_EINVAL (sizes < 1, 9 * ny * round_up(nx, 64) >= 2^31 (e.g.
 * beyond about 15000 x 15000), bad precision, unsupported boundary
 * combination, non-positive cv / nu / lambda, w_dot outside (0,1)),
 * LBM_ENOMEM, LBM_ECUDA.  *out is NULL on failure. */
int lbm_create(int nx, int ny, const lbm_params* params, const lbm_bc* bc, int prec,
               void* stream, void* device_mem, size_t device_bytes, lbm_ctx** out);

/* Sets the state at t = 0 from host fields (each [ny][nx], double):
 * f = f^eq(rho, u) of Eq. 3, g = w^ T (Eq. 22), P history cleared; the first
 * step then takes d_t^2 T = 0.  Clears the sticky error.  Synchronises. */
int lbm_init_fields(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                    const double* T);

/* Queues n coupled time steps (n >= 0), asynchronous on the context stream.
 * One step is the paper's full update: moments (Eqs. 11, 25), EOS and psi
 * (Eq. 10), the interaction force (Eq. 9) with the buoyancy of Section 4.3,
 * the D2Q9 MRT collision with the forcing of Eq. 8 (Eqs. 5, 7) and pull
 * streaming (Eq. 6), the source Q of Eq. 20 with the local gradient of
 * Eqs. 49-50 and S of Eq. 24, the D2Q5 MRT collision and the rho c_v-weighted
 * streaming of Eq. 39.
 * Returns LBM_ESTATE before initialisation, LBM_ECUDA on launch failure; a
 * sticky device error from an earlier step is returned without queuing. */
int lbm_step(lbm_ctx* ctx, int n);

/* Copies rho, u = (sum c f + F/2)/rho (Eq. 11) and T of the current state to
 * host arrays [ny][nx]; any pointer may be NULL.  Synchronises and returns
 * the sticky device error if one is set. */
int lbm_get_rho_u_T(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* T);

/* Diagnostics of the current state; rho_l and rho_g set the interface level
 * and the smooth liquid fraction; sessile selects the half-disc diameter.
 * Synchronises. */
int lbm_diagnostics(lbm_ctx* ctx, double rho_l, double rho_g, int sessile, lbm_diag* out);

/* Populations of the current state as absolute values (not deviations):
 * f [9][ny][nx], g [5][ny][nx], P [ny][nx] (P = Q/(rho c_v) of the last
 * step); any pointer may be NULL.  Synchronises. */
int lbm_get_populations(lbm_ctx* ctx, double* f, double* g, double* P);

/* Replaces the state by host populations (same layout, absolute values),
 * sets the step counter to `step` (step 0 takes d_t^2 T = 0 on its first
 * step) and the mean density of the previous step used by the buoyancy
 * force to rho_ave_prev.  Clears the sticky error.  Synchronises. */
int lbm_set_populations(lbm_ctx* ctx, const double* f, const double* g, const double* P,
                        long long step, double rho_ave_prev);

/* Makes the context stop at step count `target` (> 0; 0 removes the stop):
 * the launches of lbm_step or lbm_batch_step leave a context that has
 * reached it untouched (state, step counter, buoyancy history), so domains
 * with different step counts can share chunks of batched launches and each
 * end exactly at its own.  Ordered with the steps on the stream that runs
 * them (the batch's while attached).  lbm_init_fields, lbm_set_populations
 * and lbm_load remove the stop.  The paper has no counterpart. */
int lbm_set_target(lbm_ctx* ctx, long long target);

/* Number of completed steps. */
long long lbm_step_count(const lbm_ctx* ctx);

/* Waits for queued work; returns the sticky device error, if any. */
int lbm_sync(lbm_ctx* ctx);

/* Checkpoint: a raw binary of the current-state device buffers, the step
 * counter, the buoyancy mass history, params and bc, with a header and a
 * CRC-32.  The paper has no counterpart (it prescribes no implementation);
 * what is saved is the full state the time step of Eqs. 5-6 and 39 reads:
 * f, g, the P^{n-1} history behind S of Eq. 24, and the previous step's
 * density sum behind rho_ave of Section 4.3.  lbm_load requires a context of the same nx, ny and precision and
 * restores it bit for bit.  Both synchronise.  LBM_EIO on file errors or a
 * CRC / header mismatch. */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx* ctx, const char* path);

/* One domain split into slabs of rows, one context per slab.  The paper
 * has no counterpart (it runs one domain on one machine); these calls only
 * move and combine state so that the split computes what one context of
 * the whole domain computes.  A slab context holds its own rows plus halo
 * rows copied from its neighbours before each step (three rows per step
 * between exchanges: the step reads rows up to three away), its inner edges
 * open with adiabatic temperature (they only shape halo rows, which are
 * overwritten), and the same rho_ref / T_ref as the others (set in
 * lbm_params), so that raw rows move between slabs unchanged.
 *
 * Bytes of n rows of every state plane, packed [plane][row][nx] (f 0..8, g
 * 0..4, P^{n-1}; storage types of the context's precision). */
size_t lbm_rows_bytes(const lbm_ctx* ctx, int n);
/* Copies rows [y0, y0 + n) of the current state into / from a device buffer
 * of lbm_rows_bytes(ctx, n) bytes in that layout, queued on the context
 * stream (after its queued steps; no host wait).  LBM_EINVAL for rows outside
 * [0, ny), LBM_ESTATE before lbm_init_fields or while attached to a batch. */
int lbm_pack_rows(lbm_ctx* ctx, int y0, int n, void* dev_buf);
int lbm_unpack_rows(lbm_ctx* ctx, int y0, int n, const void* dev_buf);
/* Restricts the density sum behind rho_ave (Section 4.3) to the slab's own
 * rows [own_y0, own_y1) and takes the mean over global_nodes nodes (the
 * whole domain's count).  After each step the slabs' sums are to be added
 * into the ring slot the step published (lbm_mass_ring) before the next
 * step runs. */
int lbm_set_partition(lbm_ctx* ctx, int own_y0, int own_y1, long long global_nodes);
/* Device address of the context's three-slot density-sum ring (doubles):
 * step s publishes sum rho of its rows into slot s % 3 and reads slot
 * (s + 2) % 3 (the previous step's); lbm_init_fields sets slot 2 for step 0.
 * The caller may overwrite a slot in stream order between steps. */
int lbm_mass_ring(lbm_ctx* ctx, double** dev_ring);

/* Frees the context (synchronising first).  NULL is accepted. */
void lbm_destroy(lbm_ctx* ctx);

/* Human-readable text of the last error seen by this context (never NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Replaces the physical parameters and the boundary values of a context
 * between steps.  Section 4.2 relaxes a sessile droplet without evaporation
 * until it shows the prescribed contact angle and only then heats the wall:
 * run with frozen_thermal = 1 and the wall at the saturation temperature,
 * then call this with frozen_thermal = 0 and the heated wall.
 *  params: as for lbm_create; w_dot must be unchanged (the stored thermal
 *          deviations depend on it) and rho_ref / T_ref are ignored (the
 *          storage references set at initialisation stay).
 *  bc:     the flow kind of every edge must be unchanged (the geometry of the
 *          problem); thermal kinds, edge temperatures, the contact angle and
 *          the heater may change.
 * Takes effect for the next queued step.  LBM_EINVAL on a violated rule,
 * LBM_ESTATE while the context is attached to a batch. */
int lbm_reconfigure(lbm_ctx* ctx, const lbm_params* params, const lbm_bc* bc);

/* Contact angle of a sessile droplet on the south wall (Section 4.2).  The
 * interface is rho_mid = (rho_l + rho_g)/2; each horizontal or vertical
 * lattice link whose two densities lie on opposite sides of it gives one
 * point, linearly interpolated on the link; links touching rows below
 * skip_rows (the wetting ghost layer distorts the first rows) are left out.
 * A circle is fitted to the points by algebraic least squares and the angle
 * inside the liquid is taken where it meets the wall line y = -1/2 (halfway
 * bounce-back): cos(theta) = (-1/2 - y_c)/R.  The field must hold one droplet
 * that does not cross a periodic seam.  Sums are accumulated in double on
 * the device in a fixed order (the result does not vary between runs).
 * Synchronises.  LBM_EINVAL if the south edge is not a wall, rho_l <= rho_g,
 * skip_rows < 0 or fewer than 3 points (out->n_points is then still set). */
typedef struct {
    double theta_deg;        /* contact angle inside the liquid, degrees */
    double xc, yc, radius;   /* fitted circle, lattice units, node (0,0) at origin */
    double base_width;       /* chord of the circle on the wall line */
    double height;           /* apex height above the wall line */
    int n_points;            /* interface points in the fit */
} lbm_contact;
int lbm_contact_angle(lbm_ctx* ctx, double rho_l, double rho_g, int skip_rows, lbm_contact* out);

/* 4-connected regions of one phase of the current density field: nodes with
 * rho < threshold (below != 0, vapour) or rho > threshold (below == 0,
 * liquid), connected across the seams of periodic axes.  Each region's label
 * is the smallest node index y * nx + x it contains (unique, independent of
 * the order of work on the device).  A bubble has departed from the south
 * wall (Section 4.3) when its region no longer touches row 0; its equivalent
 * diameter is 2 sqrt(area / pi).
 *  labels:   host int array [ny][nx] receiving each node's label, -1 outside
 *            the phase; may be NULL.
 *  regions:  host array of max_regions entries, filled in increasing label
 *            order; may be NULL when max_regions is 0.
 *  n_regions: receives the number of regions; when it exceeds max_regions,
 *            the max_regions regions with the smallest labels are written.
 * Device scratch of 32 bytes per node is allocated on first use and kept
 * with the context.  Synchronises.  LBM_EINVAL on bad arguments, LBM_ECUDA if
 * the labelling reports that a capped loop ran out (it cannot by
 * construction; the cap guards against a defect). */
typedef struct {
    long long label;         /* smallest node index in the region */
    long long area;          /* nodes */
    long long sum_y;         /* sum of the nodes' row indices (centroid height) */
    int y_min, y_max;        /* row range */
    int touches_w, touches_e, touches_s, touches_n;   /* has a node on that edge */
} lbm_region;
int lbm_regions(lbm_ctx* ctx, double threshold, int below, int* labels, lbm_region* regions,
                int max_regions, int* n_regions);

/* ---- batched stepping of independent domains --------------------------- *
 * A batch advances every attached context by one coupled step per launch of
 * one persistent kernel that walks a shared work list of (domain, tile)
 * units, so hundreds of domains of uneven size share the GPU.  Attached
 * contexts must have the same precision and the same physical parameters
 * (everything in lbm_params except rho_ref / T_ref); sizes, boundaries and
 * edge temperatures may differ.  Each context's own stream is not used while
 * it is attached: the batch's stream is. */

/* stream: as in lbm_create. */
int lbm_batch_create(void* stream, lbm_batch** out);
/* Adds / removes a context.  A context belongs to at most one batch.
 * LBM_EINVAL on precision or parameter mismatch.  Neither call waits on the
 * host for queued work: attach makes the batch stream wait for the work
 * queued so far on the context's stream (its initialisation), detach makes
 * the context's stream wait for the batch steps queued so far, so what the
 * context does next on its own stream (readback, destroy) sees their result.
 * The batch's instance table and work list are rebuilt in stream order
 * (freed and allocated on the batch stream), so launches already queued
 * keep theirs. */
int lbm_batch_attach(lbm_batch* b, lbm_ctx* ctx);
int lbm_batch_detach(lbm_batch* b, lbm_ctx* ctx);
/* Queues, on the batch stream, a copy of every attached context's sticky
 * device error word (LBM error bits; 0 = none) into host_out[i], i in
 * attach order (the order the batch lists its members), for
 * lbm_batch_size(b) ints.  host_out must be page-locked (pinned) host memory
 * and is valid once the batch stream has passed this point (an event
 * recorded after the call).  Lets a scheduler check a chunk of steps for
 * errors without waiting for the chunks queued after it.  The paper has no
 * counterpart. */
int lbm_batch_errors_async(lbm_batch* b, int* host_out);
/* Number of attached contexts. */
int lbm_batch_size(const lbm_batch* b);
/* Queues n steps of every attached context on the batch stream. */
int lbm_batch_step(lbm_batch* b, int n);
/* Waits for the batch stream; returns the first sticky device error among
 * the attached contexts (and records it in that context). */
int lbm_batch_sync(lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);
/* Chooses the batch's tile (load path, threads, rows) by timing each
 * candidate for steps_per_trial steps on a shadow batch: scratch domains of
 * the members' sizes, precision, boundaries and parameters in a uniform
 * state, so the members' states are untouched (the shadow needs as much
 * device memory as the members, for the duration of the call).  The choice
 * is kept while members attach and detach (staging drops out while some
 * member cannot take it).  Without it a batch uses the lbm_create defaults
 * with 64-row segments.  lbm_batch_get_tile reports the tile in use. */
int lbm_batch_autotune(lbm_batch* b, int steps_per_trial);
int lbm_batch_get_tile(const lbm_batch* b, int* threads, int* rows, int* staged);

/* ---- launch configuration ------------------------------------------------ *
 * Tile of the fused step: a strip of (threads - 8) columns swept over a
 * segment of `rows` rows.  threads is 128, 192, 224 or 256; rows >= 1.
 * Without tuning, lbm_create takes the height that makes the units fill the
 * persistent grid in one wave.  The autotuner times load paths x thread
 * counts x heights (powers of two and the whole-wave heights) on a scratch
 * domain of the same size and precision, applies the fastest and caches the
 * choice per (precision, size). */
int lbm_set_tile(lbm_ctx* ctx, int threads, int rows);
int lbm_get_tile(const lbm_ctx* ctx, int* threads, int* rows);
int lbm_autotune(lbm_ctx* ctx, int steps_per_trial);

/* Load path of the fused FP32 / FP32_G16 step (no counterpart in the paper, which
 * prescribes no implementation).  on = 1: each row of f, g and P^{n-1} that a
 * tile needs is brought into shared memory by bulk asynchronous copies
 * (cp.async.bulk, completion tracked by an mbarrier) two rows ahead of its
 * use (three on the 128- and 192-thread tiles); on = 0: each thread loads its
 * own column a half row ahead into registers.  Both paths do the same
 * arithmetic in the same order: with LBM_FP32 the populations are equal bit
 * for bit; with LBM_FP32_G16 they agree to the FP16 rounding of a stored g
 * (the kernels are compiled separately, and a multiply-add contracted
 * differently can flip one such rounding).  Staging needs LBM_FP32 or
 * LBM_FP32_G16 and either open x edges or a periodic x axis with nx >= 32 a
 * multiple of 4 (LBM_FP32) or 8 (LBM_FP32_G16); lbm_create turns it on
 * (with a 224-thread tile) for wall-free domains wide enough for 216-column
 * strips, lbm_autotune times both paths.  Returns LBM_EINVAL when on = 1 is
 * not possible, LBM_ESTATE for a context in a batch.  A
 * staged launch that waits more than about a second for a row reports
 * LBM_ETIMEOUT (sticky) instead of hanging.  lbm_get_staging returns 0 or 1
 * (LBM_EINVAL for NULL).  A batch stages (224-thread tile) when every member
 * can and has no walls, and its members are wide enough as a whole. */
int lbm_set_staging(lbm_ctx* ctx, int on);
int lbm_get_staging(const lbm_ctx* ctx);

/* Test hook for the staged path's failure detection (no counterpart in the
 * paper).  on = 1: every CTA of the context's next staged launches also waits
 * on an mbarrier that nothing ever arms; that wait is bounded like the row
 * waits (about 2^31 clocks, roughly a second), runs out, and the launch
 * records LBM_ETIMEOUT in the sticky error word.  The row pipeline keeps its
 * own waits, so the step's results are unchanged and no copy is left in
 * flight; the GPU is never faulted.  No effect on the register-prefetch path
 * or on batches.  Returns LBM_EINVAL for NULL, LBM_ESTATE in a batch. */
int lbm_set_wait_probe(lbm_ctx* ctx, int on);

/* ---- diagnostics without any allocation -------------------------------- *
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory: a process whose GPU memory is owned by another
 * framework's pool, a loop that cannot afford cudaMalloc's implicit device
 * synchronisation, or a plugin that is handed device pointers and a stream
 * and nothing else.  It computes the same sums as lbm_diagnostics, but from
 * device field arrays the caller provides, and keeps its scratch (per-block
 * partial sums) in one fixed-size array inside the library (256 KB per GPU,
 * held from the first call until the process exits) instead of allocating.
 *
 *  rho, ux, uy, T: device arrays of n doubles each (any node order).
 *  out7: device array receiving 7 doubles: sum rho, sum rho cv T, liquid mass
 *        and liquid node count above (rho_l + rho_g)/2, the smooth liquid
 *        area sum clamp((rho - rho_g)/(rho_l - rho_g), 0, 1), max |u| and the
 *        number of nodes with a non-finite value.
 *  stream: cudaStream_t as void* (NULL: the legacy default stream); the call
 *        is asynchronous on it.
 * Returns LBM_EINVAL for NULL pointers, n < 0 or rho_l <= rho_g, LBM_ETOOBIG
 * for n > LBM_NOALLOC_MAX_NODES (the capacity of the fixed scratch), and
 * LBM_ECUDA if the CUDA runtime refuses a call.  It never calls cudaMalloc or
 * cudaFree.  The first call on each device looks up the device address of the
 * scratch array for that device (with that device current); make that first
 * call before any stream capture.  All calls on a device share the array:
 * calls whose kernels may overlap on the GPU (unordered streams) race, so
 * keep them on one stream. */
#define LBM_NOALLOC_MAX_NODES 33554432LL
int lbm_diag_reduce_noalloc(const double* rho, const double* ux, const double* uy,
                            const double* T, long long n, double cv, double rho_l,
                            double rho_g, double* out7, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
