/*
 * lbm.h -- C ABI of the two-component D2Q9 lattice-Boltzmann library for
 * GB300 (sm_103a).
 *
 * The library advances two immiscible species ("o", oil, index 0 and "w",
 * water, index 1) on a 2-D lattice with the method of Otomo et al.,
 * "Simulation of residual oil displacement in a sinusoidal channel with the
 * lattice Boltzmann method", Section 2:
 *   - BGK relaxation at the per-node mixture relaxation time
 *     tau_mix = nu_mix/T0 + 1/2, nu_mix = (rho^o nu^o + rho^w nu^w)/rho,
 *     nu^a = T0 (tau^a - 1/2), T0 = 1/3 (Eq. LBM_BGK and the two relations
 *     after it);
 *   - the third-order equilibrium of Eq. (feq);
 *   - the inter-component force of Eq. (comp_interaction),
 *     F^a(x) = G rho^a(x) sum_i w_i c_i rho^b(x + c_i), with the wall
 *     potentials rho_s^a replacing the density of solid neighbours;
 *   - the force carried by the equilibrium velocity shift of
 *     Eq. (collision_term), u_mix + F^a/rho^a, with u_mix the mixture
 *     velocity; the non-equilibrium part is f - f^eq(rho^a, u_mix);
 *   - the homogeneous body-force acceleration g of Section 3.4;
 *   - halfway bounce-back at solid nodes of a wall mask.
 *
 * Conventions shared by every call:
 *   - Host arrays are owned by the caller and are read or written
 *     synchronously before the call returns.
 *   - Device memory is owned by the library, or carved from a caller-owned
 *     device arena (lbm_params.workspace) that must outlive the handle.
 *   - Every call returns an lbm_status; none aborts the process.  The text of
 *     the last error of a handle is available from lbm_last_error(h); errors
 *     of lbm_create (no handle yet) are kept per thread and read with
 *     lbm_last_error(NULL).
 *   - Grids are [ny][nx] row-major with x fastest.  A node mask byte is 0 for
 *     fluid and non-zero for solid.  A direction that is not periodic must
 *     have solid nodes on both of its boundary lines (else LBM_EINVAL).
 */
#ifndef GB300_LBM_H
#define GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_t lbm_t; /* opaque handle */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,    /* bad argument, size, mask or parameter */
    LBM_ENOMEM = -2,    /* device allocation failed or arena too small */
    LBM_ECUDA = -3,     /* a CUDA call failed; see lbm_last_error */
    LBM_EUNSTABLE = -4, /* a fluid node reached a NaN or negative density */
    LBM_ETIMEOUT = -5   /* a bounded device wait gave up */
} lbm_status;

/* Storage of the populations.  Arithmetic is FP64 for LBM_FP64 and FP32
 * otherwise.  The 16-bit formats store s_i = f_i - w_i rhohat^a(x), the
 * population minus the rest equilibrium at the writing node's own density
 * rounded to the 16-bit format, rhohat^a(x), which is kept in two extra
 * planes; a reader adds back w_i rhohat^a of the source node, so only the
 * small non-equilibrium part is rounded to 16 bits.
 * LBM_FP32C stores FP32 like LBM_FP32 and compensates the two arithmetic
 * stages whose FP32 rounding dominates the error against exact arithmetic:
 * the density sums (rho carried as an unevaluated pair hi + lo through
 * Fast2Sum) and the composition of each stored population from w_i rho
 * (an FMA TwoProduct, with the FP32 weights' own rounding folded in) and the
 * equilibrium and non-equilibrium parts, so that each stored population is
 * rounded once.  Everything else stays plain FP32.  The cost and the
 * accuracy of both FP32 forms are measured in this library's tests and
 * benchmark. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16S = 2, LBM_BF16S = 3, LBM_FP32C = 4 } lbm_precision;

typedef struct {
    int32_t nx, ny;                 /* lattice size, both >= 1 */
    int32_t periodic_x, periodic_y; /* 1 = periodic in that direction */
    double tau[2];                  /* tau^o, tau^w, each > 1/2 (Section 2) */
    double G;                       /* Eq. (comp_interaction); repulsive when G < 0 */
    double rho_wall[2];             /* rho_s^o, rho_s^w (end of Section 2) */
    double g[2];                    /* body-force acceleration (x, y) (Section 3.4) */
    int32_t precision;              /* lbm_precision */
    int32_t eq_order;               /* 3 = Eq. (feq) as printed, 2 = without cubic terms */
    int32_t variant;                /* step kernel: 0 = autotuned, 1 = simple (register pull),
                                       2 = staged (TMA row pipeline, CTA barrier per row),
                                       3 = pipelined (TMA rows, warps march independently),
                                       4 = private (each warp stages its own row windows,
                                       densities exchanged by shuffles, no CTA barrier);
                                       5 = persistent (many steps per cooperative launch, a
                                       grid-wide barrier between steps; for small grids:
                                       with 0 the library times it, with tiles of 1, 2, 4 and
                                       8 rows, against the graph path on the first lbm_step
                                       of 160 steps or more when the grid has at most 2^21
                                       fluid nodes and keeps the fastest);
                                       results agree to rounding */
    int32_t collision;              /* non-equilibrium part f' of Eq. (LBM_BGK): 0 = f - f^eq
                                       (plain BGK); 1 = regularised, Eq. (Regualize): the
                                       second-order Hermite projection w_i Q_i : Pi / (2 T0^2)
                                       of the non-equilibrium momentum flux Pi */
    void *cuda_stream;              /* cudaStream_t for all work, or NULL = legacy default */
    void *workspace;                /* optional device arena (>= lbm_workspace_size bytes,
                                       256-byte aligned), or NULL: the library allocates */
    size_t workspace_bytes;
} lbm_params;

/* Observables of the most recent step (Section 3.4 tracks the slug by its
 * centre of oil mass). */
typedef struct {
    double mass[2];   /* sum over fluid nodes of rho^o, rho^w */
    double oil_mom_x; /* sum over fluid nodes of j^o_x + F^o_x / 2 */
    double oil_disp_x;/* running sum over all steps of oil_mom_x / mass[0]: the
                         unwrapped x displacement of the oil centre of mass */
    double max_u;     /* max over fluid nodes of |u|, u = (sum_a j^a + F^a/2)/rho */
    int64_t step;     /* steps taken since lbm_create or the last lbm_load */
    int32_t nan_flag; /* 1 once any fluid node had a NaN or negative density */
    int32_t timeout_flag; /* 1 once a bounded device wait gave up (that step's data invalid) */
} lbm_obs;

/* Bytes of device memory a handle with parameters p needs (for the
 * workspace arena).  Returns LBM_EINVAL on bad sizes or precision. */
int lbm_workspace_size(const lbm_params *p, size_t *bytes);

/* Create a simulation.
 *   mask     host uint8 [ny][nx], 1 = solid (required)
 *   rho_init host double [2][ny][nx] initial densities of species o then w
 *            at fluid nodes (values at solid nodes are ignored); the stored
 *            state starts at the rest equilibrium f*_i = w_i rho_init
 *   p        parameters; copied, so the caller may free it afterwards
 *   out      receives the handle
 * Errors: LBM_EINVAL (NULL pointer, size, tau <= 1/2, precision, eq_order,
 * open boundary without solid lines, a fluid node whose initial densities
 * are not finite, negative, or sum to 0: checked on the device after the
 * upload), LBM_ENOMEM, LBM_ECUDA. */
int lbm_create(const uint8_t *mask, const double *rho_init, const lbm_params *p, lbm_t **out);

/* Advance nsteps >= 0 time steps (Eq. basic_LBM_eq with the collision of
 * Eq. LBM_BGK, its non-equilibrium part as lbm_params.collision says),
 * asynchronously on the handle's stream.  Returns the launch status:
 * LBM_EINVAL for a NULL handle or nsteps < 0, LBM_ECUDA when a launch (or
 * the capture of the 32-step graph) fails; instability and a bounded wait
 * that gave up are reported by lbm_observables. */
int lbm_step(lbm_t *h, int64_t nsteps);

/* Synchronise the stream and copy the observables of the latest step
 * (Section 3.4 tracks the slug by its centre of oil mass; the sums are the
 * lbm_obs fields above).  Returns LBM_EINVAL for a NULL argument,
 * LBM_ETIMEOUT once timeout_flag is set, else LBM_EUNSTABLE once nan_flag is
 * set (*out is filled in both cases), LBM_ECUDA when the copy fails. */
int lbm_observables(lbm_t *h, lbm_obs *out);

/* Macroscopic fields of the current state (the state a next step would pull
 * and collide), copied to host FP64 arrays; any pointer may be NULL:
 *   rho [2][ny][nx]  species densities (rho_s^a at solid nodes)
 *   u   [2][ny][nx]  mixture velocity planes u_x then u_y,
 *                    u = (j^o + j^w + (F^o + F^w)/2)/(rho^o + rho^w), 0 at solid
 *   p   [ny][nx]     pressure T0 (rho^o + rho^w) - G T0 rho^o rho^w, 0 at solid
 * The arrays are written by device-to-host copies (at full speed when they
 * are in pinned memory); the call returns when they are complete. */
int lbm_get_fields(lbm_t *h, double *rho, double *u, double *p);

/* Change the body-force acceleration (Section 3.4's homogeneous driving
 * force) used by the following steps; synchronises the stream.  LBM_EINVAL
 * for a NULL handle or a value that is not finite. */
int lbm_set_body_force(lbm_t *h, double gx, double gy);

/* Copy the stored post-collision populations f*_i^a (Eq. basic_LBM_eq) to /
 * from a host FP64 array f[2][9][ny][nx] (species, direction, y, x;
 * directions c_0 = (0,0), c_1..c_4 = (1,0),(0,1),(-1,0),(0,-1),
 * c_5..c_8 = (1,1),(-1,1),(-1,-1),(1,-1)), synchronously.  lbm_save writes 0
 * at solid nodes; lbm_load ignores them and stores each value in the
 * handle's format (rounded for FP32 and the 16-bit forms).  lbm_load also
 * resets the observables (step count, displacement, NaN flag).  LBM_EINVAL
 * for a NULL argument, LBM_ECUDA when a copy fails. */
int lbm_save(lbm_t *h, double *f);
int lbm_load(lbm_t *h, const double *f);

/* Launch configuration the autotuner chose for the step kernel:
 * info[0] = variant (1 simple, 2 staged, 3 pipelined, 4 private, 5
 * persistent: then info[2] = rows per tile, info[3] = CTAs of the
 * cooperative launch); info[1] =
 * rows issued ahead of the three a march reads (1 or 2, variants 2..4);
 * info[2] = rows per CTA strip (variant 1)
 * or columns per CTA (2..4); info[3] = strips per column block (2..4);
 * info[4] = 1 when the staged kernel's strips sit at the same absolute rows
 * in every column block, 0 when each block's fluid rows are split into
 * equal strips (and for the other variants).  Not part of the paper's
 * method: a report of this library's tuning. */
int lbm_kernel_info(const lbm_t *h, int32_t info[5]);

/* Self-test of the device-side wait limit.  Every wait of the step kernels
 * (for a row copy to land, for a ring slot) is bounded: after about 0.5 s
 * (measured on GB300) the kernel gives up, marks the step (LBM_ETIMEOUT from lbm_observables)
 * and returns, so a lost copy cannot hang the GPU.  This call runs that same
 * bounded wait on a barrier that nothing ever completes, on cuda_stream
 * (NULL = legacy default), and returns LBM_ETIMEOUT when the wait gave up as
 * it must (any other status is a failure); *seconds (may be NULL) receives
 * how long the wait took.  The CUDA context stays usable afterwards.
 * Allocates 4 bytes of device memory for the duration of the call.  Not part
 * of the paper's method: a check of this library's failure handling. */
int lbm_wait_selftest(void *cuda_stream, double *seconds);

/* One FP32 time step that allocates nothing, for callers that cannot call
 * cudaMalloc: code running while a CUDA graph is being captured, real-time
 * loops that must not allocate, plug-ins whose device memory belongs to a
 * host framework's allocator.  The paper has no counterpart; this is a
 * calling convention of this library.
 *   mask  device uint8 [ny][nx], 1 = solid (same rules as lbm_create)
 *   f_in  device float [2][9][ny][nx] stored populations (the lbm_save layout,
 *         dense, no padding)
 *   f_out device float, same layout; receives the next stored state at fluid
 *         nodes (solid nodes are not written)
 *   obs   device lbm_obs receiving this step's observables (step = 1,
 *         oil_disp_x = this step's displacement), or NULL
 *   p     host parameters: precision must be LBM_FP32; nx * ny <= 2097152
 *         (any shape within that, e.g. 1 x 2097152); tau, G, g and rho_wall
 *         are checked as in lbm_create; p->cuda_stream is the stream of all
 *         work; variant and workspace fields are ignored
 * Pulls and force neighbours always wrap in both directions: periodic_x and
 * periodic_y are ignored, and the mask cannot be checked on the host (it is
 * device memory).  For a direction meant to be closed, keep its first and
 * last line solid, as lbm_create requires; a fluid node on such a line
 * would be stepped as if the lattice were periodic there.
 * The scratch is one static device array of 4 MiB + 1 KiB that every GPU
 * which loads this library holds until the process exits.  The first call on
 * a device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.
 * Every call shares the array: calls that may overlap on the GPU (on
 * different streams, or from several threads) race; serialise them.  The
 * call is asynchronous and returns LBM_EINVAL for sizes beyond the limit, a
 * precision other than LBM_FP32 or NULL pointers. */
int lbm_step_noalloc(const uint8_t *mask, const float *f_in, float *f_out, lbm_obs *obs,
                     const lbm_params *p);

/* ---------------------------------------------------------------------------
 * The same step on the paper's own lattice, D3Q19 (Section 2)
 *
 * Nineteen velocities in three dimensions: c_0 = 0; c_1..c_6 the face
 * neighbours +x, -x, +y, -y, +z, -z (weight 1/18); c_7..c_18 the edge
 * neighbours (+x+y), (-x-y), (+x-y), (-x+y), (+x+z), (-x-z), (+x-z), (-x+z),
 * (+y+z), (-y-z), (+y-z), (-y+z) (weight 1/36); rest 1/3; T0 = 1/3.  The
 * method is the one of lbm_create (interaction and wall force, body force,
 * mixture relaxation, force through the equilibrium shift, BGK or
 * regularised non-equilibrium part, halfway bounce-back).  Grids are
 * [nz][ny][nx] with x fastest; populations f[2][19][nz][ny][nx].  FP64 and
 * FP32 storage.  Two launches per step: a density pass and a pull
 * collide-stream pass that reads the neighbour densities of the force from
 * the density field.  The paper's sinusoidal tube (Section 3.4, circular
 * cross sections) is a mask of this kind.
 * ------------------------------------------------------------------------- */
typedef struct lbm3d_t lbm3d_t; /* opaque */

typedef struct {
    int32_t nx, ny, nz;           /* lattice size, each in [1, 2^21], 38 nx ny nz < 2^40 */
    int32_t periodic[3];          /* 1 = periodic along x, y, z (else solid boundary planes) */
    double tau[2];                /* tau^o, tau^w (> 1/2) */
    double G;                     /* Eq. (comp_interaction) */
    double rho_wall[2];           /* rho_s^o, rho_s^w */
    double g[3];                  /* body-force acceleration */
    int32_t precision;            /* LBM_FP64 or LBM_FP32 */
    int32_t eq_order;             /* 3 = Eq. (feq) as printed, 2 = without cubic terms */
    int32_t collision;            /* 0 BGK, 1 regularised (Eq. Regualize) */
    void *cuda_stream;            /* stream of all work, or NULL */
} lbm3d_params;

/* Create from a host mask [nz][ny][nx] (1 = solid) and host initial
 * densities [2][nz][ny][nx] (the state starts at f*_i = w_i rho_init).
 * Errors: LBM_EINVAL (sizes, parameters: tau > 1/2 and finite, G, g and
 * rho_wall finite, precision, eq_order, collision; a non-periodic direction
 * whose boundary planes hold fluid; densities at fluid nodes not finite,
 * negative or both zero: all checked on the host before any device work),
 * LBM_ENOMEM, LBM_ECUDA. */
int lbm3d_create(const uint8_t *mask, const double *rho_init, const lbm3d_params *p, lbm3d_t **out);
/* Advance nsteps >= 0 steps (asynchronous on the handle's stream).
 * LBM_EINVAL for a NULL handle or nsteps < 0, LBM_ECUDA when a launch fails. */
int lbm3d_step(lbm3d_t *h, int64_t nsteps);
/* Observables of the latest step (as lbm_observables; oil_mom_x along x);
 * synchronises the stream.  LBM_EUNSTABLE once nan_flag is set (*out
 * filled).  The two D3Q19 passes hold no device-side wait, so timeout_flag
 * stays 0. */
int lbm3d_observables(lbm3d_t *h, lbm_obs *out);
/* Densities rho [2][nz][ny][nx] and mixture velocity u [3][nz][ny][nx]
 * (with half the force) of the current state; either may be NULL.
 * Allocates a temporary device buffer of 40 bytes per node (LBM_ECUDA when
 * that fails) and returns when the host arrays are written. */
int lbm3d_get_fields(lbm3d_t *h, double *rho, double *u);
/* Stored populations to / from a host array f[2][19][nz][ny][nx]
 * (synchronous; 0 at solid nodes on save, ignored there on load; load
 * resets the observables).  LBM_EINVAL for a NULL argument. */
int lbm3d_save(lbm3d_t *h, double *f);
int lbm3d_load(lbm3d_t *h, const double *f);
/* Free the handle and its device memory (after its stream's work); NULL is
 * ignored. */
void lbm3d_destroy(lbm3d_t *h);
/* Text of the last error of h, or, when h is NULL, of the calling thread's
 * last 3-D call that failed without a handle (lbm3d_create, or a call given
 * NULL). */
const char *lbm3d_last_error(const lbm3d_t *h);

/* Free the handle and the device memory it owns.  NULL is ignored. */
void lbm_destroy(lbm_t *h);

/* Text of the last error of h, or of the calling thread's last lbm_create
 * when h is NULL.  Valid until the next call on the same handle / thread. */
const char *lbm_last_error(const lbm_t *h);

/* ---------------------------------------------------------------------------
 * Batches of independent channels and the critical body force (Section 3.4)
 *
 * The paper's question: the smallest homogeneous body force g at which a
 * static oil slug in a sinusoidal channel starts to move (the critical Bond
 * number Bo = rho g L D / sigma, Eq. Bo_number).  The paper ramps g in small
 * increments (Section 3.4); here each instance is bisected on g instead:
 * every probe restarts from the state equilibrated at g = 0, runs t_obs
 * steps at the probe value, and calls the slug moving when its oil centre of
 * mass travelled more than the instance's disp_threshold.
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch_t lbm_batch_t; /* opaque */

typedef struct {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;
    double tau[2];          /* tau^o, tau^w (> 1/2) */
    double G;               /* Eq. (comp_interaction) */
    double rho_wall[2];     /* rho_s^o, rho_s^w */
    double g[2];            /* body force used by lbm_batch_step */
    const uint8_t *mask;    /* host [ny][nx], 1 = solid (same rules as lbm_create) */
    const double *rho_init; /* host [2][ny][nx] initial densities */
    double disp_threshold;  /* oil displacement over one probe window that means "moving" */
    int32_t collision;      /* as lbm_params.collision */
} lbm_instance;

/* Create n instances of uneven sizes that step together (one launch per step
 * over all of them).  The library copies the instance data; the host arrays
 * may be freed after the call.  Errors as lbm_create (per-instance text in
 * lbm_batch_last_error(NULL)).  FP32 and the 16-bit formats step with the
 * staged (TMA) march over tiles of 128 columns x R rows holding fluid; R is
 * timed among 8, 16, 32, 48, 64 and the size that fills four waves of
 * resident CTAs (a few steps from the initial state into the second buffer,
 * which leave the state and the observables as created), or pinned by the
 * environment variable GB300LBM_BATCH_ROWS; FP64 steps with the
 * register-pull march. */
int lbm_batch_create(const lbm_instance *inst, int32_t n, int32_t precision, int32_t eq_order,
                     void *cuda_stream, lbm_batch_t **out);

/* Advance every active instance by nsteps >= 0 (asynchronous; runs of 16
 * steps replay a captured CUDA graph).  LBM_EINVAL for a NULL batch or
 * nsteps < 0, LBM_ECUDA when a launch fails. */
int lbm_batch_step(lbm_batch_t *b, int64_t nsteps);

/* Observables of every instance (out[n]); LBM_EUNSTABLE if any NaN flag,
 * else LBM_ETIMEOUT if a bounded device wait gave up in some step. */
int lbm_batch_observables(lbm_batch_t *b, lbm_obs *out);

/* Step kernel of the batch: info[0] = 2 staged (TMA) march, 1 register-pull
 * march; info[1] = rows per strip of the staged tiles (0 otherwise);
 * info[2] = CTAs per step.  Not part of the paper's method: a report of this
 * library's tiling. */
int lbm_batch_kernel_info(const lbm_batch_t *b, int32_t info[3]);

/* Set the x body force (Section 3.4) of every instance from the host
 * array gx[n]; synchronises the stream.  LBM_EINVAL for a NULL argument or
 * a value that is not finite. */
int lbm_batch_set_body_force(lbm_batch_t *b, const double *gx);

/* Stored populations of instance i as lbm_save does for a single grid
 * (f[2][9][ny_i][nx_i], synchronous).  LBM_EINVAL for a NULL argument or
 * i outside [0, n). */
int lbm_batch_save(lbm_batch_t *b, int32_t i, double *f);

typedef struct {
    double rel_bracket;    /* stop when g_hi - g_lo <= rel_bracket * g_hi (e.g. 0.02) */
    int64_t t_eq;          /* steps at g = 0 before the first probe */
    int64_t t_obs;         /* steps per probe */
    int32_t max_probes;    /* per instance, bracket checks included */
    int32_t check_bracket; /* 1: first check that g_hi moves and g_lo does not,
                              doubling g_hi / halving g_lo on failure; 0: trust the bracket */
    double timeout_s;      /* host wall-clock limit (<= 0: none) */
} lbm_bisect_opts;

typedef struct {
    double g_lo, g_hi;     /* final bracket: static at g_lo, moving at g_hi */
    int32_t probes;        /* probe windows this instance took part in */
    int32_t status;        /* 0 converged, 1 max_probes reached, 2 unstable, 3 timeout
                              (timeout_s ran out, or a bounded device wait gave up) */
} lbm_crit_result;

/* Bisect every instance of b on its x body force, starting from the brackets
 * [g_lo[i], g_hi[i]]; all instances probe in lockstep, finished ones drop
 * out of the launches.  Classification and bracket updates run on the
 * device in FP64.  LBM_EINVAL unless 0 < g_lo[i] < g_hi[i] < infinity for
 * every instance, rel_bracket > 0, t_obs >= 1, t_eq >= 0 and max_probes >= 1.
 * Returns LBM_ETIMEOUT (results filled, status 3) when timeout_s ran out. */
int lbm_critical_pressure_batch(lbm_batch_t *b, const double *g_lo, const double *g_hi,
                                const lbm_bisect_opts *o, lbm_crit_result *out);

/* Free the batch and its device memory (after its stream's work); NULL is
 * ignored. */
void lbm_batch_destroy(lbm_batch_t *b);
/* Text of the last error of b, or, when b is NULL, of the calling thread's
 * last batch call that failed without a batch (lbm_batch_create, or a call
 * given NULL). */
const char *lbm_batch_last_error(const lbm_batch_t *b);

/* ---------------------------------------------------------------------------
 * Surrogate of the critical body force (not in the paper)
 *
 * A small network that maps a channel description to a predicted log g_crit
 * with an uncertainty; it only seeds the brackets of
 * lbm_critical_pressure_batch, which alone decides.  Network 5 -> 128 ->
 * 128 -> 128 -> 2, SiLU hidden units, outputs (mu, s): mu the predicted
 * log g_crit, s the log predicted variance; per-sample loss
 * 0.5 (exp(-s) (y - mu)^2 + s).  34050 FP32 parameters, flat order
 * W1 [128x5], b1 [128], W2 [128x128], b2, W3 [128x128], b3, W4 [2x128], b4 [2].
 * Host arrays in, host arrays out; the network lives on the device.
 * ------------------------------------------------------------------------- */
typedef struct lbm_mlp_t lbm_mlp_t;

/* params: 34050 floats, or NULL for a seeded uniform(+-1/sqrt(fan_in)) init. */
int lbm_mlp_create(const float *params, uint64_t seed, void *cuda_stream, lbm_mlp_t **out);
/* Copy the parameters out (out_params may be NULL) and/or in (in_params may
 * be NULL; loading resets the Adam moments). */
int lbm_mlp_params(lbm_mlp_t *h, float *out_params, const float *in_params);
/* out[B][2] = network(x[B][5]); 1 <= B <= 65536. */
int lbm_mlp_forward(lbm_mlp_t *h, const float *x, int32_t B, float *out);
/* Mean loss over the batch and its gradient (grad[34050], may be NULL). */
int lbm_mlp_loss_grad(lbm_mlp_t *h, const float *x, const float *y, int32_t B, float *loss, float *grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient. */
int lbm_mlp_adam(lbm_mlp_t *h, float lr);
/* epochs of minibatch Adam over (x[n][5], y[n]), shuffled with seed;
 * *last_loss = loss of the last minibatch. */
int lbm_mlp_train(lbm_mlp_t *h, const float *x, const float *y, int32_t n, int32_t epochs, int32_t batch,
                  float lr, uint64_t seed, float *last_loss);
void lbm_mlp_destroy(lbm_mlp_t *h);
const char *lbm_mlp_last_error(void);

/* ---------------------------------------------------------------------------
 * The paper's question from channel descriptions (Sections 3.1, 3.3, 3.4)
 *
 * Section 3.4 states the problem as: a periodic sinusoidal channel holds an
 * oil slug in water; for the channel's geometry, the slug's length, the
 * wall's wettability (a contact angle) and the two viscosities, find the
 * homogeneous body force g at which the static slug starts to move, and
 * report it as a Bond number Bo = rho g L D / sigma (Eq. Bo_number).  The
 * calls below take exactly that description and do every set-up step in the
 * library.  Readings fixed here (the paper leaves them open): planar 2-D
 * channel, fluid iff |y - y_c| <= h(x) = h0 - A cos(2 pi x / lambda) with
 * h0 = 0.1875 lambda, n_periods periods, height 2 ceil(h0 + A) + 2, n_slugs
 * identical slugs on equally spaced necks (one slug: the neck at
 * x = lambda floor(n_periods / 2)) with tanh ends of width 2 (densities
 * 1.0 / 0.03); G = -1.79; tau^w = 1 and
 * tau^o = max(3 r nu^w + 1/2, 0.75) for the viscosity ratio r = nu^o / nu^w;
 * "moving" = the oil centre of mass travels more than lambda / 2 in one
 * probe window; L = nx (the periodic length), D = h0 - A (the neck
 * half-width).  Host arrays in and out; errors of these calls are read with
 * lbm_channel_last_error().
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t lambda;               /* wavelength in nodes, 8 .. 65536 */
    double amp_ratio;             /* A / h0, in [0, 0.95] */
    double slug_len_over_lambda;  /* slug length / lambda, in (0, n_periods - 1] */
    double theta_deg;             /* contact angle through water, in (0, 180) degrees */
    double visc_ratio;            /* nu^o / nu^w, > 0 */
    int32_t n_periods;            /* periods along x, 2 .. 64 (0 = 4) */
    int32_t n_slugs;              /* identical slugs (0 = 1), dividing n_periods; slug k is centred on
                                     the neck at x = lambda (n_periods / (2 n_slugs) + k n_periods / n_slugs);
                                     each slug at most n_periods / n_slugs - 1/4 wavelengths long (one
                                     slug: n_periods - 1) */
} lbm_channel_spec;

/* Lattice size of a channel: nx = lambda n_periods, ny = 2 ceil(h0 + A) + 2.
 * LBM_EINVAL for a spec out of range. */
int lbm_channel_shape(const lbm_channel_spec *s, int32_t *nx, int32_t *ny);

/* Wall mask (host uint8 [ny][nx], 1 = solid) and initial densities (host
 * double [2][ny][nx]) of a channel with its slug; either pointer may be NULL.
 * No GPU work. */
int lbm_channel_geometry(const lbm_channel_spec *s, uint8_t *mask, double *rho_init);

/* Section 3.3 on the GPU: the contact angle (degrees, through water) of a
 * slug between flat plates H = 32 apart (192 columns, periodic in x, oil
 * over the middle half, tau = 1, G = -1.79), after `steps` steps, for each
 * signed wall potential r[i] (r > 0: rho_s^w = r, r < 0: rho_s^o = -r;
 * |r| <= 2).  Interface points where the oil fraction crosses 1/2 on every
 * row at least 3 rows from a wall, Pratt's algebraic circle fit,
 * Eq. (contact_angle); theta[i] is the mean of the slug's two ends.  All n
 * slugs run as one batch in `precision`, on cuda_stream (NULL = legacy
 * default). */
int lbm_wetting_calibrate(const double *r, int32_t n, int64_t steps, int32_t precision, void *cuda_stream,
                          double *theta);

/* Section 3.1 on the GPU: surface tension of the model (G = -1.79, tau = 1)
 * from the Laplace law over four static droplets (R = 12, 16, 20, 24 in a
 * 128 x 128 periodic box, `steps` steps): radius from where rho^o crosses
 * its mid value along the central row and column, pressure jump between
 * the centre and the far corner from p = T0 rho - G T0 rho^o rho^w, least
 * squares dp = sigma / R + c.  *rho_bulk = rho^o + rho^w in the middle of
 * a phase of a flat interface (two bands in a periodic 128 x 4 strip, run
 * in the same batch): the bulk total density at zero curvature. */
int lbm_surface_tension(int64_t steps, int32_t precision, void *cuda_stream, double *sigma, double *rho_bulk);

/* Section 3.4, planar form (host, FP64): rho g_crit L / sigma of a slug of
 * oil area `area` in a channel h(x) = h0 - amp cos(2 pi x / lam), resting
 * with its rear contact line near x_rest, contact angle theta_deg through
 * water.  Menisci are arcs centred on the axis meeting the wall (inclined
 * by atan h'(x)) at theta; at rest rho g L equals sigma times the front
 * curvature minus the rear one; the front follows the rear by conservation
 * of the oil area (the channel between the contact chords plus the circular
 * segments beyond them); loaded quasi-statically the slug climbs each
 * rising branch of that balance and jumps ahead past each local maximum,
 * and it counts as moving at the first jump longer than lam / 2.  0 when
 * the channel offers no capillary resistance. */
int lbm_planar_critical_balance(double theta_deg, double area, double h0, double amp, double lam, double x_rest,
                                double *balance);

/* The same balance with contact-angle hysteresis: the front meniscus (oil
 * advancing, water receding) meets the wall at theta_front_deg, the rear one
 * (water advancing) at theta_rear_deg, both through water; equal angles give
 * lbm_planar_critical_balance.  A receding water angle below the advancing
 * one raises the critical force (the Section 3.4 analysis with
 * Delta theta != 0). */
int lbm_planar_critical_balance_hysteresis(double theta_front_deg, double theta_rear_deg, double area, double h0,
                                           double amp, double lam, double x_rest, double *balance);

/* Contact angles of the two menisci of a slug in the planar sinusoidal
 * channel h(x) = h0 - amp cos(2 pi x / lam) about y_c = (ny - 1) / 2, from
 * host densities rho [2][ny][nx] (host, FP64).  For each meniscus: the
 * oil-fraction crossings of 1/2 on every fluid row at least two nodes from
 * the wall, Pratt's circle through them, its intersection with the wall,
 * and the angle there between the wall and the interface, through water.
 * out[6] = {theta_rear, theta_front (degrees), x_rear, x_front (contact
 * positions), R_rear, R_front (radii)}.  The slug must lie inside the
 * period on the centre row. */
int lbm_meniscus_angles(const double *rho, int32_t nx, int32_t ny, double h0, double amp, double lam, double *out);

/* Contact angle (degrees, through water) of one end of a slug between flat
 * plates with fluid rows y_lo..y_hi, from host densities rho [2][ny][nx]
 * (host, FP64): the measurement inside lbm_wetting_calibrate.  right = 1:
 * the slug's right end, 0: its left end.  LBM_EINVAL when fewer than three
 * rows show an interface. */
int lbm_contact_angle(const double *rho, int32_t nx, int32_t ny, int32_t y_lo, int32_t y_hi, int32_t right,
                      double *theta);

/* Oil area of a slug (the planar analogue of the slug volume of Section
 * 3.4) from host densities rho [2][ny][nx] and the mask [ny][nx] (1 =
 * solid), both host arrays the caller owns.  out[0]: fluid nodes whose oil
 * fraction rho^o / (rho^o + rho^w) exceeds 1/2.  out[1]: the paper's volume
 * detection, in which the slug splits into a bulk region, summed whole, and
 * interface regions, summed only where the oil density exceeds 90 % of the
 * total: a column whose fluid nodes are all oil-rich (fraction above 1/2)
 * is bulk and counts every fluid node; a column that an interface crosses
 * (some fluid nodes above 1/2, some not) counts the nodes above 9/10.
 * LBM_EINVAL for NULL pointers or nx, ny < 1. */
int lbm_slug_area(const double *rho, const uint8_t *mask, int32_t nx, int32_t ny, double *out);

/* Wall potentials (rho_s^o, rho_s^w) whose calibrated contact angle is
 * theta_deg, from a table r[n] (ascending) -> theta[n] (descending): linear
 * interpolation of r in theta, clipped to the table's range, then r > 0 ->
 * rho_s^w = r, r < 0 -> rho_s^o = -r (host). */
int lbm_wall_potentials(const double *r, const double *theta, int32_t n, double theta_deg, double *rho_wall);

typedef struct {
    double rel_bracket;          /* stop at (g_hi - g_lo) <= rel_bracket g_hi (<= 0: 0.02) */
    int64_t t_eq, t_obs;         /* steps at g = 0 before the probes; steps per probe (>= 1) */
    int32_t max_probes;          /* per channel, bracket checks included (<= 0: 24) */
    int32_t precision;           /* storage of the channels' populations (lbm_precision) */
    int32_t collision;           /* as lbm_params.collision (1, regularised, keeps low tau stable) */
    int32_t use_surrogate;       /* 1: start from the surrogate's bracket */
    lbm_mlp_t *surrogate;        /* the network (use_surrogate = 1) */
    float feature_mean[5];       /* feature normalisation the network was trained with: */
    float feature_std[5];        /*   x = (features - mean) / std (std 0 taken as 1) */
    double k_sigma;              /* surrogate bracket exp(mu -+ k_sigma sigma) (<= 0: 2), at least 5 % wide */
    double bracket_lo, bracket_hi; /* otherwise: these factors of the planar balance's force (<= 0: 0.5, 2) */
    const double *calib_r;       /* calibration table (ascending r, descending theta), or */
    const double *calib_theta;   /*   calib_n = 0: the library runs lbm_wetting_calibrate */
    int32_t calib_n;             /*   over 13 potentials in [-0.6, 0.6] (20 000 FP32 steps, cached) */
    double sigma, rho_bulk;      /* of the Bond number; <= 0: lbm_surface_tension (6000 FP32 steps, cached) */
    double timeout_s;            /* host wall-clock limit of the bisection (<= 0: none) */
    void *cuda_stream;           /* stream of all GPU work, or NULL */
} lbm_channel_opts;

typedef struct {
    double g_lo, g_hi;           /* final bracket: static at g_lo, moving at g_hi */
    double bo_lo, bo_hi;         /* the same as Bond numbers rho g L D / sigma */
    double g_start_lo, g_start_hi; /* starting bracket (planar balance or surrogate) */
    double g_analytic;           /* planar balance's critical force of the initial fill (n_slugs times
                                    one slug's: every slug holds the same capillary balance) */
    double rho_wall[2];          /* wall potentials used */
    double tau[2];               /* relaxation times used */
    double sigma, rho_bulk;      /* of the Bond number */
    int32_t nx, ny;              /* lattice of the channel */
    int32_t probes;              /* probe windows taken */
    int32_t status;              /* as lbm_crit_result.status */
} lbm_channel_result;

/* Bisect the critical body force of every channel (all in one batch, one
 * launch per step, decisions in FP64 on the device): channel and slug from
 * the spec, wall potentials for theta from the calibration table, tau from
 * the viscosity ratio, starting bracket from the planar balance (bracket
 * checks widen it when wrong) or the surrogate, then
 * lbm_critical_pressure_batch.  Returns LBM_ETIMEOUT (results filled) when
 * timeout_s ran out. */
int lbm_critical_pressure_channels(const lbm_channel_spec *specs, int32_t n, const lbm_channel_opts *o,
                                   lbm_channel_result *out);
const char *lbm_channel_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LBM_H */
