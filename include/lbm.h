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
 * asynchronously on the handle's stream.  Returns the launch status;
 * instability is reported by lbm_observables. */
int lbm_step(lbm_t *h, int64_t nsteps);

/* Synchronise the stream and copy the observables of the latest step.
 * Returns LBM_ETIMEOUT once timeout_flag is set, else LBM_EUNSTABLE once
 * nan_flag is set (*out is filled in both cases). */
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

/* Change the body-force acceleration used by the following steps. */
int lbm_set_body_force(lbm_t *h, double gx, double gy);

/* Copy the stored post-collision populations to / from a host FP64 array
 * f[2][9][ny][nx] (species, direction, y, x; directions c_0 = (0,0),
 * c_1..c_4 = (1,0),(0,1),(-1,0),(0,-1), c_5..c_8 = (1,1),(-1,1),(-1,-1),(1,-1)).
 * lbm_load also resets the observables (step count, displacement, NaN flag). */
int lbm_save(lbm_t *h, double *f);
int lbm_load(lbm_t *h, const double *f);

/* Launch configuration the autotuner chose for the step kernel:
 * info[0] = variant (1 simple, 2 staged, 3 pipelined, 4 private); info[1] =
 * rows in flight (variants 2..4); info[2] = rows per CTA strip (variant 1)
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
 *   p     host parameters: precision must be LBM_FP32; nx * ny <= 2097152;
 *         p->cuda_stream is the stream of all work; variant and workspace
 *         fields are ignored
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

/* Advance every active instance by nsteps (asynchronous). */
int lbm_batch_step(lbm_batch_t *b, int64_t nsteps);

/* Observables of every instance (out[n]); LBM_EUNSTABLE if any NaN flag,
 * else LBM_ETIMEOUT if a bounded device wait gave up in some step. */
int lbm_batch_observables(lbm_batch_t *b, lbm_obs *out);

/* Step kernel of the batch: info[0] = 2 staged (TMA) march, 1 register-pull
 * march; info[1] = rows per strip of the staged tiles (0 otherwise);
 * info[2] = CTAs per step.  Not part of the paper's method: a report of this
 * library's tiling. */
int lbm_batch_kernel_info(const lbm_batch_t *b, int32_t info[3]);

/* Set the x body force of every instance (gx[n]). */
int lbm_batch_set_body_force(lbm_batch_t *b, const double *gx);

/* Stored populations of instance i as lbm_save does for a single grid. */
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
 * device in FP64.  Returns LBM_ETIMEOUT (results filled, status 3) when
 * timeout_s ran out. */
int lbm_critical_pressure_batch(lbm_batch_t *b, const double *g_lo, const double *g_hi,
                                const lbm_bisect_opts *o, lbm_crit_result *out);

void lbm_batch_destroy(lbm_batch_t *b);
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

#ifdef __cplusplus
}
#endif

#endif /* GB300_LBM_H */
