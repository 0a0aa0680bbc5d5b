/*
 * mgenkf.h -- C ABI of the GB300 (sm_103a) multigrid ensemble Kalman filter.
 *
 * The library runs the analysis cycle of the Multigrid EnKF (MGEnKF,
 * Algorithm 4 of the paper) on one GPU:
 *   - one fine-grid model run x^F and Ne coarse-grid members x^C,(i), advanced
 *     by the discretised model between observations (Algorithm 4 step 2,
 *     Algorithm 3 step 2; model form Eq. x_mdl);
 *   - restriction x^C* = Pi_C(x^F,f) (Algorithm 4 step 4);
 *   - the stochastic EnKF analysis of the members on the coarse mesh, with
 *     perturbed observations (Eq. perturbed_y), normalised anomalies X, Y
 *     (Eq. Ensemble_Anomaly, Algorithm 3 step 7) and the gain
 *     K = X Y^T (Y Y^T + R)^-1 (Algorithm 3 step 8), R = sigma^2 I diagonal
 *     (Sec. 2.1.1);
 *   - the coarse correction x^C' - x^C* = K (y^o - H^C(x^C*)) prolonged onto
 *     the fine run, x^F,a = x^F,f + Pi_F(x^C' - x^C*) (Algorithm 4 step 5).
 * Pi_C / Pi_F are 4th-order (4-point) Lagrange interpolators on vertex-centred
 * nested periodic grids (end of Sec. 2.2); Pi_C is injection.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an mgenkf_status and never aborts or traps.
 *   - The handle owns all device memory it allocates; caller pointers are
 *     only read (or written) during the call.
 *   - Work is enqueued on the handle's CUDA stream.  Entry points that take
 *     host pointers for outputs (get_state, rmse with a host `out`) synchronise
 *     that stream; the others are asynchronous.
 *   - Device-side failures (non-positive pivot of the innovation matrix,
 *     non-finite observations passed by device pointer) are recorded on the
 *     device; the kernels after the failing one leave the members and the fine
 *     run unchanged, and mgenkf_sync() returns the recorded status.
 *   - A pointer argument is treated as device memory if CUDA reports it as
 *     device or managed memory, otherwise as host memory.
 *   - One handle must not be used from two threads at once.
 */
#ifndef MGENKF_H
#define MGENKF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mgenkf_ctx *mgenkf_handle;

typedef enum {
    MGENKF_OK = 0,
    MGENKF_ERR_INVALID_ARG = 1, /* a size, pointer or option is out of range */
    MGENKF_ERR_OOM = 2,         /* device allocation failed */
    MGENKF_ERR_CUDA = 3,        /* a CUDA runtime call failed (text in last_error) */
    MGENKF_ERR_NOT_SPD = 4,     /* innovation matrix had a non-positive pivot */
    MGENKF_ERR_NONFINITE = 5,   /* observation vector holds NaN or Inf */
    MGENKF_ERR_UNSUPPORTED = 6, /* valid request this build does not implement */
    MGENKF_ERR_TIMEOUT = 7      /* a bounded wait inside a kernel expired (state left unchanged) */
} mgenkf_status;

/* models (Eq. burgers; Eqs. Mass, Momentum, Energy) */
#define MGENKF_BURGERS1D 1
#define MGENKF_NS2D 2
/* arithmetic of the cycle */
#define MGENKF_FP64 0  /* every step in FP64 */
#define MGENKF_MIXED 1 /* FP32 forecasts and states, BF16 anomaly products with
                          FP32 accumulation, FP64 means, covariances, Cholesky */
/* form of the gain solve (identical in exact arithmetic) */
#define MGENKF_GAIN_ENSEMBLE 0 /* T = (I + Y^T R^-1 Y)^-1 Y^T R^-1 [D | d*], Ne x Ne Cholesky */
#define MGENKF_GAIN_DIRECT 1   /* W = (Y Y^T + R)^-1 [D | d*], Ny x Ny Cholesky, T = Y^T W */
/* prolongation of the coarse correction */
#define MGENKF_PROLONG_LAGRANGE4 0

typedef struct {
    int32_t model;     /* MGENKF_BURGERS1D or MGENKF_NS2D */
    int32_t n_fine;    /* fine points per side, N_F */
    int32_t ratio;     /* coarsening ratio r_C; N_F % r_C == 0; coarse N_C = N_F / r_C */
    int32_t n_members; /* Ne >= 2 */
    int32_t n_obs;     /* Ny >= 1 scalar observations */
    int32_t precision; /* MGENKF_FP64 or MGENKF_MIXED */
    int32_t gain_form; /* MGENKF_GAIN_ENSEMBLE or MGENKF_GAIN_DIRECT */
    int32_t prolong;   /* MGENKF_PROLONG_LAGRANGE4 */
    double length;     /* side of the periodic domain (2 pi for Burgers, 1 for NS) */
    double dt;         /* model time step, the same on both grids */
    double nu;         /* Burgers viscosity, or mu = 1/Re for NS */
    double gamma;      /* NS ratio of specific heats */
    double prandtl;    /* NS Prandtl number */
    double obs_sigma;  /* R = obs_sigma^2 I */
    uint64_t seed;     /* key of the Philox4x64-10 stream of observation perturbations */
} mgenkf_config;

/* Create a handle.  obs_index[j]: flat fine-grid node of observation j
 * (x in 1-D, y * N_F + x in 2-D); obs_var[j]: observed variable (0 for
 * Burgers; 0..3 = rho, rho u, rho v, E for NS).  Both host arrays of n_obs
 * entries.  cuda_stream: a cudaStream_t, or NULL for the legacy default
 * stream.  Allocates every device buffer of the cycle; size limits are
 * reported as MGENKF_ERR_INVALID_ARG with a message in mgenkf_last_error. */
mgenkf_status mgenkf_create(const mgenkf_config *cfg, const int32_t *obs_index,
                            const int32_t *obs_var, void *cuda_stream, mgenkf_handle *out);

/* Load the fine state (V * N_F^dim FP64 values, variable-major planes, x
 * fastest) and the members (Ne x V * N_C^dim FP64, member-major).  Host or
 * device pointers.  In MGENKF_MIXED the values are rounded to FP32.
 * Resets the analysis counter that keys the perturbation stream. */
mgenkf_status mgenkf_set_state(mgenkf_handle h, const double *fine, const double *members);

/* Advance the fine run and every member by nsteps SSP-RK3 steps of the model
 * (Algorithm 4 step 2, Algorithm 3 step 2).  nsteps >= 0. */
mgenkf_status mgenkf_forecast(mgenkf_handle h, int32_t nsteps);

/* Layout of the FP32 NS-2D forecast of a mixed-precision handle (Section 6
 * model, SSP-RK3 step of Algorithm 4 step 2 and Algorithm 3 step 2): per grid
 * (members, fine run) a choice c in [0, 16) of the column march, as described
 * at mgenkf_batch_autotune (rows per segment and band width; the two grids
 * then run on two streams), or -1 for both grids: the 2-D tile kernel, both
 * grids in one launch per model step.  The per-point arithmetic, and so every
 * result, is the same for all choices.  The default is set at create from the
 * grid sizes: narrow bands above 256 points per side and the longest segments
 * that still give each grid two units per SM.
 * mgenkf_forecast_autotune times `reps` repetitions (after one warm-up) of
 * ten model steps written to the stage buffers (the states are not touched)
 * for every choice, each grid alone, then both at once as the forecast runs
 * them, and keeps the choice whose fastest repetition is fastest; synchronous.  It does nothing for other handles.
 * mgenkf_set_forecast_choice returns MGENKF_ERR_INVALID_ARG for other handles,
 * for a choice out of range, or for -1 on one grid only. */
mgenkf_status mgenkf_forecast_autotune(mgenkf_handle h, int32_t reps);
mgenkf_status mgenkf_get_forecast_choice(mgenkf_handle h, int32_t *members, int32_t *fine);
mgenkf_status mgenkf_set_forecast_choice(mgenkf_handle h, int32_t members, int32_t fine);

/* Analysis at the current time (Algorithm 4 steps 4-5 first line, Algorithm 3
 * steps 2-3 and 7-8): restriction, predicted observations, anomalies, gain
 * solve, member update and coarse correction dC = x^C' - x^C*.
 * y_obs: n_obs observations (host or device).  eps: Ne x n_obs observation
 * perturbations eps^(i) (member-major, already scaled, host or device), or
 * NULL to draw them on the GPU as obs_sigma * N(0,1) from Philox4x64-10 with
 * key (seed, 0x45505300) and counter (analysis index, n / 4, 0, 0) for
 * n = i * n_obs + j, Box-Muller on lane pairs (0,1) and (2,3).
 * Host-side checks: non-finite host y_obs -> MGENKF_ERR_NONFINITE (nothing
 * enqueued).  Increments the analysis counter. */
mgenkf_status mgenkf_analyse(mgenkf_handle h, const double *y_obs, const double *eps);

/* x^F,a = x^F,f + Pi_F(dC) (Algorithm 4 step 5, second line), plus the
 * residual of the learned correction if one is attached (mgenkf_set_prolong_cnn). */
mgenkf_status mgenkf_prolong_correct(mgenkf_handle h);

/* Attach (or, with NULL, detach) a learned correction (mgk_cnn_t of
 * mgenkf_ops.h, passed as void*): prolong_correct then adds its residual to
 * Pi_F(dC).  Needs MGENKF_NS2D, MGENKF_MIXED, ratio 4 and a CNN built for this
 * handle's coarse size; otherwise MGENKF_ERR_INVALID_ARG.  The handle does not
 * own the CNN. */
mgenkf_status mgenkf_set_prolong_cnn(mgenkf_handle h, void *cnn);

/* One whole cycle: forecast(nsteps), analyse(y_obs, NULL), prolong_correct,
 * and, if truth_fine != NULL, the relative RMSE of the fine run written to
 * rmse_out (V FP64 values; device pointer, or host pointer which makes the
 * call synchronous).  All pointers host or device.  A host truth_fine is copied
 * to the device beside the forecast; the copy has finished when the call
 * returns, so the caller may reuse that buffer at once.  rmse_out is required
 * with truth_fine (MGENKF_ERR_INVALID_ARG otherwise, before any work). */
mgenkf_status mgenkf_cycle(mgenkf_handle h, int32_t nsteps, const double *y_obs,
                           const double *truth_fine, double *rmse_out);

/* Copy the states out as FP64 (host or device pointers; NULL skips one). */
mgenkf_status mgenkf_get_state(mgenkf_handle h, double *fine, double *members);

/* Relative RMSE of the fine run against truth_fine (Eq. L2norm_u), one value
 * per variable: sqrt(sum (x - x_true)^2 / sum x_true^2).  truth_fine: V *
 * N_F^dim FP64 (host or device); out: V FP64 (host or device). */
mgenkf_status mgenkf_rmse(mgenkf_handle h, const double *truth_fine, double *out);

/* Intermediate fields of the last analysis, copied out as FP64 (host or device):
 *   MGENKF_FIELD_XSTAR  x^C* = Pi_C(x^F,f)                  V * N_C^dim
 *   MGENKF_FIELD_YF     H^C x^f,(i) (rows 0..Ne-1), H^C x^C* (row Ne)   (Ne+1) x Ny
 *   MGENKF_FIELD_T      T = Y^T (Y Y^T + R)^-1 [D | d*], column c contiguous  (Ne+1) x Ne
 *   MGENKF_FIELD_DC     dC = x^C' - x^C*                    V * N_C^dim
 *   MGENKF_FIELD_EPS    observation perturbations used      Ne x Ny
 *   MGENKF_FIELD_GAMMA  conservativity residual of the fine  V x N_F^dim
 *                       run (Eq. Conservativity_rhov), see mgenkf_set_regularisation
 *   MGENKF_FIELD_RATE   its time-derivative term (x - x_prev)/dt, V x N_F^dim
 *   MGENKF_FIELD_GAMMA_NORM  Gamma* = Gamma / C per variable, C = the largest
 *                       |x - x_prev| / dt of that variable over the grid (Sec. 6,
 *                       the normalisation of the conservativity maps: C = max
 *                       |d(rho v)/dt|; a variable that did not change keeps
 *                       Gamma), V x N_F^dim
 * count: number of doubles the caller can receive (must be >= the size). */
#define MGENKF_FIELD_XSTAR 0
#define MGENKF_FIELD_YF 1
#define MGENKF_FIELD_T 2
#define MGENKF_FIELD_DC 3
#define MGENKF_FIELD_EPS 4
#define MGENKF_FIELD_GAMMA 5
#define MGENKF_FIELD_RATE 6
#define MGENKF_FIELD_GAMMA_NORM 7
mgenkf_status mgenkf_get_field(mgenkf_handle h, int32_t field, double *out, size_t count);

/* Wait for the handle's stream and return (and clear) the first device-side
 * status recorded since the last call (MGENKF_OK if none). */
mgenkf_status mgenkf_sync(mgenkf_handle h);

/* Limit, in SM clock cycles, of the tensor-core member update's wait for its
 * operands (mixed-precision handles whose update runs on the tensor cores;
 * default about one second at 2 GHz; 0 = one non-blocking test of each
 * operand copy, which gives up unless the copy has already landed).  The paper has no counterpart: every device wait of this library is
 * bounded so that a stalled copy returns MGENKF_ERR_TIMEOUT instead of
 * hanging the GPU, and this sets that bound.  A wait that runs out records
 * MGENKF_ERR_TIMEOUT (reported by mgenkf_sync); the CTA issues no further
 * tensor-core work, waits with the default bound for the copies and products
 * it has in flight, frees its tensor memory and returns, and the kernels after
 * it in the cycle leave the fine run unchanged.  Member tiles a CTA finished
 * before its wait ran out keep their update; with a bound of 0 the first wait
 * runs out before any tile is updated and the members stay unchanged.
 * Errors: MGENKF_ERR_INVALID_ARG for cycles < 0. */
mgenkf_status mgenkf_set_wait_limit(mgenkf_handle h, int64_t cycles);

/* Checkpoint: write / read fine state, members and analysis counter to a file
 * (binary, native endianness, with a header that records the sizes). */
mgenkf_status mgenkf_save(mgenkf_handle h, const char *path);
mgenkf_status mgenkf_load(mgenkf_handle h, const char *path);

/* Text of the last error of this handle (never NULL; empty if none).  Owned by
 * the handle, valid until the next call on it. */
const char *mgenkf_last_error(mgenkf_handle h);

/* Free every device buffer and the handle.  NULL is accepted. */
mgenkf_status mgenkf_destroy(mgenkf_handle h);

/* Final fine-grid iteration (Algorithm 4 step 6) with relaxation alpha (the
 * paper's tailoring in Sec. 3 uses one iteration and alpha = 0.5).  Reading:
 * the last model step of each forecast in implicit-Euler form, x - dt L(x) =
 * x_prev, and one relaxed Jacobi sweep from the analysed fine state:
 *   x <- x + alpha D^-1 (x_prev + dt L(x) - x),
 * D the diagonal of I - dt dL/dx (Burgers: 1 + 2 nu dt / dx^2; NS-2D per
 * point: 1 for rho, 1 + dt (14/3) mu / (rho h^2) for the momenta, 1 + dt 4
 * kappa (gamma - 1) / (rho h^2) for E).  alpha in [0, 1]: from now on every
 * forecast records x_prev (one extra launch and a copy of the fine state) and
 * mgenkf_prolong_correct applies the sweep after Pi_F (and after the learned
 * correction) when alpha > 0; MGENKF_FIELD_GAMMA then returns
 * Gamma = (x - x_prev)/dt - L(x) of the current fine state.  alpha < 0 turns
 * recording off (the default).  Residual and sweep are evaluated in FP64.
 * Not available for handles in a batch.  Errors: MGENKF_ERR_INVALID_ARG for
 * alpha > 1 or not finite. */
mgenkf_status mgenkf_set_regularisation(mgenkf_handle h, double alpha);

/* Centred sixth-order filter of the NS-2D model (the paper's Euler and NS runs
 * damp spurious oscillations with one, Secs. 5 and 6, citing Bogey and
 * Bailly).  Reading: the 7-point stencil u_j -= sigma/64 (-u_{j-3} + 6u_{j-2}
 * - 15u_{j-1} + 20u_j - 15u_{j+1} + 6u_{j+2} - u_{j+3}), transfer function
 * 1 - sigma sin^6(k h/2), along x then y on the four conserved planes.  With
 * sigma > 0 every model step of the members and the fine run (forecast) is the
 * RK3 step followed by the filter; sigma = 0 (default) turns it off.  Not
 * available for handles in a batch.  Errors: MGENKF_ERR_INVALID_ARG for a
 * Burgers handle or sigma outside [0, 1]. */
mgenkf_status mgenkf_set_filter(mgenkf_handle h, double sigma);

/* Fine-to-coarse feedback (the paper's conclusion names projecting the fine
 * run's information onto the ensemble as the next step; reading: re-centring).
 * on != 0: every analysis first re-centres the forecast ensemble on the
 * restricted fine forecast, x^(i) <- x^(i) - mean_i x^(i) + x^C* (FP64 mean),
 * which leaves the anomalies and so the gain unchanged and centres the
 * analysed ensemble on x^C' up to the mean perturbation.  Off by default.
 * If the analysis then fails (status), the members stay re-centred. */
mgenkf_status mgenkf_set_recentre(mgenkf_handle h, int32_t on);

/* ---- Dual EnKF parameter estimation on the Burgers inlet model -----------
 * Sec. 4 (Eq. burgers with the inlet condition Eq. inlet-1D-Burgers:
 * u(0, t) = u0 (1 + theta1 sin(omega t + theta2)), outlet extrapolated) and
 * Algorithm 3 with its parameter rows, run inside Algorithm 4, FP64.  Model:
 * nodes x_j = j length / n_fine, flux-form central scheme, SSP-RK3 with the
 * inlet set at each stage time.  One cycle: fine forecast with the analysed
 * parameter mean; parameter random walk theta^f = theta^a + tau, tau ~ N(0,
 * theta_q I) (Philox4x64-10, key (seed, "THTA"), counter (cycle, n/4, 0, 0));
 * member forecast with theta^f; parameter update theta^a = theta^f + Theta T
 * with T = (I + Y^T R^-1 Y)^-1 Y^T R^-1 D (R = obs_sigma^2 I, perturbations as
 * in mgenkf_analyse); member forecast again from the previous analysis with
 * theta^a and state update with the same perturbations; fine correction with
 * the open-grid 4-point Lagrange Pi_F (one-sided at the ends).  H^C is the
 * Pi_F row at each observed fine node.  Limits: n_fine <= 1024 (one CTA per
 * grid), n_fine / ratio >= 8, ratio in [1, 16], 2 <= n_members <= 256. */
typedef struct mgenkf_dual *mgenkf_dual_t;
typedef struct {
    int32_t n_fine, ratio, n_members, n_obs;
    double length, dt, nu, u0, omega, obs_sigma, theta_q;
    uint64_t seed;
} mgenkf_dual_config;
/* obs_index: n_obs fine-node indices (host); cuda_stream: the stream of every
 * call (NULL = legacy stream).  Errors: MGENKF_ERR_INVALID_ARG, MGENKF_ERR_OOM. */
mgenkf_status mgenkf_dual_create(const mgenkf_dual_config *cfg, const int32_t *obs_index, void *cuda_stream,
                                 mgenkf_dual_t *out);
/* fine (n_fine), members (n_members x n_fine/ratio), theta (n_members x 2:
 * amplitude, phase), theta_fine (2): host or device; t0: the model time. */
mgenkf_status mgenkf_dual_set_state(mgenkf_dual_t d, const double *fine, const double *members,
                                    const double *theta, const double *theta_fine, double t0);
/* nsteps model steps without analysis (fine with theta_fine, members with theirs) */
mgenkf_status mgenkf_dual_free_run(mgenkf_dual_t d, int32_t nsteps);
/* one forecast / analysis cycle of nsteps model steps; y_obs: n_obs values (host or device) */
mgenkf_status mgenkf_dual_cycle(mgenkf_dual_t d, int32_t nsteps, const double *y_obs);
/* copies out (host or device; NULL skips) after waiting for the stream; returns
 * a device-side failure (non-positive pivot) recorded since creation */
mgenkf_status mgenkf_dual_get_state(mgenkf_dual_t d, double *fine, double *members, double *theta,
                                    double *theta_fine);
const char *mgenkf_dual_last_error(mgenkf_dual_t d);
mgenkf_status mgenkf_dual_destroy(mgenkf_dual_t d);

/* ---- batches of independent problems -------------------------------------
 * Many independent NS-2D MGEnKF problems (uneven grid sizes, ensemble sizes
 * and observation counts) advanced together: the forecast of every problem's
 * members and fine run is one launch per model step and grid size over a
 * table of all grids of that size (the sizes on separate streams), and each
 * problem's analysis and prolongation run on one of 16
 * streams (MGENKF_BATCH_STREAMS overrides: 1 to 128).  The whole cycle is captured once into a CUDA graph and replayed by
 * one graph launch per cycle (recaptured if nsteps changes).  The handles stay
 * owned by the caller and must outlive the batch; they must all be
 * MGENKF_NS2D / MGENKF_MIXED with equal gamma, mu and Pr.  While a batch
 * exists its handles must not be used on their own. */
typedef struct mgenkf_batch *mgenkf_batch_t;
/* stream: the stream the batch launches on (cudaStream_t; NULL = a stream
 * the batch creates, ordered with the legacy default stream) */
mgenkf_status mgenkf_batch_create(const mgenkf_handle *handles, int32_t n, void *stream, mgenkf_batch_t *out);
/* One cycle of every problem: forecast(nsteps), analysis with the observations
 * y_obs (all problems' n_obs values concatenated in handle order; host or
 * device; copied before the graph launch) and prolongation (Algorithm 4).
 * innov_out (NULL, or n doubles, host or device): per problem the RMS of the
 * innovation y^o - H^C x^C* of this cycle's fine forecast, copied after the
 * cycle (a pageable host buffer makes the call wait for it).  Otherwise
 * asynchronous. */
mgenkf_status mgenkf_batch_cycle(mgenkf_batch_t b, int32_t nsteps, const double *y_obs, double *innov_out);
/* the forecast part alone, not captured (used to time it) */
mgenkf_status mgenkf_batch_forecast(mgenkf_batch_t b, int32_t nsteps);
/* wait for the batch stream; returns the first device status of any problem */
mgenkf_status mgenkf_batch_sync(mgenkf_batch_t b);
/* Autotuner: for every grid size time `reps` repetitions of one model step
 * (written to scratch: the states are not touched) with each choice of the
 * forecast and keep the fastest.  A choice c in [0, 16) sets the rows per
 * segment of the column march (c mod 8: 0 = 32, 1 = 16, 2 = 64, 3 = 128,
 * 4 = 256, 5 = 24, 6 = 48, 7 = 20) and its band width (c / 8: 0 = the whole
 * width up to 512 points per side, 1 = bands of at most 122 columns with
 * recomputed 3-column halos, about 64 threads per CTA).
 * Then, size by size from the slowest, every choice is timed again with all
 * grid sizes stepping at once on their own streams, as the forecast runs them,
 * and the fastest joint choice is kept.  The arithmetic does not depend on the
 * choice.  Synchronous; invalidates the captured graph. */
mgenkf_status mgenkf_batch_autotune(mgenkf_batch_t b, int32_t reps);
/* read (up to max entries) / set the forecast choice per grid size (`shapes`,
 * each in [0, 16)) */
mgenkf_status mgenkf_batch_tiles(mgenkf_batch_t b, int32_t *sizes, int32_t *shapes, int32_t max, int32_t *count);
mgenkf_status mgenkf_batch_set_tiles(mgenkf_batch_t b, const int32_t *sizes, const int32_t *shapes, int32_t count);
const char *mgenkf_batch_last_error(mgenkf_batch_t b);
mgenkf_status mgenkf_batch_destroy(mgenkf_batch_t b);

#ifdef __cplusplus
}
#endif
#endif /* MGENKF_H */
