/*
 * mgenkf_ops.h -- stateless GPU entry points of the MGEnKF library.
 *
 * These run single steps of the cycle on caller-owned device memory.  They
 * serve truth runs (the synthetic reference trajectory that observations are
 * sampled from, Sec. 4 and Sec. 6 of the paper) and step-level checks.  Same
 * conventions as mgenkf.h: status return, asynchronous on `stream`
 * (a cudaStream_t or NULL), no allocation of persistent memory.
 */
#ifndef MGENKF_OPS_H
#define MGENKF_OPS_H

#include <stddef.h>
#include <stdint.h>

#include "mgenkf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Advance nprob independent periodic grids by nsteps SSP-RK3 steps of the
 * model (Eq. x_mdl with M = the discretised Eq. burgers, or Eqs. Mass,
 * Momentum, Energy for MGENKF_NS2D).
 *   state: device pointer to nprob consecutive states of V * n^dim values,
 *          FP64 if precision == MGENKF_FP64, FP32 if MGENKF_MIXED; updated in place.
 *   n: points per side; length: domain side; dt: time step; nu: viscosity
 *   (Burgers) or mu = 1/Re (NS); gamma, prandtl: NS gas constants (ignored for
 *   Burgers).
 * Limits: Burgers n in [4, 32768]; NS n in [8, 4096] and n % 8 == 0; NS FP32
 * states start on a 16-byte boundary (the halo is copied in 16-byte chunks).
 * Outside them: MGENKF_ERR_INVALID_ARG. */
mgenkf_status mgk_forecast(int32_t model, int32_t precision, void *state, int32_t nprob, int32_t n,
                           double length, double dt, double nu, double gamma, double prandtl,
                           int32_t nsteps, void *stream);

/* count standard normals into the device array `out` (FP64), drawn exactly as
 * the analysis draws its perturbations: Philox4x64-10 (Salmon et al., SC'11)
 * with key (seed, tag) and counter (ctr0, n / 4, 0, 0), uniforms
 * ((x >> 11) + 1) * 2^-53, Box-Muller on lane pairs (0,1) and (2,3). */
mgenkf_status mgk_normals(uint64_t seed, uint64_t tag, uint64_t ctr0, int64_t count, double *out,
                          void *stream);

/* ---- learned correction of the prolongation ------------------------------
 * The paper's conclusion names better projection operators between the grids
 * as a direction; this object is a small CNN that predicts the part of the fine
 * correction that Pi_F(dC) misses (residual over Pi_F), trained on corrections
 * of a full-resolution EnKF.  Input: the 8 coarse channels [dC (4), x^C* (4)]
 * of an NS-2D analysis (n_coarse^2 each), normalised as (v - mu_in) / s_in.
 * Three 3x3 convolutions with periodic padding, 8 -> 32 -> 32 -> 64 channels,
 * ReLU after the first two; the 64 channels are pixel-shuffled by 4 into 4 fine
 * channels (fine (4y+sy, 4x+sx) of channel c = channel 16c + 4sy + sx) and
 * scaled by s_out[c].  BF16 weights and activations, FP32 accumulation, FP32
 * master weights and Adam state.  Parameters: 30080 floats in the order
 * W1 (32x8x3x3), b1 (32), W2 (32x32x3x3), b2 (32), W3 (64x32x3x3), b3 (64).
 * All arrays are FP32 device pointers unless stated; one object per thread. */
typedef struct mgk_cnn *mgk_cnn_t;
mgenkf_status mgk_cnn_create(int32_t n_coarse, int32_t batch_max, mgk_cnn_t *out);
mgenkf_status mgk_cnn_destroy(mgk_cnn_t cnn);
/* coarse points per side the object was built for (0 for NULL) */
int32_t mgk_cnn_coarse_size(mgk_cnn_t cnn);
/* params: 30080 floats (host or device) or NULL; stats: mu_in[8], s_in[8],
 * s_out[4] (host or device) or NULL.  Setting params resets the Adam state. */
mgenkf_status mgk_cnn_set_params(mgk_cnn_t cnn, const float *params, const float *stats);
/* copy out the master parameters and/or the last gradients (host or device; NULL skips) */
mgenkf_status mgk_cnn_get_params(mgk_cnn_t cnn, float *params, float *grads);
/* residual (batch x 4 x (4n)^2) = s_out * shuffle(CNN(dC, x*)), written, or added if accumulate != 0.
 * dC, xstar: batch x 4 x n^2. */
mgenkf_status mgk_cnn_forward(mgk_cnn_t cnn, const float *dC, const float *xstar, int32_t batch,
                              float *residual, int32_t accumulate, void *stream);
/* loss = mean(((Pi_F(dC) + residual - target) / s_out)^2) over batch, channels and
 * fine points, and its gradient with respect to every parameter (kept in the
 * object).  target: batch x 4 x (4n)^2 fine corrections.  loss_out: one float
 * (host or device) or NULL. */
mgenkf_status mgk_cnn_loss_grad(mgk_cnn_t cnn, const float *dC, const float *xstar, const float *target,
                                int32_t batch, float *loss_out, void *stream);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) with the last gradients */
mgenkf_status mgk_cnn_adam_step(mgk_cnn_t cnn, float lr, void *stream);

/* Ensemble-space gain solve that allocates nothing.
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc (an application whose own pool owns all device memory, a process
 * under a fixed device-memory budget, code that must not make allocation calls
 * that synchronise the device).  It computes, in FP64, the same T as the
 * handle's analysis with MGENKF_GAIN_ENSEMBLE:
 *   S = I + Y^T Y / sigma^2,  S = L L^T,  T = S^-1 Y^T [D | d*] / sigma^2.
 *   Y: device, n_members x n_obs, row i = normalised observation anomaly of member i;
 *   Z: device, (n_members + 1) x n_obs, rows D_i = y^o + eps_i - y^f_i, last row d* = y^o - H^C x^C*;
 *   T: device output, (n_members + 1) x n_members, column c of T contiguous (T[c * n_members + a]);
 *   info: optional device int32 set to 0, or MGENKF_ERR_NOT_SPD if a pivot was not positive.
 * Y, Z, T and info must be device (or managed) memory of the current device:
 * other pointers return MGENKF_ERR_INVALID_ARG before any work.  A CUDA error
 * left pending by earlier work is reported as MGENKF_ERR_CUDA (and left
 * pending for its owner) without launching anything.
 * Scratch (S, L^T, status) lives in a fixed array compiled into the library,
 * held by every GPU that loads it until exit (256 KB); hence n_members <= 128,
 * larger sizes return MGENKF_ERR_INVALID_ARG with a message.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All
 * calls share the array (its status word is cleared at the start of each call):
 * calls whose work overlaps on the GPU race and must be serialised by the caller.
 * Asynchronous on `stream`. */
mgenkf_status mgk_gain_ensemble_noalloc(const double *Y, const double *Z, int32_t n_members,
                                        int32_t n_obs, double obs_sigma, double *T, int32_t *info,
                                        void *stream);

/* Throughput probe of the FMA pipes.  The paper has no counterpart: this is
 * the denominator of the arithmetic roofline that the forecast (FP32) and the
 * Cholesky (FP64) are measured against, since no library routine has the
 * same pipe mix.  Launches four 256-thread CTAs per SM on `stream`, each thread
 * running eight independent chains of `iters` fused multiply-adds (FP64 if
 * fp64 != 0, else FP32), and writes one value per thread into `sink` (device,
 * mgk_fma_probe_threads() elements of double or float).  *flops (host) is set
 * to the floating-point operations of the launch (an FMA counts two); the
 * caller times the launch and divides.  Errors: MGENKF_ERR_INVALID_ARG for
 * iters < 1 or null pointers, MGENKF_ERR_CUDA for a failed launch. */
mgenkf_status mgk_fma_probe(int32_t fp64, int32_t iters, void *sink, double *flops, void *stream);
/* Elements `sink` must hold on the current device (-1 on a CUDA error). */
int32_t mgk_fma_probe_threads(void);

/* Number of GPU kernels the library has launched in this process so far
 * (every entry point counts its own launches; memsets and copies excluded). */
uint64_t mgk_kernel_launches(void);

/* Text of the last error raised by an mgk_* call on this host thread. */
const char *mgk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MGENKF_OPS_H */
