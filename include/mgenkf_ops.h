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
 * Limits: Burgers n in [4, 32768]; NS n in [8, 4096] and n % 8 == 0.  Outside
 * them: MGENKF_ERR_INVALID_ARG. */
mgenkf_status mgk_forecast(int32_t model, int32_t precision, void *state, int32_t nprob, int32_t n,
                           double length, double dt, double nu, double gamma, double prandtl,
                           int32_t nsteps, void *stream);

/* count standard normals into the device array `out` (FP64), drawn exactly as
 * the analysis draws its perturbations: Philox4x64-10 (Salmon et al., SC'11)
 * with key (seed, tag) and counter (ctr0, n / 4, 0, 0), uniforms
 * ((x >> 11) + 1) * 2^-53, Box-Muller on lane pairs (0,1) and (2,3). */
mgenkf_status mgk_normals(uint64_t seed, uint64_t tag, uint64_t ctr0, int64_t count, double *out,
                          void *stream);

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

/* Number of GPU kernels the library has launched in this process so far
 * (every entry point counts its own launches; memsets and copies excluded). */
uint64_t mgk_kernel_launches(void);

/* Text of the last error raised by an mgk_* call on this host thread. */
const char *mgk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MGENKF_OPS_H */
