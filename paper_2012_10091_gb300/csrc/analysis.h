// analysis.h -- kernels of the coarse-mesh EnKF analysis and the multigrid
// correction (internal to the library).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mgenkf.h"

typedef struct mgk_cnn *mgk_cnn_t;

namespace mgk {

// mgk_cnn_forward with the tensor-core timeout recorded in `status` (the
// handle's status word when the correction runs inside a cycle)
mgenkf_status cnn_forward_status(mgk_cnn_t c, const float *dC, const float *xstar, int batch, float *residual,
                                 int accumulate, int *status, cudaStream_t s);

constexpr int kMaxRatio = 16;

// Lagrange weights of Pi_F for each fine offset m = 0..r-1 (s = m / r).
struct ProlongWeights {
    double w[kMaxRatio][4];
};

// device status codes written by the analysis kernels (values of mgenkf_status)
constexpr int kStNotSpd = 4;
constexpr int kStNonFinite = 5;

// x^C* = Pi_C(x^F): injection at coincident nodes (Algorithm 4 step 4).
template <typename T>
void launch_restrict(const T *fine, T *xstar, int dim, int V, int nc, int r, cudaStream_t s);

// yf[i][j] = sum_t w[j][t] x_i[idx[j][t]] for members i < ne and x^C* (row ne);
// FP32 states with wh, wl (the weights split into FP32 pairs) are summed in
// double-FP32 arithmetic, otherwise in FP64.
template <typename T>
void launch_obs_apply(const T *members, const T *xstar, size_t nx, int ne, int ny, int taps,
                      const int32_t *tap_idx, const double *tap_w, double *yf, cudaStream_t s,
                      const float *wh = nullptr, const float *wl = nullptr);

// FP32 hi/lo copies of Y [ne][ny] and Z [ne+1][ny] (x = hi + lo up to 2^-48
// |x|), the operands of the double-FP32 gain products of the mixed path;
// NULL pointers: none
struct DfOperands {
    float *Yh = nullptr, *Yl = nullptr, *Zh = nullptr, *Zl = nullptr;
};

// ybar_j, innovation of x^C* (row ne of Z), finiteness check of y^o; Zh, Zl
// (if not NULL) receive the split of row ne of Z.
void launch_obs_mean(const double *yf, const double *yo, int ne, int ny, double *ybar, double *Z,
                     int *status, cudaStream_t s, float *Zh = nullptr, float *Zl = nullptr);

// eps (drawn or given), Y = (yf - ybar)/sqrt(ne-1), Z[i] = yo + eps_i - yf_i.
// cycle: device pointer to the analysis counter (Philox counter word 0)
// RMS over the ny innovations d* = y^o - H^C x^C* (row ne of Z) into out[0]
void launch_innov_rms(const double *Z, int ne, int ny, double *out, cudaStream_t s);
// Final fine-grid iteration (Algorithm 4 step 6) and conservativity residual
// (Eq. Conservativity_rhov) of the fine run x against x_prev, the state one
// model step earlier: out (if not NULL) = x - alpha dt D^-1 Gamma, gamma_out
// (if not NULL, FP64) = Gamma = (x - x_prev)/dt - L(x).  model 1 = Burgers,
// 2 = NS-2D (n points per side, 4 planes).  out must not alias x.
template <typename T>
void launch_fine_residual(int model, const T *x, const T *prev, int n, double length, double nu, double gamma,
                          double prandtl, double dt, double alpha, T *out, double *gamma_out, const int *status,
                          cudaStream_t s);

// centred sixth-order filter (Secs. 5, 6) of nprob NS grids of n x n points,
// 4 conserved planes each, in place; tmp holds one copy of them
template <typename T>
cudaError_t launch_ns2d_filter6(T *q, T *tmp, int n, int nprob, double sigma, cudaStream_t s);

// out = (x - prev) / dt in FP64 (count values)
template <typename T>
void launch_state_rate(const T *x, const T *prev, size_t count, double dt, double *out, cudaStream_t s);

// gamma (V planes of `plane` FP64 values) divided in place, per plane, by
// max |x - prev| / dt of that plane (left as is where the plane did not change)
template <typename T>
void launch_gamma_norm(const T *x, const T *prev, int V, size_t plane, double dt, double *gamma, cudaStream_t s);

// fine-to-coarse feedback: members re-centred on x^C* (FP64 mean and shift)
template <typename T>
void launch_recentre(T *members, size_t nx, int ne, const T *xstar, const int *status, cudaStream_t s);

// gen_eps: 0 = eps given, 1 = perturbations drawn in FP64, 2 = the same Philox
// words with the Box-Muller transform in FP32 (mixed precision)
void launch_obs_perturb(const double *yf, const double *ybar, const double *yo, double *eps,
                        int gen_eps, uint64_t seed, const uint64_t *cycle, double sigma, int ne, int ny,
                        double *Y, double *Z, cudaStream_t s, const DfOperands &df = DfOperands());
void launch_bump_counter(uint64_t *c, cudaStream_t s);

// normalised state anomalies X (Eq. Ensemble_Anomaly); FP64 [ne][nx] or BF16 [nx][ne].
template <typename T>
void launch_ens_anom(const T *members, size_t nx, int ne, double *X64, __nv_bfloat16 *X16,
                     const int *status, cudaStream_t s);

// out1[a][c] = diag*(a==c) + scale*sum_k A[a][k] B1[c][k]   (c < n1, row-major, ld n1)
// out2[c][a] = scale*sum_k A[a][k] B2[c][k]                 (c < n2, "column c contiguous")
// part: optional scratch of gemm_nt_splits(...) * m * (n1 + n2) doubles; with
// it, long K is split over more CTAs and the chunks are summed in order.
void launch_gemm_nt_f64(const double *A, int m, const double *B1, int n1, const double *B2, int n2,
                        int K, double scale, double diag, double *out1, double *out2,
                        const int *status, cudaStream_t s, double *part = nullptr);
int gemm_nt_splits(int m, int n1, int n2, int K);
// S = I + Y^T R^-1 Y (ne x ne) and Bt = Y^T R^-1 [D | d*] (column c of Bt
// contiguous) as launch_gemm_nt_f64 (same split of K with `part`), from the
// double-FP32 operands, summed in double-FP32 arithmetic (mixed precision).
void launch_gemm_df(const DfOperands &df, int ne, int ny, double s2, double *S, double *Bt, const int *status,
                    cudaStream_t s, double *part);

// C[j][l] = sum_i Y[i][j] Y[i][l] + diag*(j==l), j,l < ny (direct form).
void launch_gemm_tn_f64(const double *Y, int ne, int ny, double diag, double *C, const int *status,
                        cudaStream_t s);

// In-place Cholesky of the n x n SPD matrix A (row-major); writes L (lower,
// row-major, upper zeroed) over A and its transpose to Lt.  Sets NOT_SPD.
void launch_cholesky(double *A, double *Lt, int n, int *status, cudaStream_t s);

// Solve L L^T x_c = rhs_c for ncol columns of length n; x -> out (FP64) and,
// if out16 != NULL, BF16 copy to out16 with row stride ld16.
void launch_chol_solve(const double *L, const double *Lt, int n, const double *rhs, double *out,
                       int ncol, __nv_bfloat16 *out16, int ld16, const int *status, cudaStream_t s);

// members[c] += X T[c] (c < ne), dC = X T[ne]   (T column c contiguous, (ne+1) x ne)
template <typename T>
void launch_update_f64(T *members, T *dC, const double *X, const double *Tm, size_t nx, int ne,
                       const int *status, cudaStream_t s);
void launch_update_bf16(float *members, float *dC, const __nv_bfloat16 *Xt, const __nv_bfloat16 *Tt,
                        int ldT, size_t nx, int ne, const int *status, cudaStream_t s);

// fine += Pi_F(dC)
template <typename T>
void launch_prolong_add(T *fine, const T *dC, int dim, int V, int nc, int r,
                        const ProlongWeights &w, const int *status, cudaStream_t s);

// relative RMSE per variable (Eq. L2norm_u): partial sums + final reduction.
template <typename T>
void launch_rmse(const T *x, const double *truth, int V, size_t npts, double *partials,
                 int nblocks, double *out, cudaStream_t s);
constexpr int kRmseBlocks = 304;

// Tt[c][a] = bf16(T[c][a]) for c <= ne, a < ne (row stride ld, padding untouched).
void launch_tt_bf16(const double *Tm, __nv_bfloat16 *Tt, int ne, int ld, const int *status,
                    cudaStream_t s);

template <typename Tin, typename Tout>
void launch_convert(const Tin *in, Tout *out, size_t n, cudaStream_t s);

void launch_normals(uint64_t seed, uint64_t tag, uint64_t ctr0, int64_t count, double *out,
                    cudaStream_t s);

}  // namespace mgk
