// analysis.cu -- kernels of the coarse-mesh EnKF analysis (Algorithm 3, state
// part: steps 2-3, 7-8) and of the multigrid correction (Algorithm 4 steps 4-5).
//
// Layout (per analysis): members [ne][nx] (member-major, state vector of one
// member contiguous), predicted observations yf [ne+1][ny] (row ne = H^C x^C*),
// anomalies Y [ne][ny], innovations Z [ne+1][ny] (row i = y^o + eps_i - yf_i,
// row ne = y^o - H^C x^C*), gain coefficients T [(ne+1)][ne] (column c of
// T = Y^T C^-1 [D | d*] contiguous).  Every covariance-type reduction, the
// Cholesky factorisation and the triangular solves run in FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>

#include "analysis.h"
#include "batch_analysis.h"
#include "common.cuh"
#include "update_tc.h"

namespace mgk {
namespace cg = cooperative_groups;

static inline int grid_for(size_t n, int block, int cap = 8 * kNumSMs) {
    long long g = (long long)((n + block - 1) / block);
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------------------
// restriction Pi_C (injection), Algorithm 4 step 4
// ---------------------------------------------------------------------------
// Kernel bodies take their block index and block count as arguments, so that
// the grouped analysis of many problems (one launch per step, blocks mapped to
// problems by a table) runs the same per-element arithmetic as one handle.
template <typename T>
__device__ __forceinline__ void restrict_body(const T *__restrict__ fine, T *__restrict__ xs, int dim, int V,
                                              int nc, int r, size_t blk, size_t nblk, T *__restrict__ zero) {
    const size_t nf = (size_t)nc * r;
    const size_t cpl = dim == 1 ? (size_t)nc : (size_t)nc * nc;
    const size_t fpl = dim == 1 ? nf : nf * nf;
    const size_t total = (size_t)V * cpl;
    for (size_t i = blk * blockDim.x + threadIdx.x; i < total; i += nblk * blockDim.x) {
        const size_t v = i / cpl, k = i % cpl;
        size_t src;
        if (dim == 1) {
            src = (size_t)r * k;
        } else {
            const size_t jy = k / nc, jx = k % nc;
            src = (size_t)r * jy * nf + (size_t)r * jx;
        }
        xs[i] = fine[v * fpl + src];
        if (zero) zero[i] = T(0);  // the coarse correction, cleared before the analysis writes it
    }
}

template <typename T>
__global__ void k_restrict(const T *__restrict__ fine, T *__restrict__ xs, int dim, int V, int nc, int r) {
    restrict_body<T>(fine, xs, dim, V, nc, r, blockIdx.x, gridDim.x, nullptr);
}

template <typename T>
void launch_restrict(const T *fine, T *xstar, int dim, int V, int nc, int r, cudaStream_t s) {
    count_launches(1);
    const size_t total = (size_t)V * (dim == 1 ? (size_t)nc : (size_t)nc * nc);
    k_restrict<T><<<grid_for(total, 256), 256, 0, s>>>(fine, xstar, dim, V, nc, r);
}

// ---------------------------------------------------------------------------
// predicted observations H^C x (Algorithm 3 step 2): sparse 4- or 16-tap rows
// ---------------------------------------------------------------------------
// Thread: observation j = bx * blockDim.x + threadIdx.x, rows i = i0 .. i0 +
// rows - 1 of yf (members, then x^C* as row ne); its taps (<= 16) stay in
// registers for those rows.  One problem alone takes 2 rows per thread (enough
// threads to hide the gathers); a grouped launch over many problems 8.
constexpr int kObsRows = 8, kObsRowsOne = 2;

// With FP32 states and the weights split into FP32 pairs (wh, wl: w = wh + wl
// up to 2^-48 |w|, mixed precision) the taps are summed in double-FP32
// arithmetic on the FP32 pipes: wh x exactly as p + e (e by FMA), wl x
// rounded, the products summed into a running FP32 sum and the FP32 sum of its
// rounding errors (error-free two-sum); otherwise in FP64.
template <typename T>
__device__ __forceinline__ void obs_apply_body(const T *__restrict__ members, const T *__restrict__ xstar,
                                               size_t nx, int ne, int ny, int taps,
                                               const int32_t *__restrict__ tap_idx,
                                               const double *__restrict__ tap_w, double *__restrict__ yf, int bx,
                                               int i0, int rows, const float *__restrict__ wh = nullptr,
                                               const float *__restrict__ wl = nullptr) {
    const int j = bx * blockDim.x + threadIdx.x;
    if (j >= ny) return;
    int32_t idx[16];
    const int i1 = min(i0 + rows, ne + 1);
    if constexpr (std::is_same<T, float>::value) {
        if (wh) {
            float w1[16], w2[16];
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if (t < taps) {
                    idx[t] = tap_idx[(size_t)j * taps + t];
                    w1[t] = wh[(size_t)j * taps + t];
                    w2[t] = wl[(size_t)j * taps + t];
                }
            for (int i = i0; i < i1; ++i) {
                const float *x = i < ne ? members + (size_t)i * nx : xstar;
                float s = 0.f, c = 0.f;
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (t < taps) {
                        const float xv = x[idx[t]];
                        const float p = __fmul_rn(w1[t], xv), e = __fmaf_rn(w1[t], xv, -p);
                        const float q = __fmul_rn(w2[t], xv);
                        const float u = __fadd_rn(s, p), bv = __fsub_rn(u, s);
                        c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(u, bv)), __fsub_rn(p, bv)),
                                                   __fadd_rn(e, q)));
                        s = u;
                    }
                yf[(size_t)i * ny + j] = (double)s + (double)c;
            }
            return;
        }
    }
    double w[16];
#pragma unroll
    for (int t = 0; t < 16; ++t)
        if (t < taps) {
            idx[t] = tap_idx[(size_t)j * taps + t];
            w[t] = tap_w[(size_t)j * taps + t];
        }
    for (int i = i0; i < i1; ++i) {
        const T *x = i < ne ? members + (size_t)i * nx : xstar;
        double acc = 0.0;
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (t < taps) acc = fma(w[t], (double)x[idx[t]], acc);
        yf[(size_t)i * ny + j] = acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_obs_apply(const T *__restrict__ members, const T *__restrict__ xstar,
                                                   size_t nx, int ne, int ny, int taps,
                                                   const int32_t *__restrict__ tap_idx,
                                                   const double *__restrict__ tap_w, double *__restrict__ yf,
                                                   const float *__restrict__ wh, const float *__restrict__ wl) {
    obs_apply_body<T>(members, xstar, nx, ne, ny, taps, tap_idx, tap_w, yf, blockIdx.x, blockIdx.y * kObsRowsOne,
                      kObsRowsOne, wh, wl);
}

template <typename T>
void launch_obs_apply(const T *members, const T *xstar, size_t nx, int ne, int ny, int taps,
                      const int32_t *tap_idx, const double *tap_w, double *yf, cudaStream_t s, const float *wh,
                      const float *wl) {
    count_launches(1);
    dim3 grid(ceil_div(ny, 128), ceil_div(ne + 1, kObsRowsOne));
    k_obs_apply<T><<<grid, 128, 0, s>>>(members, xstar, nx, ne, ny, taps, tap_idx, tap_w, yf, wh, wl);
}

// ---------------------------------------------------------------------------
// observation means and innovations (Algorithm 1 step 4; Algorithm 4 step 5)
// ---------------------------------------------------------------------------
// x = hi[o] + lo[o] up to 2^-48 |x|: hi = x rounded to FP32, lo = the
// remainder (exact in FP64) rounded to FP32.  The operands of the
// double-FP32 gain products (mixed precision).
__device__ __forceinline__ void split_df(double x, float *__restrict__ hi, float *__restrict__ lo, size_t o) {
    const float h = __double2float_rn(x);
    hi[o] = h;
    lo[o] = __double2float_rn(__dsub_rn(x, (double)h));
}

// yo_copy (if not NULL) receives y^o as read; Zh, Zl (if not NULL) the
// double-FP32 split of row ne of Z
__device__ __forceinline__ void obs_mean_body(const double *__restrict__ yf, const double *__restrict__ yo, int ne,
                                              double inv_ne, int ny, double *__restrict__ ybar,
                                              double *__restrict__ Z, int *status, int blk,
                                              double *__restrict__ yo_copy, float *__restrict__ Zh = nullptr,
                                              float *__restrict__ Zl = nullptr) {
    // 32 observations per CTA (lane), 8 slices of the members (warp); the slice
    // sums are combined in a fixed order.
    __shared__ double part[8][33];
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int j = blk * 32 + lane;
    double acc = 0.0;
    if (j < ny)
        for (int i = slice; i < ne; i += 8) acc += yf[(size_t)i * ny + j];
    part[slice][lane] = acc;
    __syncthreads();
    if (slice == 0 && j < ny) {
        double sum = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) sum += part[q][lane];
        ybar[j] = sum * inv_ne;
        const double y = yo[j];
        if (!isfinite(y)) atomicCAS(status, 0, kStNonFinite);
        if (yo_copy) yo_copy[j] = y;
        const double d = y - yf[(size_t)ne * ny + j];
        Z[(size_t)ne * ny + j] = d;
        if (Zh) split_df(d, Zh, Zl, (size_t)ne * ny + j);
    }
}

__global__ void __launch_bounds__(256) k_obs_mean(const double *__restrict__ yf, const double *__restrict__ yo,
                                                  int ne, double inv_ne, int ny, double *__restrict__ ybar,
                                                  double *__restrict__ Z, int *status, float *__restrict__ Zh,
                                                  float *__restrict__ Zl) {
    obs_mean_body(yf, yo, ne, inv_ne, ny, ybar, Z, status, blockIdx.x, nullptr, Zh, Zl);
}

void launch_obs_mean(const double *yf, const double *yo, int ne, int ny, double *ybar, double *Z,
                     int *status, cudaStream_t s, float *Zh, float *Zl) {
    count_launches(1);
    k_obs_mean<<<ceil_div(ny, 32), 256, 0, s>>>(yf, yo, ne, 1.0 / ne, ny, ybar, Z, status, Zh, Zl);
}

// RMS of the innovation d* = y^o - H^C x^C* (one value; fixed-order FP64 sums)
__device__ __forceinline__ void innov_rms_body(const double *__restrict__ d, int ny, double *__restrict__ out) {
    __shared__ double part[256];
    double acc = 0.0;
    for (int j = threadIdx.x; j < ny; j += 256) acc = fma(d[j], d[j], acc);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(part[0] / ny);
}

__global__ void __launch_bounds__(256) k_innov_rms(const double *__restrict__ d, int ny, double *__restrict__ out) {
    innov_rms_body(d, ny, out);
}

void launch_innov_rms(const double *Z, int ne, int ny, double *out, cudaStream_t s) {
    k_innov_rms<<<1, 256, 0, s>>>(Z + (size_t)ne * ny, ny, out);
    count_launches(1);
}

// perturbed observations (Eq. perturbed_y) and normalised anomalies Y (Algorithm 3 step 7)
// One thread per Philox block: the 4 consecutive elements o = 4b .. 4b + 3 of
// the Ne x Ny perturbation matrix (flat index o = i Ny + j).  gen_eps: 0 = eps
// given, 1 = normals in FP64, 2 = Box-Muller in FP32 (the mixed path).
template <bool F32>
__device__ __forceinline__ void obs_perturb_body(const double *__restrict__ yf, const double *__restrict__ ybar,
                                                 const double *__restrict__ yo, double *__restrict__ eps,
                                                 int gen_eps, uint64_t seed, const uint64_t *__restrict__ cycle,
                                                 double sigma, int ne, int ny, double isq, double *__restrict__ Y,
                                                 double *__restrict__ Z, size_t blk, float *__restrict__ Yh = nullptr,
                                                 float *__restrict__ Yl = nullptr, float *__restrict__ Zh = nullptr,
                                                 float *__restrict__ Zl = nullptr) {
    const size_t total = (size_t)ne * ny;
    const size_t b = blk * blockDim.x + threadIdx.x;
    if (4 * b >= total) return;
    double z[4];
    if (gen_eps) {
        if (F32)
            philox_normals4_f32(seed, kEpsTag, *cycle, (uint64_t)b, z);
        else
            philox_normals4(seed, kEpsTag, *cycle, (uint64_t)b, z);
    }
    int i = (int)((4 * b) / ny), j = (int)(4 * b - (size_t)i * ny);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const size_t o = 4 * b + l;
        if (o < total) {
            // explicit roundings: no contraction into an FMA, whatever the
            // kernel the body is inlined into
            double e;
            if (gen_eps) {
                e = __dmul_rn(sigma, z[l]);
                eps[o] = e;
            } else {
                e = eps[o];
            }
            const double f = yf[o];
            const double yv = __dmul_rn(__dsub_rn(f, ybar[j]), isq), zv = __dsub_rn(__dadd_rn(yo[j], e), f);
            Y[o] = yv;
            Z[o] = zv;
            if (Yh) {
                split_df(yv, Yh, Yl, o);
                split_df(zv, Zh, Zl, o);
            }
        }
        if (++j == ny) {
            j = 0;
            ++i;
        }
    }
}

template <bool F32>
__global__ void k_obs_perturb(const double *__restrict__ yf, const double *__restrict__ ybar,
                              const double *__restrict__ yo, double *__restrict__ eps, int gen_eps, uint64_t seed,
                              const uint64_t *__restrict__ cycle, double sigma, int ne, int ny, double isq,
                              double *__restrict__ Y, double *__restrict__ Z, float *__restrict__ Yh,
                              float *__restrict__ Yl, float *__restrict__ Zh, float *__restrict__ Zl) {
    obs_perturb_body<F32>(yf, ybar, yo, eps, gen_eps, seed, cycle, sigma, ne, ny, isq, Y, Z, blockIdx.x, Yh, Yl, Zh,
                          Zl);
}

void launch_obs_perturb(const double *yf, const double *ybar, const double *yo, double *eps,
                        int gen_eps, uint64_t seed, const uint64_t *cycle, double sigma, int ne, int ny,
                        double *Y, double *Z, cudaStream_t s, const DfOperands &df) {
    count_launches(1);
    const size_t blocks = ((size_t)ne * ny + 3) / 4;
    // isq = 1/sqrt(Ne - 1) from the host (an FP64 division and square root per thread on the device)
    const unsigned grid = (unsigned)ceil_div(blocks, 128);
    const double isq = 1.0 / std::sqrt((double)(ne - 1));
    if (gen_eps == 2)
        k_obs_perturb<true><<<grid, 128, 0, s>>>(yf, ybar, yo, eps, 1, seed, cycle, sigma, ne, ny, isq, Y, Z, df.Yh,
                                                 df.Yl, df.Zh, df.Zl);
    else
        k_obs_perturb<false><<<grid, 128, 0, s>>>(yf, ybar, yo, eps, gen_eps, seed, cycle, sigma, ne, ny, isq, Y, Z,
                                                  df.Yh, df.Yl, df.Zh, df.Zl);
}

// Fine-to-coarse feedback: the forecast ensemble re-centred on the restricted
// fine forecast, x^(i) += x^C* - mean_i x^(i) (FP64 mean and shift).  One
// thread per point; members member-major.
template <typename T>
__global__ void __launch_bounds__(256) k_recentre(T *__restrict__ m, size_t nx, int ne, const T *__restrict__ xstar,
                                                  const int *status) {
    if (*status) return;
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (p >= nx) return;
    double s = 0.0;
    for (int i = 0; i < ne; ++i) s += (double)m[(size_t)i * nx + p];
    const double shift = (double)xstar[p] - s / ne;
    for (int i = 0; i < ne; ++i) m[(size_t)i * nx + p] = (T)((double)m[(size_t)i * nx + p] + shift);
}

template <typename T>
void launch_recentre(T *members, size_t nx, int ne, const T *xstar, const int *status, cudaStream_t s) {
    count_launches(1);
    k_recentre<T><<<(unsigned)ceil_div(nx, 256), 256, 0, s>>>(members, nx, ne, xstar, status);
}
template void launch_recentre<float>(float *, size_t, int, const float *, const int *, cudaStream_t);
template void launch_recentre<double>(double *, size_t, int, const double *, const int *, cudaStream_t);

// ---------------------------------------------------------------------------
// ensemble mean and normalised anomalies X
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void ens_anom_body(const T *__restrict__ m, size_t nx, int ne, double inv_ne, double isq,
                                              double *__restrict__ X64, __nv_bfloat16 *__restrict__ X16, int ldx,
                                              const int *status, size_t blk) {
    // CTA: 32 consecutive points (lane) x the members split over the 8 warps.
    // Mean: per-warp slice sums combined in a fixed order by warp 0; then the
    // normalised anomalies: FP64 member-major rows, or BF16 point-major rows
    // assembled in shared memory so every row of ldx values is stored
    // contiguously.  GB300 runs about 2 FP64 FMAs per clock per SM, so FP32
    // states are averaged without FP64 operations (below), and 1/Ne and
    // 1/sqrt(Ne - 1) come from the host.
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double *part = reinterpret_cast<double *>(sm_raw);                        // [8][32]
    double *mean = part + 8 * 32;                                             // [32]
    __nv_bfloat16 *tile = reinterpret_cast<__nv_bfloat16 *>(mean + 32);      // [32][ldx + 8]
    if (*status) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const size_t p0 = blk * 32;
    const size_t p = p0 + lane;
    const bool ok = p < nx;
    // FP32 states: slice sums in floats [0, 256) of `part`, x_ref and the mean
    // offset per lane in floats [256, 320)
    float *rfm = reinterpret_cast<float *>(part) + 256;
    if constexpr (std::is_same<T, float>::value) {
        // FP32 states: the mean as x_ref + dm, x_ref = member 0's value at the
        // point and dm the mean of the differences x_i - x_ref.  Members at a
        // point lie within a small spread of each other, so the differences
        // are exact (Sterbenz) and their FP32 sum carries an error of order
        // 2^-24 of the spread, not of the state.  Slice q (members q, q + 8,
        // ...) is summed in member order, the 8 slices in slice order (the
        // tensor-core update forms its anomalies with these same operations).
        const float xr = ok ? (float)m[p] : 0.f;
        float ps = 0.f;
        if (ok)
            for (int i = wp; i < ne; i += 8) ps = __fadd_rn(ps, __fsub_rn((float)m[(size_t)i * nx + p], xr));
        float *partf = reinterpret_cast<float *>(part);
        partf[wp * 32 + lane] = ps;
        __syncthreads();
        if (wp == 0) {
            float D = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) D = __fadd_rn(D, partf[q * 32 + lane]);
            const float dm = __fmul_rn(D, (float)inv_ne);
            rfm[lane] = xr;
            rfm[32 + lane] = dm;
            mean[lane] = (double)xr + (double)dm;
        }
    } else {
        double acc = 0.0;
        if (ok)
            for (int i = wp; i < ne; i += 8) acc += (double)m[(size_t)i * nx + p];
        part[wp * 32 + lane] = acc;
        __syncthreads();
        if (wp == 0) {
            double sum = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) sum += part[q * 32 + lane];
            mean[lane] = sum * inv_ne;
        }
    }
    __syncthreads();
    const double xb = mean[lane];
    const int ldt = ldx + 8;
    if (X64) {
        if (ok)
            for (int i = wp; i < ne; i += 8) X64[(size_t)i * nx + p] = ((double)m[(size_t)i * nx + p] - xb) * isq;
        return;
    }
    // BF16 path (FP32 states): FP32 centring on the exact differences,
    // ((x_i - x_ref) - dm) / sqrt(Ne - 1), then BF16 rounding (2^-9 of the
    // anomaly, far above the FP32 errors of the centring)
    const float isqf = (float)isq, xr = rfm[lane], dm = rfm[32 + lane];
    for (int i = wp; i < ldx; i += 8)
        tile[lane * ldt + i] = __float2bfloat16(
            (ok && i < ne) ? __fmul_rn(__fsub_rn(__fsub_rn((float)m[(size_t)i * nx + p], xr), dm), isqf) : 0.f);
    __syncthreads();
    // store: row r of the tile (point p0 + r) is ldx bf16 = ldx/8 16-byte chunks
    const int chunks = ldx / 8;
    for (int e = threadIdx.x; e < 32 * chunks; e += blockDim.x) {
        const int r = e / chunks, cidx = e % chunks;
        if (p0 + r < nx)
            reinterpret_cast<uint4 *>(X16 + (p0 + r) * ldx)[cidx] =
                reinterpret_cast<const uint4 *>(tile + r * ldt)[cidx];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_ens_anom(const T *__restrict__ m, size_t nx, int ne, double inv_ne,
                                                  double isq, double *__restrict__ X64,
                                                  __nv_bfloat16 *__restrict__ X16, int ldx, const int *status) {
    ens_anom_body<T>(m, nx, ne, inv_ne, isq, X64, X16, ldx, status, blockIdx.x);
}

// dynamic shared memory of the anomaly kernel for BF16 rows of ldx values
static size_t ens_anom_smem(int ldx) {
    return sizeof(double) * 9 * 32 + sizeof(__nv_bfloat16) * 32 * (size_t)(ldx + 8);
}

template <typename T>
void launch_ens_anom(const T *members, size_t nx, int ne, double *X64, __nv_bfloat16 *X16,
                     const int *status, cudaStream_t s) {
    count_launches(1);
    const int ldx = (ne + 15) / 16 * 16;
    const size_t smem = ens_anom_smem(ldx);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_ens_anom<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ens_anom<T><<<ceil_div(nx, 32), 256, smem, s>>>(members, nx, ne, 1.0 / ne, 1.0 / std::sqrt((double)(ne - 1)),
                                                       X64, X16, ldx, status);
}

// ---------------------------------------------------------------------------
// FP64 GEMMs of the gain (Algorithm 3 step 8)
// ---------------------------------------------------------------------------
// [out1 | out2^T] = A [B1; B2]^T / divisor (+ diag on out1's diagonal), FP64.
// One 16 x 16 output tile per CTA of 256 threads, one output per thread, k in
// chunks of 32 staged in shared memory; the next chunk's loads are issued
// before the current chunk's FMAs, so they are in flight while GB300's slow
// FP64 pipe works.  When B1 is A and n1 = m, out1 = A A^T / divisor + diag I is
// symmetric: tiles strictly below its diagonal are not computed (a quarter of
// the FMAs of S = I + Y^T R^-1 Y [Y | D | d*]), their values are the mirror
// of the tiles above (the same products, so the same bits).
__device__ __forceinline__ double gemm_nt_tile(const double *__restrict__ A, int m, const double *__restrict__ B1,
                                               int n1, const double *__restrict__ B2, int n2, int K, int kb,
                                               int ke, int a0, int c0, double (&As)[16][33],
                                               double (&Bs)[16][33]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const double *arow[2], *brow[2];
    int rr[2], kq[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int e = threadIdx.x + 256 * q;
        rr[q] = e >> 5;
        kq[q] = e & 31;
        const int a = a0 + rr[q], c = c0 + rr[q];
        arow[q] = a < m ? A + (size_t)a * K : nullptr;
        brow[q] = c < n1 ? B1 + (size_t)c * K : (c < n1 + n2 ? B2 + (size_t)(c - n1) * K : nullptr);
    }
    double va[2], vb[2];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = k0 + kq[q];
            va[q] = (arow[q] && k < ke) ? arow[q][k] : 0.0;
            vb[q] = (brow[q] && k < ke) ? brow[q][k] : 0.0;
        }
    };
    fetch(kb);
    double acc = 0.0;
    for (int k0 = kb; k0 < ke; k0 += 32) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            As[rr[q]][kq[q]] = va[q];
            Bs[rr[q]][kq[q]] = vb[q];
        }
        __syncthreads();
        if (k0 + 32 < ke) fetch(k0 + 32);
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) acc = fma(As[ty][kk], Bs[tx][kk], acc);
        __syncthreads();
    }
    return acc;
}

// Output tile (bx, by) of [out1 | out2^T]: over the whole of K with the
// epilogue (part == NULL), or over K chunk bz into the split-K partial sums.
__device__ __forceinline__ void gemm_nt_block(const double *__restrict__ A, int m, const double *__restrict__ B1,
                                              int n1, const double *__restrict__ B2, int n2, int K, double divisor,
                                              double diag, double *__restrict__ out1, double *__restrict__ out2,
                                              int bx, int by, int bz, int kchunk, double *__restrict__ part) {
    const bool sym = B1 == A && n1 == m;
    if (sym && bx < by) return;  // mirrored from tile (by, bx) (by the reduce when split)
    __shared__ double As[16][33];
    __shared__ double Bs[16][33];
    const int a0 = by * 16, c0 = bx * 16;
    const int kb = part ? bz * kchunk : 0, ke = part ? min(K, kb + kchunk) : K;
    const double acc = gemm_nt_tile(A, m, B1, n1, B2, n2, K, kb, ke, a0, c0, As, Bs);
    const int a = a0 + (threadIdx.x >> 4), c = c0 + (threadIdx.x & 15);
    if (part) {
        if (a < m && c < n1 + n2) part[((size_t)bz * m + a) * (n1 + n2) + c] = acc;
        return;
    }
    if (a < m) {
        if (c < n1) {
            out1[(size_t)a * n1 + c] = (a == c ? diag : 0.0) + acc / divisor;
            if (sym && bx > by) out1[(size_t)c * n1 + a] = acc / divisor;
        } else if (c < n1 + n2) {
            out2[(size_t)(c - n1) * m + a] = acc / divisor;
        }
    }
}

__global__ void k_gemm_nt(const double *__restrict__ A, int m, const double *__restrict__ B1, int n1,
                          const double *__restrict__ B2, int n2, int K, double divisor, double diag,
                          double *__restrict__ out1, double *__restrict__ out2, const int *status) {
    if (status && *status) return;
    gemm_nt_block(A, m, B1, n1, B2, n2, K, divisor, diag, out1, out2, blockIdx.x, blockIdx.y, 0, K, nullptr);
}

// Partial sums of k_gemm_nt over K chunks (split-K), combined in chunk order.
__global__ void k_gemm_nt_split(const double *__restrict__ A, int m, const double *__restrict__ B1,
                                int n1, const double *__restrict__ B2, int n2, int K, int kchunk,
                                double *__restrict__ part, const int *status) {
    if (status && *status) return;
    gemm_nt_block(A, m, B1, n1, B2, n2, K, 1.0, 0.0, nullptr, nullptr, blockIdx.x, blockIdx.y, blockIdx.z, kchunk,
                  part);
}

__device__ __forceinline__ void gemm_nt_reduce_body(const double *__restrict__ part, int nsplit, int m, int n1,
                                                    int n2, bool sym, double divisor, double diag,
                                                    double *__restrict__ out1, double *__restrict__ out2, int blk,
                                                    int nblk) {
    const int ncol = n1 + n2;
    for (int e = blk * blockDim.x + threadIdx.x; e < m * ncol; e += nblk * blockDim.x) {
        const int a = e / ncol, c = e % ncol;
        // below the diagonal tiles of a symmetric out1: the mirrored element
        const bool mirror = sym && c < n1 && (c >> 4) < (a >> 4);
        const int ra = mirror ? c : a, rc = mirror ? a : c;
        double acc = 0.0;
        for (int z = 0; z < nsplit; ++z) acc += part[((size_t)z * m + ra) * ncol + rc];
        if (c < n1)
            out1[(size_t)a * n1 + c] = (a == c ? diag : 0.0) + acc / divisor;
        else
            out2[(size_t)(c - n1) * m + a] = acc / divisor;
    }
}

__global__ void k_gemm_nt_reduce(const double *__restrict__ part, int nsplit, int m, int n1, int n2, bool sym,
                                 double divisor, double diag, double *__restrict__ out1,
                                 double *__restrict__ out2, const int *status) {
    if (status && *status) return;
    gemm_nt_reduce_body(part, nsplit, m, n1, n2, sym, divisor, diag, out1, out2, blockIdx.x, gridDim.x);
}

int gemm_nt_splits(int m, int n1, int n2, int K) {
    const int tiles = ceil_div(n1 + n2, 16) * ceil_div(m, 16);
    int splits = 1;
    while (tiles * splits * 2 <= 2 * kNumSMs && K / (splits * 2) >= 128) splits *= 2;
    return splits;
}

// ---------------------------------------------------------------------------
// The gain products of the mixed path in double-FP32 arithmetic on the FP32
// pipes (GB300 runs FP32 FMAs about 64 times faster than FP64 ones): each FP64
// operand is a pair hi + lo of FP32 values (split_df); a b = ah bh + ah bl +
// al bh (+ al bl, below 2^-48 |a b|, dropped), ah bh exactly as p + e with
// e = fma(ah, bh, -p); the products are summed into a running FP32 sum s and
// the FP32 sum c of its rounding errors (error-free two-sum) and of the small
// terms.  The result s + c carries a relative error of order 2^-44 of the sum
// of |a b|, far below the BF16 rounding of T that follows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &s, float &c) {
    const float p = __fmul_rn(ah, bh);
    const float e = __fmaf_rn(ah, bh, -p);
    const float x = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
    const float t = __fadd_rn(s, p), bv = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv)), x));
    s = t;
}

constexpr int kDfThreads = 64;  // a 16 x 16 output tile, 2 x 2 outputs per thread
constexpr int kDfK = 32;        // K chunk staged in shared memory

// Output tile (bx, by) of [S | Y^T R^-1 [D | d*]] as gemm_nt_block (A = B1 = Y,
// m = n1 = ne, B2 = Z, n2 = ne + 1, symmetric S: tiles with bx < by are not
// computed), from the double-FP32 operands.
__device__ __forceinline__ void gemm_df_block(const DfOperands &df, int ne, int K, double divisor, double diag,
                                              double *__restrict__ out1, double *__restrict__ out2, int bx, int by,
                                              int bz, int kchunk, double *__restrict__ part) {
    if (bx < by) return;
    __shared__ float sAh[16][kDfK + 1], sAl[16][kDfK + 1], sBh[16][kDfK + 1], sBl[16][kDfK + 1];
    const int m = ne, n1 = ne, n2 = ne + 1;
    const int a0 = by * 16, c0 = bx * 16;
    const int kb = part ? bz * kchunk : 0, ke = part ? min(K, kb + kchunk) : K;
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    // staging: row tid / 4 of the A and B tiles, k = (tid mod 4) * 8 .. + 7 of the chunk
    const int sr = tid >> 2, sk = (tid & 3) * 8;
    const int ar = a0 + sr, cr = c0 + sr;
    const float *ah = ar < m ? df.Yh + (size_t)ar * K : nullptr, *al = ar < m ? df.Yl + (size_t)ar * K : nullptr;
    const float *bh = cr < n1 ? df.Yh + (size_t)cr * K : (cr < n1 + n2 ? df.Zh + (size_t)(cr - n1) * K : nullptr);
    const float *bl = cr < n1 ? df.Yl + (size_t)cr * K : (cr < n1 + n2 ? df.Zl + (size_t)(cr - n1) * K : nullptr);
    float va[2][8], vb[2][8];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + sk + j;
            const bool ok = k < ke;
            va[0][j] = (ah && ok) ? ah[k] : 0.f;
            va[1][j] = (al && ok) ? al[k] : 0.f;
            vb[0][j] = (bh && ok) ? bh[k] : 0.f;
            vb[1][j] = (bl && ok) ? bl[k] : 0.f;
        }
    };
    float s[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, c[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    fetch(kb);
    for (int k0 = kb; k0 < ke; k0 += kDfK) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sAh[sr][sk + j] = va[0][j];
            sAl[sr][sk + j] = va[1][j];
            sBh[sr][sk + j] = vb[0][j];
            sBl[sr][sk + j] = vb[1][j];
        }
        __syncthreads();
        if (k0 + kDfK < ke) fetch(k0 + kDfK);  // in flight during the chunk's products
#pragma unroll 4
        for (int kk = 0; kk < kDfK; ++kk) {
            float xh[2], xl[2], yh[2], yl[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                xh[i] = sAh[2 * ty + i][kk];
                xl[i] = sAl[2 * ty + i][kk];
                yh[i] = sBh[2 * tx + i][kk];
                yl[i] = sBl[2 * tx + i][kk];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) df_mac(xh[i], xl[i], yh[j], yl[j], s[i][j], c[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int a = a0 + 2 * ty + i, cc = c0 + 2 * tx + j;
            const double acc = (double)s[i][j] + (double)c[i][j];
            if (part) {
                if (a < m && cc < n1 + n2) part[((size_t)bz * m + a) * (n1 + n2) + cc] = acc;
                continue;
            }
            if (a < m) {
                if (cc < n1) {
                    out1[(size_t)a * n1 + cc] = (a == cc ? diag : 0.0) + acc / divisor;
                    if (bx > by) out1[(size_t)cc * n1 + a] = acc / divisor;
                } else if (cc < n1 + n2) {
                    out2[(size_t)(cc - n1) * m + a] = acc / divisor;
                }
            }
        }
}

__global__ void __launch_bounds__(kDfThreads) k_gemm_df(DfOperands df, int ne, int K, double divisor, double diag,
                                                        double *__restrict__ out1, double *__restrict__ out2,
                                                        int kchunk, double *__restrict__ part, const int *status) {
    if (*status) return;
    gemm_df_block(df, ne, K, divisor, diag, out1, out2, blockIdx.x, blockIdx.y, blockIdx.z, kchunk, part);
}

void launch_gemm_df(const DfOperands &df, int ne, int ny, double s2, double *S, double *Bt, const int *status,
                    cudaStream_t s, double *part) {
    const int splits = part ? gemm_nt_splits(ne, ne, ne + 1, ny) : 1;
    const int kchunk = ceil_div(ceil_div(ny, splits), 32) * 32;
    dim3 grid(ceil_div(2 * ne + 1, 16), ceil_div(ne, 16), splits);
    count_launches(splits > 1 ? 2 : 1);
    k_gemm_df<<<grid, kDfThreads, 0, s>>>(df, ne, ny, s2, 1.0, S, Bt, kchunk, splits > 1 ? part : nullptr, status);
    if (splits > 1)
        k_gemm_nt_reduce<<<grid_for((size_t)ne * (2 * ne + 1), 256), 256, 0, s>>>(part, splits, ne, ne, ne + 1, true,
                                                                                s2, 1.0, S, Bt, status);
}

void launch_gemm_nt_f64(const double *A, int m, const double *B1, int n1, const double *B2, int n2,
                        int K, double scale_div, double diag, double *out1, double *out2,
                        const int *status, cudaStream_t s, double *part) {
    const int splits = part ? gemm_nt_splits(m, n1, n2, K) : 1;
    if (splits > 1) {
        count_launches(2);
        const int kchunk = ceil_div(ceil_div(K, splits), 32) * 32;
        dim3 grid(ceil_div(n1 + n2, 16), ceil_div(m, 16), splits);
        k_gemm_nt_split<<<grid, 256, 0, s>>>(A, m, B1, n1, B2, n2, K, kchunk, part, status);
        k_gemm_nt_reduce<<<grid_for((size_t)m * (n1 + n2), 256), 256, 0, s>>>(
            part, splits, m, n1, n2, B1 == A && n1 == m, scale_div, diag, out1, out2, status);
        return;
    }
    count_launches(1);
    dim3 grid(ceil_div(n1 + n2, 16), ceil_div(m, 16));
    k_gemm_nt<<<grid, 256, 0, s>>>(A, m, B1, n1, B2, n2, K, scale_div, diag, out1, out2, status);
}

__global__ void k_gemm_tn(const double *__restrict__ Y, int ne, int ny, double diag,
                          double *__restrict__ C, const int *status) {
    if (*status) return;
    __shared__ double As[32][17];
    __shared__ double Bs[32][17];
    const int j0 = blockIdx.y * 16, l0 = blockIdx.x * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc = 0.0;
    for (int k0 = 0; k0 < ne; k0 += 32) {
        for (int e = threadIdx.x; e < 32 * 16; e += 256) {
            const int kk = e >> 4, r = e & 15, k = k0 + kk;
            As[kk][r] = (k < ne && j0 + r < ny) ? Y[(size_t)k * ny + j0 + r] : 0.0;
            Bs[kk][r] = (k < ne && l0 + r < ny) ? Y[(size_t)k * ny + l0 + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) acc = fma(As[kk][ty], Bs[kk][tx], acc);
        __syncthreads();
    }
    const int j = j0 + ty, l = l0 + tx;
    if (j < ny && l < ny) C[(size_t)j * ny + l] = acc + (j == l ? diag : 0.0);
}

void launch_gemm_tn_f64(const double *Y, int ne, int ny, double diag, double *C, const int *status,
                        cudaStream_t s) {
    count_launches(1);
    dim3 grid(ceil_div(ny, 16), ceil_div(ny, 16));
    k_gemm_tn<<<grid, 256, 0, s>>>(Y, ne, ny, diag, C, status);
}

// ---------------------------------------------------------------------------
// Cholesky (right-looking, one CTA) and the two triangular solves
// ---------------------------------------------------------------------------
template <bool SMEM>
__device__ __forceinline__ void cholesky_body(double *A, double *Lt, int n, int *status) {
    // Right-looking Cholesky by one CTA.  Column k: pivot l = sqrt(A_kk) and its
    // reciprocal (one division per column), scale the column below it, then the
    // rank-1 update of the trailing lower triangle.  Rows padded to n+1 doubles
    // in shared memory.
    extern __shared__ double sm[];
    __shared__ double s_inv;
    if (*status) return;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int tx = tid & 31, ty = tid >> 5, nty = nth >> 5;
    const int ld = SMEM ? n + 1 : n;
    double *M = SMEM ? sm : A;
    if (SMEM) {
        for (int e = tid; e < n * n; e += nth) sm[(e / n) * ld + e % n] = A[e];
        __syncthreads();
    }
    for (int k = 0; k < n; ++k) {
        const double d = M[(size_t)k * ld + k];
        if (!(d > 0.0) || !isfinite(d)) {  // uniform: every thread read the same pivot
            if (tid == 0) atomicCAS(status, 0, kStNotSpd);
            return;
        }
        __syncthreads();  // every thread has read the pivot before it is overwritten
        if (tid == 0) {
            const double l = sqrt(d);
            M[(size_t)k * ld + k] = l;
            s_inv = 1.0 / l;
        }
        __syncthreads();
        const double inv = s_inv;
        for (int i = k + 1 + tid; i < n; i += nth) M[(size_t)i * ld + k] *= inv;
        __syncthreads();
        for (int i = k + 1 + ty; i < n; i += nty) {
            const double lik = M[(size_t)i * ld + k];
            for (int j = k + 1 + tx; j <= i; j += 32)
                M[(size_t)i * ld + j] = fma(-lik, M[(size_t)j * ld + k], M[(size_t)i * ld + j]);
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += nth) {
        const int i = e / n, j = e % n;
        const double val = j <= i ? M[(size_t)i * ld + j] : 0.0;
        A[e] = val;
        Lt[(size_t)j * n + i] = val;
    }
}

template <bool SMEM>
__global__ void __launch_bounds__(256) k_cholesky(double *A, double *Lt, int n, int *status) {
    cholesky_body<SMEM>(A, Lt, n, status);
}

// Cholesky by a cluster of 8 CTAs (n <= 256).  CTA q owns the columns
// [q w, q w + w), w = ceil(n / 8), all n rows, in shared memory.  Panel p is
// CTA p's block of columns.  For p = 0 .. 7: CTA p factors its panel column by
// column (pivot sqrt and one reciprocal, scale the column, rank-1 update of
// the panel's remaining columns; a ninth warp updates the next diagonal entry
// and forms its pivot while the eight others update the rest, so the pivot's
// FP64 chain is off the update's path); cluster barrier; every CTA q > p copies the
// rows >= q w of panel p from CTA p's shared memory (distributed shared
// memory) and subtracts the panel's rank-w product from its own columns.  One
// cluster barrier per panel; the FP64 work of the trailing updates spreads
// over 8 SMs.  A non-positive pivot sets the status and the kernel runs to
// the end (every CTA must reach every cluster barrier) without writing L.
constexpr int kCholCluster = 8;

// y = 1/sqrt(d) for a Cholesky pivot: FP32 rsqrtf seed, then two Newton steps
// y <- y (3 - d y^2) / 2 in FP64 (each squares the relative error: 2^-23 ->
// 2^-46 -> FP64 rounding).  A pivot that is not positive and finite sets the
// status and yields y = 1 so the factorisation runs on without dividing.
__device__ __forceinline__ void chol_pivot(double d, double *y_out, int *status, int *fail) {
    if (!(d > 0.0) || !isfinite(d)) {
        atomicCAS(status, 0, kStNotSpd);
        *fail = 1;
        *y_out = 1.0;
        return;
    }
    double y;
    if (d > 1e-30 && d < 1e30) {
        y = (double)rsqrtf((float)d);
        y = y * fma(-0.5 * d, y * y, 1.5);
        y = y * fma(-0.5 * d, y * y, 1.5);
    } else {
        y = 1.0 / sqrt(d);
    }
    *y_out = y;
}

__device__ __forceinline__ void cholesky_cluster_body(double *A, double *Lt, int n, int *status) {
    extern __shared__ double csm[];
    __shared__ int s_fail;
    __shared__ double s_y[32];  // 1/sqrt of the panel's pivots
    cg::cluster_group cl = cg::this_cluster();
    if (*status) return;  // every CTA reads it before any CTA can write it (after the first barrier)
    const int q = (int)cl.block_rank();
    const int w = (n + kCholCluster - 1) / kCholCluster, ldp = w + 1;
    const int c0 = q * w, c1 = min(n, c0 + w), wq = max(0, c1 - c0);
    const int tid = threadIdx.x, nth = blockDim.x;
    // 2-D view of the CTA for column-parallel loops: nx2 column lanes x ny2 row lanes
    const int nupd = 256, kPiv = 256;  // threads [0, 256) update, thread 256 forms the pivots
    const int nx2 = w <= 8 ? 8 : (w <= 16 ? 16 : 32), ny2 = nupd / nx2;
    const int tx2 = tid % nx2, ty2 = tid / nx2;
    double *P = csm;             // [n][ldp]: rows of this CTA's columns
    double *Lp = csm + n * ldp;  // [n][ldp]: copy of the panel being applied
    if (tid == 0) s_fail = 0;
    for (int e = tid; e < n * wq; e += nth) {
        const int i = e / wq, c = e - i * wq;
        P[i * ldp + c] = A[(size_t)i * n + c0 + c];
    }
    cl.sync();
    for (int p = 0; p < kCholCluster; ++p) {
        const int pc0 = p * w, wp = min(n, pc0 + w) - pc0;
        if (wp <= 0) break;  // the same for every CTA
        if (q == p) {
            // Outer-product form on unscaled columns: with d_k the pivot,
            // A_ij -= A_ik A_jk / d_k for the panel's later columns, one barrier
            // per column.  The thread that updates the next diagonal entry
            // (thread 0) forms that pivot's 1/sqrt(d) at once; the square roots
            // and column scalings follow once per panel.
            __syncthreads();
            if (tid == kPiv) chol_pivot(P[pc0 * ldp], &s_y[0], status, &s_fail);
            for (int c = 0; c < wp; ++c) {
                const int k = pc0 + c;
                __syncthreads();
                const double y = s_y[c], idk = y * y;
                if (tid < nupd) {
                    // thread (tx, ty): panel column c + 1 + tx, rows k + 1 + ty, + ny, ... (rows >= that column)
                    const int cc = c + 1 + tx2;
                    if (cc < wp) {
                        const int r = pc0 + cc;
                        const double ljk = P[r * ldp + c] * idk;
                        for (int ii = k + 1 + ty2; ii < n; ii += ny2)
                            if (ii > r || (ii == r && cc != c + 1)) P[ii * ldp + cc] = fma(-P[ii * ldp + c], ljk, P[ii * ldp + cc]);
                    }
                } else if (tid == kPiv && c + 1 < wp) {
                    // the next diagonal entry, updated here, and its pivot
                    const int r = k + 1;
                    const double ljk = P[r * ldp + c] * idk;
                    const double dn = fma(-P[r * ldp + c], ljk, P[r * ldp + c + 1]);
                    P[r * ldp + c + 1] = dn;
                    chol_pivot(dn, &s_y[c + 1], status, &s_fail);
                }
            }
            __syncthreads();
            // L_ik = A_ik / sqrt(d_k) below the diagonal, L_kk = sqrt(d_k) = d_k y_k
            for (int e = tid; e < n * wp; e += nth) {
                const int i = e / wp, c = e - i * wp, k = pc0 + c;
                if (i > k) P[i * ldp + c] *= s_y[c];
            }
            __syncthreads();
            for (int c = tid; c < wp; c += nth) {
                const int k = pc0 + c;
                const double d = P[k * ldp + c];
                P[k * ldp + c] = (d > 0.0 && isfinite(d)) ? d * s_y[c] : 1.0;
            }
        }
        cl.sync();
        if (q > p && wq > 0) {
            const double *rp = cl.map_shared_rank(P, p);
            for (int e = tid; e < (n - c0) * wp; e += nth) {
                const int i = c0 + e / wp, c = e % wp;
                Lp[i * ldp + c] = rp[i * ldp + c];
            }
            __syncthreads();
            // thread (tx, ty): own column jj = tx, tx + nx2, ...; rows j + ty, + ny2, ...
            for (int jj = tx2; tid < nupd && jj < wq; jj += nx2) {
                const int j = c0 + jj;
                for (int i = j + ty2; i < n; i += ny2) {
                    double acc = P[i * ldp + jj];
                    for (int c = 0; c < wp; ++c) acc = fma(-Lp[i * ldp + c], Lp[j * ldp + c], acc);
                    P[i * ldp + jj] = acc;
                }
            }
        }
    }
    __syncthreads();
    if (!s_fail && !*status) {
        for (int e = tid; e < n * wq; e += nth) {
            const int i = e / wq, c = e - i * wq, j = c0 + c;
            const double val = i >= j ? P[i * ldp + c] : 0.0;
            A[(size_t)i * n + j] = val;
            Lt[(size_t)j * n + i] = val;
        }
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

__global__ void __cluster_dims__(kCholCluster, 1, 1) __launch_bounds__(288)
    k_cholesky_cluster(double *A, double *Lt, int n, int *status) {
    cholesky_cluster_body(A, Lt, n, status);
}

// dynamic shared memory of the clustered Cholesky of order n
static size_t cholesky_cluster_smem(int n) {
    return sizeof(double) * 2 * (size_t)n * ((n + kCholCluster - 1) / kCholCluster + 1);
}

void launch_cholesky(double *A, double *Lt, int n, int *status, cudaStream_t s) {
    count_launches(1);
    if (n >= 32 && n <= 256) {
        const size_t bytes = cholesky_cluster_smem(n);
        static OncePerDevice attr;
        attr.run([](int) {
            return cudaFuncSetAttribute(k_cholesky_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        });
        k_cholesky_cluster<<<kCholCluster, 288, bytes, s>>>(A, Lt, n, status);
        return;
    }
    const size_t bytes = sizeof(double) * (size_t)n * (n + 1);
    if (bytes <= 210 * 1024) {
        static OncePerDevice attr;
        attr.run([](int) {
            return cudaFuncSetAttribute(k_cholesky<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
        });
        k_cholesky<true><<<1, 256, bytes, s>>>(A, Lt, n, status);
    } else {
        k_cholesky<false><<<1, 256, 0, s>>>(A, Lt, n, status);
    }
}

// Triangular solves with the factor staged in shared memory: one warp per
// right-hand side, lanes own rows lane + 32 m.  A CTA solves the columns
// c0 .. c0 + ncols - 1 (warp w: column c0 + w): one column per CTA spreads the
// FP64 work of one problem's columns over the SMs; the grouped analysis of many
// problems gives each CTA several columns, so the factor is staged once for them.
template <int MAXR>
__device__ __forceinline__ void chol_solve_body(const double *__restrict__ L, int n, const double *rhs, double *out,
                                                int ncol, __nv_bfloat16 *out16, int ld16, const int *status, int c0,
                                                int ncols) {
    // the CTA stages the unit lower factor U = L D^-1 (D = diag L) in shared
    // memory, then each solving warp runs both substitutions for its
    // right-hand side: S x = U D^2 U^T x = b as U y = b, then U^T x = D^-2 y.
    // With the unit diagonal no step of either substitution waits on an FP64
    // multiplication before its broadcast.
    extern __shared__ double sL[];  // [n][n+1]: U strictly below the diagonal; then inv_diag[n]
    if (*status) return;
    const int c = c0 + (threadIdx.x >> 5), lane = threadIdx.x & 31, ld = n + 1;
    double *inv = sL + (size_t)n * ld;
    for (int j = threadIdx.x; j < n; j += blockDim.x) inv[j] = 1.0 / L[(size_t)j * n + j];
    __syncthreads();
    for (int i = threadIdx.x >> 5; i < n; i += blockDim.x >> 5)
        for (int j = lane; j < i; j += 32) sL[(size_t)i * ld + j] = L[(size_t)i * n + j] * inv[j];
    __syncthreads();
    if ((threadIdx.x >> 5) >= ncols || c >= ncol) return;
    double b[MAXR];
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
        const int i = lane + 32 * m;
        b[m] = i < n ? rhs[(size_t)c * n + i] : 0.0;
    }
    // forward, column by column: y_j is final once the columns before j are applied
#pragma unroll
    for (int s = 0; s < MAXR; ++s) {
        if (s * 32 >= n) break;
        for (int l = 0; l < 32; ++l) {
            const int j = s * 32 + l;
            if (j >= n) break;
            const double yj = __shfl_sync(0xffffffffu, b[s], l);
#pragma unroll
            for (int m = s; m < MAXR; ++m) {
                const int i = lane + 32 * m;
                if (i > j && i < n) b[m] = fma(-sL[(size_t)i * ld + j], yj, b[m]);
            }
        }
    }
    // right-hand side of the backward substitution: D^-2 y
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
        const int i = lane + 32 * m;
        if (i < n) b[m] *= inv[i] * inv[i];
    }
#pragma unroll
    for (int s = MAXR - 1; s >= 0; --s) {
        if (s * 32 >= n) continue;
        for (int l = 31; l >= 0; --l) {
            const int j = s * 32 + l;
            if (j >= n) continue;
            const double xj = __shfl_sync(0xffffffffu, b[s], l);
#pragma unroll
            for (int m = 0; m <= s; ++m) {
                const int i = lane + 32 * m;
                if (i < j) b[m] = fma(-sL[(size_t)j * ld + i], xj, b[m]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
        const int i = lane + 32 * m;
        if (i < n) {
            out[(size_t)c * n + i] = b[m];
            if (out16) out16[(size_t)c * ld16 + i] = __double2bfloat16(b[m]);
        }
    }
}

template <int MAXR>
__global__ void __launch_bounds__(256) k_chol_solve_smem(const double *__restrict__ L, int n, const double *rhs,
                                                         double *out, int ncol, __nv_bfloat16 *out16, int ld16,
                                                         const int *status) {
    chol_solve_body<MAXR>(L, n, rhs, out, ncol, out16, ld16, status, blockIdx.x, 1);
}

// shared memory of the staged factor of order n
static size_t chol_solve_smem(int n) { return sizeof(double) * ((size_t)n * (n + 1) + n); }

template <int MAXR>
__global__ void __launch_bounds__(32) k_chol_solve(const double *__restrict__ L,
                                                   const double *__restrict__ Lt, int n,
                                                   const double *rhs, double *out, int ncol,
                                                   __nv_bfloat16 *out16, int ld16,
                                                   const int *status) {
    if (*status) return;
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    if (c >= ncol) return;
    double b[MAXR];
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
        const int i = lane + 32 * m;
        b[m] = i < n ? rhs[(size_t)c * n + i] : 0.0;
    }
    // forward substitution L z = b (column-oriented: after z_j, b_i -= L_ij z_j)
#pragma unroll
    for (int s = 0; s < MAXR; ++s) {
        if (s * 32 >= n) break;
        for (int l = 0; l < 32; ++l) {
            const int j = s * 32 + l;
            if (j >= n) break;
            if (lane == l) b[s] = b[s] / L[(size_t)j * n + j];
            const double zj = __shfl_sync(0xffffffffu, b[s], l);
#pragma unroll
            for (int m = s; m < MAXR; ++m) {
                const int i = lane + 32 * m;
                if (i > j && i < n) b[m] = fma(-Lt[(size_t)j * n + i], zj, b[m]);
            }
        }
    }
    // back substitution L^T x = z (after x_j, z_i -= L_ji x_j for i < j)
#pragma unroll
    for (int s = MAXR - 1; s >= 0; --s) {
        if (s * 32 >= n) continue;
        for (int l = 31; l >= 0; --l) {
            const int j = s * 32 + l;
            if (j >= n) continue;
            if (lane == l) b[s] = b[s] / L[(size_t)j * n + j];
            const double xj = __shfl_sync(0xffffffffu, b[s], l);
#pragma unroll
            for (int m = 0; m <= s; ++m) {
                const int i = lane + 32 * m;
                if (i < j) b[m] = fma(-L[(size_t)j * n + i], xj, b[m]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
        const int i = lane + 32 * m;
        if (i < n) {
            out[(size_t)c * n + i] = b[m];
            if (out16) out16[(size_t)c * ld16 + i] = __double2bfloat16(b[m]);
        }
    }
}

void launch_chol_solve(const double *L, const double *Lt, int n, const double *rhs, double *out,
                       int ncol, __nv_bfloat16 *out16, int ld16, const int *status, cudaStream_t s) {
    count_launches(1);
    const size_t smem = chol_solve_smem(n);
    if (n <= 160 && smem <= 210 * 1024) {
        static OncePerDevice attr[2];
        if (n <= 128) {
            attr[0].run([](int) {
                return cudaFuncSetAttribute(k_chol_solve_smem<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            210 * 1024);
            });
            k_chol_solve_smem<4><<<ncol, 256, smem, s>>>(L, n, rhs, out, ncol, out16, ld16, status);
        } else {
            attr[1].run([](int) {
                return cudaFuncSetAttribute(k_chol_solve_smem<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            210 * 1024);
            });
            k_chol_solve_smem<8><<<ncol, 256, smem, s>>>(L, n, rhs, out, ncol, out16, ld16, status);
        }
        return;
    }
    if (n <= 128)
        k_chol_solve<4><<<ncol, 32, 0, s>>>(L, Lt, n, rhs, out, ncol, out16, ld16, status);
    else if (n <= 512)
        k_chol_solve<16><<<ncol, 32, 0, s>>>(L, Lt, n, rhs, out, ncol, out16, ld16, status);
    else
        k_chol_solve<64><<<ncol, 32, 0, s>>>(L, Lt, n, rhs, out, ncol, out16, ld16, status);
}

// ---------------------------------------------------------------------------
// member update x^a,(i) = x^f,(i) + X T_i and coarse correction dC = X T_ne
// (Eq. ensemble_update with K = X T; Algorithm 4 step 5)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_update_f64(T *__restrict__ members, T *__restrict__ dC,
                                                    const double *__restrict__ X,
                                                    const double *__restrict__ Tm, size_t nx, int ne,
                                                    const int *status) {
    extern __shared__ double Ts[];  // [32 columns][ne]
    if (*status) return;
    const int c0 = blockIdx.y * 32;
    for (int e = threadIdx.x; e < 32 * ne; e += blockDim.x) {
        const int cc = e / ne, a = e % ne;
        Ts[e] = c0 + cc <= ne ? Tm[(size_t)(c0 + cc) * ne + a] : 0.0;
    }
    __syncthreads();
    const size_t p = blockIdx.x * (size_t)64 + (threadIdx.x & 63);
    const int cg = threadIdx.x >> 6;
    if (p >= nx) return;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (int a = 0; a < ne; ++a) {
        const double x = X[(size_t)a * nx + p];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = fma(x, Ts[(cg * 8 + q) * ne + a], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = c0 + cg * 8 + q;
        if (c < ne)
            members[(size_t)c * nx + p] = (T)((double)members[(size_t)c * nx + p] + acc[q]);
        else if (c == ne)
            dC[p] = (T)acc[q];
    }
}

template <typename T>
void launch_update_f64(T *members, T *dC, const double *X, const double *Tm, size_t nx, int ne,
                       const int *status, cudaStream_t s) {
    count_launches(1);
    dim3 grid(ceil_div(nx, 64), ceil_div(ne + 1, 32));
    const size_t smem = sizeof(double) * 32 * (size_t)ne;  // <= 128 KB for ne <= 512
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_update_f64<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_update_f64<T><<<grid, 256, smem, s>>>(members, dC, X, Tm, nx, ne, status);
}

// BF16 anomaly product with FP32 accumulation (CUDA-core version): X^T tile of
// 64 points and T tile of 32 columns staged in shared memory.
__global__ void __launch_bounds__(256) k_update_bf16(float *__restrict__ members,
                                                     float *__restrict__ dC,
                                                     const __nv_bfloat16 *__restrict__ Xt,
                                                     const __nv_bfloat16 *__restrict__ Tt, int ldx,
                                                     size_t nx, int ne, const int *status) {
    extern __shared__ __nv_bfloat16 sm16[];
    if (*status) return;
    const int lds = ldx + 2;
    __nv_bfloat16 *Xs = sm16;             // [64][lds]
    __nv_bfloat16 *Tsm = sm16 + 64 * lds; // [32][lds]
    const size_t p0 = blockIdx.x * (size_t)64;
    const int c0 = blockIdx.y * 32;
    for (int e = threadIdx.x; e < 64 * ldx; e += blockDim.x) {
        const int r = e / ldx, a = e % ldx;
        Xs[r * lds + a] = p0 + r < nx ? Xt[(p0 + r) * ldx + a] : __float2bfloat16(0.f);
    }
    for (int e = threadIdx.x; e < 32 * ldx; e += blockDim.x) {
        const int r = e / ldx, a = e % ldx;
        Tsm[r * lds + a] = c0 + r <= ne ? Tt[(size_t)(c0 + r) * ldx + a] : __float2bfloat16(0.f);
    }
    __syncthreads();
    const int pl = threadIdx.x & 63, cg = threadIdx.x >> 6;
    const size_t p = p0 + pl;
    if (p >= nx) return;
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
    for (int a = 0; a < ne; ++a) {
        const float x = __bfloat162float(Xs[pl * lds + a]);
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = fmaf(x, __bfloat162float(Tsm[(cg * 8 + q) * lds + a]), acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = c0 + cg * 8 + q;
        if (c < ne)
            members[(size_t)c * nx + p] += acc[q];
        else if (c == ne)
            dC[p] = acc[q];
    }
}

void launch_update_bf16(float *members, float *dC, const __nv_bfloat16 *Xt, const __nv_bfloat16 *Tt,
                        int ldx, size_t nx, int ne, const int *status, cudaStream_t s) {
    count_launches(1);
    dim3 grid(ceil_div(nx, 64), ceil_div(ne + 1, 32));
    const size_t smem = sizeof(__nv_bfloat16) * (size_t)(64 + 32) * (ldx + 2);  // <= 99 KB
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_update_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_update_bf16<<<grid, 256, smem, s>>>(members, dC, Xt, Tt, ldx, nx, ne, status);
}

// ---------------------------------------------------------------------------
// prolongation of the coarse correction, Algorithm 4 step 5 second line
// ---------------------------------------------------------------------------
// a b + c rounded once, in the precision of T
template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c) {
    if constexpr (std::is_same<T, float>::value)
        return fmaf(a, b, c);
    else
        return fma(a, b, c);
}

// periodic index of a 4-point stencil tap: c in [-1, nc + 2)
__device__ __forceinline__ int wrap_tap(int c, int nc) {
    if (c < 0) c += nc;
    while (c >= nc) c -= nc;
    return c;
}

// fine (+)= Pi_F(dC): the 4-point Lagrange interpolant at fine offset m of
// coarse interval J (nodes J - 1 .. J + 2).  2-D is the tensor product,
// evaluated separably: four 4-tap sums along x, then one 4-tap sum along y.
// 2-D launch: x over the points of a fine row, y over the rows of all
// variables, so the only divisions are by r and the periodic wraps are
// compares.
// 2-D: fine column fx of the r fine rows of coarse interval Jy of variable v
// (vj = v nc + Jy).  The four sums along x (coarse rows Jy - 1 .. Jy + 2) are
// the same for the r rows and are formed once; each row is then its 4-tap sum
// along y.  The fine values of up to 4 rows are loaded before any of them is written.
// wt: the weights converted to T ([m][t], in shared memory).
template <typename T>
__device__ __forceinline__ void prolong2d_interval(T *__restrict__ fine, const T *__restrict__ dC, int nc, int r,
                                                   const T (*wt)[4], int fx, int vj) {
    const int nf = nc * r;
    const int v = vj / nc, Jy = vj - v * nc;
    const int Jx = fx / r, mx = fx - Jx * r;
    int cx[4];
    T wx[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        cx[t] = wrap_tap(Jx - 1 + t, nc);
        wx[t] = wt[mx][t];
    }
    const T *d = dC + (size_t)v * nc * nc;
    T sx[4];
#pragma unroll
    for (int ty = 0; ty < 4; ++ty) {
        const T *dr = d + (size_t)wrap_tap(Jy - 1 + ty, nc) * nc;
        T a = T(0);
#pragma unroll
        for (int tx = 0; tx < 4; ++tx) a = fma_t(wx[tx], dr[cx[tx]], a);
        sx[ty] = a;
    }
    T *f = fine + (size_t)v * nf * nf + (size_t)Jy * r * nf + fx;
    for (int m0 = 0; m0 < r; m0 += 4) {
        T old[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (m0 + k < r) old[k] = f[(size_t)(m0 + k) * nf];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (m0 + k < r) {
                T acc = T(0);
#pragma unroll
                for (int ty = 0; ty < 4; ++ty) acc = fma_t(wt[m0 + k][ty], sx[ty], acc);
                f[(size_t)(m0 + k) * nf] = old[k] + acc;
            }
    }
}

// the Lagrange weights of offsets 0 .. r - 1 converted to T, into shared memory
template <typename T>
__device__ __forceinline__ void prolong_stage_weights(const ProlongWeights &w, int r, T (*wt)[4]) {
    for (int e = threadIdx.x; e < 4 * r; e += blockDim.x) wt[e >> 2][e & 3] = (T)w.w[e >> 2][e & 3];
    __syncthreads();
}

template <typename T>
__global__ void k_prolong_add(T *__restrict__ fine, const T *__restrict__ dC, int dim, int V, int nc,
                              int r, ProlongWeights w, const int *status) {
    if (*status) return;
    const int nf = nc * r;
    if (dim == 1) {
        const size_t total = (size_t)V * nf;
        for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
             idx += (size_t)gridDim.x * blockDim.x) {
            const int v = (int)(idx / nf), k = (int)(idx - (size_t)v * nf);
            const T *d = dC + (size_t)v * nc;
            const int J = k / r, m = k - J * r;
            T acc = T(0);
#pragma unroll
            for (int t = 0; t < 4; ++t) acc += (T)w.w[m][t] * d[wrap_tap(J - 1 + t, nc)];
            fine[idx] += acc;
        }
        return;
    }
    __shared__ T wt[kMaxRatio][4];
    prolong_stage_weights<T>(w, r, wt);
    const int fx = blockIdx.x * blockDim.x + threadIdx.x;
    if (fx >= nf) return;
    for (int vj = blockIdx.y; vj < V * nc; vj += gridDim.y) prolong2d_interval<T>(fine, dC, nc, r, wt, fx, vj);
}

template <typename T>
void launch_prolong_add(T *fine, const T *dC, int dim, int V, int nc, int r,
                        const ProlongWeights &w, const int *status, cudaStream_t s) {
    count_launches(1);
    const int nf = nc * r;
    if (dim == 1) {
        k_prolong_add<T><<<grid_for((size_t)V * nf, 256), 256, 0, s>>>(fine, dC, dim, V, nc, r, w, status);
    } else {
        const dim3 grid(ceil_div(nf, 128), std::min(V * nc, 65535));
        k_prolong_add<T><<<grid, 128, 0, s>>>(fine, dC, dim, V, nc, r, w, status);
    }
}

// ---------------------------------------------------------------------------
// relative RMSE, Eq. L2norm_u (deterministic two-pass reduction)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_rmse_partial(const T *__restrict__ x, const double *__restrict__ truth, int V,
                               size_t npts, double *__restrict__ partials) {
    __shared__ double red[2][32];
    for (int v = 0; v < V; ++v) {
        double num = 0.0, den = 0.0;
        for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < npts;
             k += (size_t)gridDim.x * blockDim.x) {
            const double t = truth[v * npts + k];
            const double d = (double)x[v * npts + k] - t;
            num = fma(d, d, num);
            den = fma(t, t, den);
        }
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_down_sync(0xffffffffu, num, o);
            den += __shfl_down_sync(0xffffffffu, den, o);
        }
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            red[0][w] = num;
            red[1][w] = den;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                a += red[0][q];
                b += red[1][q];
            }
            partials[((size_t)blockIdx.x * V + v) * 2 + 0] = a;
            partials[((size_t)blockIdx.x * V + v) * 2 + 1] = b;
        }
        __syncthreads();
    }
}

__global__ void k_rmse_final(const double *__restrict__ partials, int nblocks, int V,
                             double *__restrict__ out) {
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (v >= V) return;
    double a = 0.0, b = 0.0;
    for (int q = lane; q < nblocks; q += 32) {
        a += partials[((size_t)q * V + v) * 2 + 0];
        b += partials[((size_t)q * V + v) * 2 + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) out[v] = sqrt(a / b);
}

template <typename T>
void launch_rmse(const T *x, const double *truth, int V, size_t npts, double *partials, int nblocks,
                 double *out, cudaStream_t s) {
    count_launches(2);
    k_rmse_partial<T><<<nblocks, 256, 0, s>>>(x, truth, V, npts, partials);
    k_rmse_final<<<1, 32 * V, 0, s>>>(partials, nblocks, V, out);
}

// ---------------------------------------------------------------------------
// conversions and normals
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout>
__global__ void k_convert(const Tin *__restrict__ in, Tout *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (Tout)in[i];
}

template <typename Tin, typename Tout>
void launch_convert(const Tin *in, Tout *out, size_t n, cudaStream_t s) {
    if (n == 0) return;
    count_launches(1);
    k_convert<Tin, Tout><<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
}

// the analysis counter that keys the perturbation stream lives on the device,
// so a captured cycle advances it on every replay
__global__ void k_bump_counter(uint64_t *c) { *c += 1; }

void launch_bump_counter(uint64_t *c, cudaStream_t s) {
    count_launches(1);
    k_bump_counter<<<1, 1, 0, s>>>(c);
}

__global__ void k_tt_bf16(const double *__restrict__ Tm, __nv_bfloat16 *__restrict__ Tt, int ne,
                          int ld, const int *status) {
    if (*status) return;
    const int total = (ne + 1) * ne;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int c = e / ne, a = e % ne;
        Tt[(size_t)c * ld + a] = __double2bfloat16(Tm[e]);
    }
}

void launch_tt_bf16(const double *Tm, __nv_bfloat16 *Tt, int ne, int ld, const int *status,
                    cudaStream_t s) {
    count_launches(1);
    k_tt_bf16<<<grid_for((size_t)(ne + 1) * ne, 256), 256, 0, s>>>(Tm, Tt, ne, ld, status);
}

// one thread per Philox block (4 normals)
__global__ void k_normals(uint64_t seed, uint64_t tag, uint64_t ctr0, int64_t count,
                          double *__restrict__ out) {
    const int64_t nblk = (count + 3) / 4;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
        double z[4];
        philox_normals4(seed, tag, ctr0, (uint64_t)b, z);
#pragma unroll
        for (int l = 0; l < 4; ++l)
            if (4 * b + l < count) out[4 * b + l] = z[l];
    }
}

void launch_normals(uint64_t seed, uint64_t tag, uint64_t ctr0, int64_t count, double *out,
                    cudaStream_t s) {
    if (count <= 0) return;
    count_launches(1);
    k_normals<<<grid_for((size_t)((count + 3) / 4), 256), 256, 0, s>>>(seed, tag, ctr0, count, out);
}

// ---------------------------------------------------------------------------
// grouped analysis of many problems: one launch per step, block b working on
// block map[b].y of problem map[b].x with the single-problem kernel body
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) kg_restrict(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const int2 e = map[blockIdx.x];
    const GroupProb &g = P[e.x];
    restrict_body<float>(g.fine, g.xstar, 2, 4, g.nc, g.r, e.y, ceil_div(g.nx, 256), g.dC);
}

__global__ void __launch_bounds__(128) kg_obs_apply(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const int2 e = map[blockIdx.x];
    const GroupProb &g = P[e.x];
    const int gx = ceil_div(g.ny, 128);
    obs_apply_body<float>(g.members, g.xstar, g.nx, g.ne, g.ny, g.taps, g.tap_idx, g.tap_w, g.yf, e.y % gx,
                          (e.y / gx) * kObsRows, kObsRows, g.tap_wh, g.tap_wl);
}

__global__ void __launch_bounds__(256) kg_obs_mean(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const int2 e = map[blockIdx.x];
    const GroupProb &g = P[e.x];
    obs_mean_body(g.yf, g.yo_in, g.ne, g.inv_ne, g.ny, g.ybar, g.Z, g.status, e.y, g.yo, g.df.Zh, g.df.Zl);
}

__global__ void __launch_bounds__(128) kg_obs_perturb(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const int2 e = map[blockIdx.x];
    const GroupProb &g = P[e.x];
    obs_perturb_body<true>(g.yf, g.ybar, g.yo, g.eps, 1, g.seed, g.cycle, g.sigma, g.ne, g.ny, g.isq, g.Y, g.Z, e.y,
                           g.df.Yh, g.df.Yl, g.df.Zh, g.df.Zl);
}

__global__ void __launch_bounds__(256) kg_innov_rms(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const GroupProb &g = P[map[blockIdx.x].x];
    innov_rms_body(g.Z + (size_t)g.ne * g.ny, g.ny, g.innov);
}

// block e.y = (z ty + by) tx + bx over the tiles of [S | Y^T R^-1 [D | d*]]
// and the K chunks z (tiles strictly below the diagonal of S are not listed)
__global__ void __launch_bounds__(kDfThreads) kg_gemm(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const int2 e = map[blockIdx.x];
    const GroupProb &g = P[e.x];
    if (*g.status) return;
    const int ne = g.ne, tx = ceil_div(2 * ne + 1, 16), ty = ceil_div(ne, 16);
    const int bx = e.y % tx, by = (e.y / tx) % ty, bz = e.y / (tx * ty);
    gemm_df_block(g.df, ne, g.ny, g.s2, 1.0, g.S, g.Bt, bx, by, bz, g.kchunk, g.splits > 1 ? g.part : nullptr);
}

__global__ void __launch_bounds__(256) kg_gemm_reduce(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const int2 e = map[blockIdx.x];
    const GroupProb &g = P[e.x];
    if (*g.status) return;
    gemm_nt_reduce_body(g.part, g.splits, g.ne, g.ne, g.ne + 1, true, g.s2, 1.0, g.S, g.Bt, e.y,
                        ceil_div((size_t)g.ne * (2 * g.ne + 1), 256));
}

// cluster c = blocks 8 c .. 8 c + 7, all of one problem (map entry per cluster)
__global__ void __cluster_dims__(kCholCluster, 1, 1) __launch_bounds__(288)
    kg_cholesky_cluster(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const GroupProb &g = P[map[blockIdx.x / kCholCluster].x];
    cholesky_cluster_body(g.S, g.Lt, g.ne, g.status);
}

__global__ void __launch_bounds__(256) kg_cholesky(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const GroupProb &g = P[map[blockIdx.x].x];
    cholesky_body<true>(g.S, g.Lt, g.ne, g.status);
}

template <int MAXR>
__global__ void __launch_bounds__(32 * kSolveColsPerCta)
    kg_chol_solve(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    const int2 e = map[blockIdx.x];
    const GroupProb &g = P[e.x];
    chol_solve_body<MAXR>(g.S, g.ne, g.Bt, g.Bt, g.ne + 1, g.Tt, g.ldx, g.status, e.y * kSolveColsPerCta,
                          kSolveColsPerCta);
}

// prolongation of the coarse intervals vj = kProlongIntervals e.y .. + 7 of
// one problem, all fine columns; the problem's scalars and weights are read
// once per block (the table entry is shared by all of the problem's blocks);
// block 0 of each problem advances its analysis counter
constexpr int kProlongIntervals = 8;

__global__ void __launch_bounds__(256) kg_prolong(const GroupProb *__restrict__ P, const int2 *__restrict__ map) {
    __shared__ float wt[kMaxRatio][4];
    __shared__ float *s_fine;
    __shared__ const float *s_dc;
    __shared__ int s_nc, s_r, s_skip;
    const int2 e = map[blockIdx.x];
    if (threadIdx.x == 0) {
        const GroupProb &g = P[e.x];
        if (e.y == 0) *g.cycle += 1;
        s_skip = *g.status;
        s_fine = g.fine;
        s_dc = g.dC;
        s_nc = g.nc;
        s_r = g.r;
    }
    __syncthreads();
    if (s_skip) return;
    const int nc = s_nc, r = s_r, nf = nc * r;
    prolong_stage_weights<float>(P[e.x].pw, r, wt);
    const int vj0 = e.y * kProlongIntervals, vj1 = min(vj0 + kProlongIntervals, 4 * nc);
    for (int fx = threadIdx.x; fx < nf; fx += blockDim.x)
        for (int vj = vj0; vj < vj1; ++vj) prolong2d_interval<float>(s_fine, s_dc, nc, r, wt, fx, vj);
}

bool group_supported(int ne, int ny) {
    // the solve's registers hold 32 MAXR rows (MAXR <= 8) and its staged
    // factor fits shared memory; the anomalies' BF16 rows fit the update
    return ne >= 2 && ne <= 160 && ny >= 1 && chol_solve_smem(ne) <= 210 * 1024;
}

void group_plan_free(GroupPlan *plan) {
    if (plan->d_probs) cudaFree(plan->d_probs);
    if (plan->d_maps) cudaFree(plan->d_maps);
    *plan = GroupPlan();
}

bool group_plan_build(GroupPlan *plan, const std::vector<GroupProb> &probs, const std::vector<CUtensorMap> &maps,
                      cudaStream_t s) {
    group_plan_free(plan);
    const int np = (int)probs.size();
    if (np < 1 || maps.size() != 2 * probs.size()) return false;
    std::vector<int2> m[kGsSteps];
    int maxne = 0;
    for (int j = 0; j < np; ++j) {
        const GroupProb &g = probs[j];
        if (!group_supported(g.ne, g.ny) || g.ldx % 16 || g.ldx < g.ne) return false;
        maxne = std::max(maxne, g.ne);
        auto add = [&](int step, long long nb) {
            for (long long b = 0; b < nb; ++b) m[step].push_back(make_int2(j, (int)b));
        };
        add(kGsRestrict, ceil_div(g.nx, 256));
        add(kGsObsApply, (long long)ceil_div(g.ny, 128) * ceil_div(g.ne + 1, kObsRows));
        add(kGsObsMean, ceil_div(g.ny, 32));
        add(kGsPerturb, ceil_div(((long long)g.ne * g.ny + 3) / 4, 128));
        add(kGsInnov, 1);
        {
            const int tx = ceil_div(2 * g.ne + 1, 16), ty = ceil_div(g.ne, 16);
            for (int z = 0; z < g.splits; ++z)
                for (int by = 0; by < ty; ++by)
                    for (int bx = by; bx < tx; ++bx) m[kGsGemm].push_back(make_int2(j, (z * ty + by) * tx + bx));
        }
        if (g.splits > 1) add(kGsReduce, ceil_div((long long)g.ne * (2 * g.ne + 1), 256));
        if (g.ne >= 32 && g.ne <= 256)
            add(kGsCholCluster, 1);
        else
            add(kGsChol, 1);
        add(kGsSolve, ceil_div(g.ne + 1, kSolveColsPerCta));
        add(kGsProlong, ceil_div(4 * g.nc, kProlongIntervals));
    }
    // launch shapes (the largest problem's shared memory)
    plan->solve_maxr = maxne <= 128 ? 4 : 8;
    plan->solve_smem = chol_solve_smem(maxne);
    plan->chol_cluster_smem = 0;
    plan->chol_smem = 0;
    for (const GroupProb &g : probs) {
        if (g.ne >= 32 && g.ne <= 256)
            plan->chol_cluster_smem = std::max(plan->chol_cluster_smem, cholesky_cluster_smem(g.ne));
        else
            plan->chol_smem = std::max(plan->chol_smem, sizeof(double) * (size_t)g.ne * (g.ne + 1));
    }
    if (plan->chol_smem > 210 * 1024) return false;
    // update: problems grouped by the CTAs per SM their shared memory and TMEM
    // columns allow, one launch per group of at most kUpdateLaunchMax
    {
        auto per_sm = [](size_t smem) { return (int)((size_t)227 * 1024 / smem); };
        std::vector<int> order(np);
        for (int j = 0; j < np; ++j) order[j] = j;
        auto need = [&](int j) {
            const GroupProb &g = probs[j];
            const size_t two = update_tc_smem(g.kblocks, g.ntile, g.ne, 2);
            return update_tc_launch_smem(two <= 200 * 1024 ? two : update_tc_smem(g.kblocks, g.ntile, g.ne, 1),
                                         g.tmem_cols);
        };
        for (int j = 0; j < np; ++j)
            if (need(j) > 200 * 1024) return false;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return per_sm(need(a)) > per_sm(need(b)); });
        for (size_t k = 0; k < order.size();) {
            GroupPlan::UpdateLaunch L;
            const int cls = per_sm(need(order[k]));
            L.map_begin = (int)m[kGsUpdate].size();
            while (k < order.size() && per_sm(need(order[k])) == cls && (int)L.probs.size() < kUpdateLaunchMax) {
                const int j = order[k++];
                const int q = (int)L.probs.size();
                L.probs.push_back(j);
                for (int t = 0; t < ceil_div(probs[j].nx, 128); ++t) m[kGsUpdate].push_back(make_int2(q, t));
            }
            L.map_end = (int)m[kGsUpdate].size();
            plan->upd.push_back(L);
        }
    }
    plan->upd_maps = maps;
    plan->upd_probs.resize(np);
    for (int j = 0; j < np; ++j) {
        const GroupProb &g = probs[j];
        UpdateProb &u = plan->upd_probs[j];
        u.members = g.members;
        u.dC = g.dC;
        u.status = g.status;
        u.nx = g.nx;
        u.ne = g.ne;
        u.kblocks = g.kblocks;
        u.ntile = g.ntile;
        u.wait_limit = g.wait_limit;
        u.inv_ne = g.inv_ne;
        u.isq = g.isq;
    }
    // one allocation for the table and every map
    size_t total = 0;
    for (int k = 0; k < kGsSteps; ++k) {
        plan->map_off[k] = (int)total;
        plan->nblocks[k] = (int)m[k].size();
        total += m[k].size();
    }
    std::vector<int2> all;
    all.reserve(total);
    for (int k = 0; k < kGsSteps; ++k) all.insert(all.end(), m[k].begin(), m[k].end());
    if (cudaMalloc(&plan->d_probs, np * sizeof(GroupProb)) != cudaSuccess ||
        cudaMalloc(&plan->d_maps, std::max<size_t>(total, 1) * sizeof(int2)) != cudaSuccess) {
        cudaGetLastError();
        group_plan_free(plan);
        return false;
    }
    plan->nprob = np;
    if (cudaMemcpyAsync(plan->d_probs, probs.data(), np * sizeof(GroupProb), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(plan->d_maps, all.data(), total * sizeof(int2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        group_plan_free(plan);
        return false;
    }
    return true;
}

cudaError_t group_analyse(const GroupPlan &plan, cudaStream_t s) {
    static OncePerDevice attr;
    cudaError_t ae = attr.run([](int) {
        cudaError_t e = cudaFuncSetAttribute(kg_cholesky_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kg_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kg_chol_solve<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kg_chol_solve<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
        return e;
    });
    if (ae != cudaSuccess) return ae;
    const GroupProb *P = plan.d_probs;
    auto M = [&](int k) { return plan.d_maps + plan.map_off[k]; };
    auto n = [&](int k) { return plan.nblocks[k]; };
    int launches = 0;
    auto step = [&](int k) {
        if (n(k)) ++launches;
        return n(k) > 0;
    };
    if (step(kGsRestrict)) kg_restrict<<<n(kGsRestrict), 256, 0, s>>>(P, M(kGsRestrict));
    if (step(kGsObsApply)) kg_obs_apply<<<n(kGsObsApply), 128, 0, s>>>(P, M(kGsObsApply));
    if (step(kGsObsMean)) kg_obs_mean<<<n(kGsObsMean), 256, 0, s>>>(P, M(kGsObsMean));
    if (step(kGsPerturb)) kg_obs_perturb<<<n(kGsPerturb), 128, 0, s>>>(P, M(kGsPerturb));
    if (step(kGsInnov)) kg_innov_rms<<<n(kGsInnov), 256, 0, s>>>(P, M(kGsInnov));
    if (step(kGsGemm)) kg_gemm<<<n(kGsGemm), kDfThreads, 0, s>>>(P, M(kGsGemm));
    if (step(kGsReduce)) kg_gemm_reduce<<<n(kGsReduce), 256, 0, s>>>(P, M(kGsReduce));
    if (step(kGsCholCluster))
        kg_cholesky_cluster<<<n(kGsCholCluster) * kCholCluster, 288, plan.chol_cluster_smem, s>>>(P, M(kGsCholCluster));
    if (step(kGsChol)) kg_cholesky<<<n(kGsChol), 256, plan.chol_smem, s>>>(P, M(kGsChol));
    if (step(kGsSolve)) {
        if (plan.solve_maxr == 4)
            kg_chol_solve<4><<<n(kGsSolve), 32 * kSolveColsPerCta, plan.solve_smem, s>>>(P, M(kGsSolve));
        else
            kg_chol_solve<8><<<n(kGsSolve), 32 * kSolveColsPerCta, plan.solve_smem, s>>>(P, M(kGsSolve));
    }
    count_launches(launches);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_update_tc_group(plan, s);
    if (e != cudaSuccess) return e;
    if (n(kGsProlong)) {
        count_launches(1);
        kg_prolong<<<n(kGsProlong), 256, 0, s>>>(P, M(kGsProlong));
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define MGK_INST(T)                                                                              \
    template void launch_restrict<T>(const T *, T *, int, int, int, int, cudaStream_t);          \
    template void launch_obs_apply<T>(const T *, const T *, size_t, int, int, int, const int32_t *, \
                                      const double *, double *, cudaStream_t, const float *,     \
                                      const float *);                                            \
    template void launch_ens_anom<T>(const T *, size_t, int, double *, __nv_bfloat16 *,          \
                                     const int *, cudaStream_t);                                 \
    template void launch_update_f64<T>(T *, T *, const double *, const double *, size_t, int,    \
                                       const int *, cudaStream_t);                               \
    template void launch_prolong_add<T>(T *, const T *, int, int, int, int,                      \
                                        const ProlongWeights &, const int *, cudaStream_t);      \
    template void launch_rmse<T>(const T *, const double *, int, size_t, double *, int, double *, \
                                 cudaStream_t);
MGK_INST(float)
MGK_INST(double)
#undef MGK_INST
template void launch_convert<double, float>(const double *, float *, size_t, cudaStream_t);
template void launch_convert<float, double>(const float *, double *, size_t, cudaStream_t);
template void launch_convert<double, double>(const double *, double *, size_t, cudaStream_t);

}  // namespace mgk
