// filter.cu -- centred sixth-order filter of the NS model (the paper's Euler
// and Navier-Stokes runs damp spurious oscillations with one, Secs. 5 and 6,
// citing Bogey and Bailly; it prints no coefficients).  Reading: the 7-point
// centred stencil
//   u_j <- u_j - sigma/64 (-u_{j-3} + 6 u_{j-2} - 15 u_{j-1} + 20 u_j - 15 u_{j+1} + 6 u_{j+2} - u_{j+3}),
// transfer function 1 - sigma sin^6(k h / 2), applied along x and then along y
// to the four conserved planes of every grid, after each model step.  Two
// out-of-place passes (x: state -> tmp, y: tmp -> state), register-blocked:
// along x a thread filters 4 consecutive points from 12 loaded values, along y
// a thread filters 8 consecutive rows of one column from 14 loaded values, so
// a point costs 3 or 1.75 loads instead of 7 and the index arithmetic is paid
// once per block.  A warp's loads and stores cover consecutive addresses.
#include <cuda_runtime.h>

#include "analysis.h"
#include "common.cuh"

namespace mgk {

// filter taps d_m, m = -3..3, and the combination u - sigma/64 sum_m d_m u_{j+m}
template <typename T>
__device__ __forceinline__ T filt6(const T *w, T s64) {
    const T D = T(-1) * w[0] + T(6) * w[1] + T(-15) * w[2] + T(20) * w[3] + T(-15) * w[4] + T(6) * w[5] +
                T(-1) * w[6];
    return w[3] - s64 * D;
}

// along x: thread t of plane z -> row t / (n/4), chunk c = t % (n/4) of 4 points
template <typename T>
__global__ void __launch_bounds__(256) k_filter6_x(const T *__restrict__ in, T *__restrict__ out, int n, T s64) {
    const int nc = n >> 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nc) return;
    const int y = t / nc, c = t - y * nc;
    const size_t row = (size_t)blockIdx.z * n * n + (size_t)y * n;
    const T *r = in + row;
    T w[12];  // points 4c - 4 .. 4c + 7
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        int cc = c - 1 + q;
        cc = cc < 0 ? cc + nc : (cc >= nc ? cc - nc : cc);
#pragma unroll
        for (int k = 0; k < 4; ++k) w[4 * q + k] = r[4 * cc + k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) out[row + 4 * c + k] = filt6(w + 1 + k, s64);
}

// along y: thread t of plane z -> column x = t % n, rows 8 (t / n) .. + 7
template <typename T>
__global__ void __launch_bounds__(256) k_filter6_y(const T *__restrict__ in, T *__restrict__ out, int n, T s64) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * (n >> 3)) return;
    const int g = t / n, x = t - g * n;
    const int y0 = g * 8;
    const size_t pl = (size_t)blockIdx.z * n * n;
    T w[14];  // rows y0 - 3 .. y0 + 10
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        int y = y0 - 3 + k;
        y = y < 0 ? y + n : (y >= n ? y - n : y);
        w[k] = in[pl + (size_t)y * n + x];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) out[pl + (size_t)(y0 + k) * n + x] = filt6(w + k, s64);
}

template <typename T>
cudaError_t launch_ns2d_filter6(T *q, T *tmp, int n, int nprob, double sigma, cudaStream_t s) {
    if (nprob <= 0) return cudaSuccess;
    if (n < 8 || n % 8 != 0) return cudaErrorInvalidValue;  // NS grids: n % 8 == 0
    count_launches(2);
    const T s64 = (T)(sigma / 64.0);
    k_filter6_x<T><<<dim3(ceil_div(n * (n / 4), 256), 1, 4 * nprob), 256, 0, s>>>(q, tmp, n, s64);
    k_filter6_y<T><<<dim3(ceil_div(n * (n / 8), 256), 1, 4 * nprob), 256, 0, s>>>(tmp, q, n, s64);
    return cudaGetLastError();
}

template cudaError_t launch_ns2d_filter6<float>(float *, float *, int, int, double, cudaStream_t);
template cudaError_t launch_ns2d_filter6<double>(double *, double *, int, int, double, cudaStream_t);

}  // namespace mgk
