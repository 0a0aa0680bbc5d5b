// filter.cu -- centred sixth-order filter of the NS model (the paper's Euler
// and Navier-Stokes runs damp spurious oscillations with one, Secs. 5 and 6,
// citing Bogey and Bailly; it prints no coefficients).  Reading: the 7-point
// centred stencil
//   u_j <- u_j - sigma/64 (-u_{j-3} + 6 u_{j-2} - 15 u_{j-1} + 20 u_j - 15 u_{j+1} + 6 u_{j+2} - u_{j+3}),
// transfer function 1 - sigma sin^6(k h / 2), applied along x and then along y
// to the four conserved planes of every grid, after each model step.  Two
// out-of-place passes (x: state -> tmp, y: tmp -> state), one thread per point;
// a warp's 32 points are consecutive in x, so every load and store is coalesced
// and the 7-point reads hit L1.
#include <cuda_runtime.h>

#include "analysis.h"
#include "common.cuh"

namespace mgk {

template <typename T, bool ALONG_X>
__global__ void __launch_bounds__(256) k_filter6(const T *__restrict__ in, T *__restrict__ out, int n, T s64) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= n) return;
    const T *p = in + (size_t)blockIdx.z * n * n;  // one conserved plane of one grid
    const T d[7] = {T(-1), T(6), T(-15), T(20), T(-15), T(6), T(-1)};
    T D = T(0);
#pragma unroll
    for (int m = -3; m <= 3; ++m) {
        int j = (ALONG_X ? x : y) + m;
        j = j < 0 ? j + n : (j >= n ? j - n : j);
        D += d[m + 3] * (ALONG_X ? p[(size_t)y * n + j] : p[(size_t)j * n + x]);
    }
    const size_t o = (size_t)blockIdx.z * n * n + (size_t)y * n + x;
    out[o] = in[o] - s64 * D;
}

template <typename T>
cudaError_t launch_ns2d_filter6(T *q, T *tmp, int n, int nprob, double sigma, cudaStream_t s) {
    if (nprob <= 0) return cudaSuccess;
    if (n < 7) return cudaErrorInvalidValue;  // the 7-point stencil wraps at most once
    count_launches(2);
    const dim3 grid(ceil_div(n, 256), n, 4 * nprob);
    const T s64 = (T)(sigma / 64.0);
    k_filter6<T, true><<<grid, 256, 0, s>>>(q, tmp, n, s64);
    k_filter6<T, false><<<grid, 256, 0, s>>>(tmp, q, n, s64);
    return cudaGetLastError();
}

template cudaError_t launch_ns2d_filter6<float>(float *, float *, int, int, double, cudaStream_t);
template cudaError_t launch_ns2d_filter6<double>(double *, double *, int, int, double, cudaStream_t);

}  // namespace mgk
