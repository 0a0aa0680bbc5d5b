// peak_probe.cu -- throughput probes of the FP32 and FP64 FMA pipes.
//
// The roofline of the forecast kernels is their FP32 arithmetic, and that of
// the Cholesky the FP64 pipe; neither peak is a library routine that could be
// timed instead.  These kernels run eight independent FMA chains per thread
// over four 256-thread CTAs per SM, enough warps to cover the FMA latency on
// every SM sub-partition, and write one value per thread so the chains stay
// live.  The caller times the launch on `stream` and divides the flops it
// reports by that time.
#include <cuda_runtime.h>

#include "../../include/mgenkf_ops.h"
#include "common.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T *sink) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = T(1) + T(t * kChains + j) * T(1e-9);
    // a <- a * b + c contracts towards c / (1 - b): no overflow, no denormals
    const T b = T(0.999999), c = T(1e-6);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    sink[t] = s;
}

}  // namespace

extern "C" mgenkf_status mgk_fma_probe(int32_t fp64, int32_t iters, void *sink, double *flops, void *stream) {
    mgk_set_error("");
    if (iters < 1 || !sink || !flops) {
        mgk_set_error("mgk_fma_probe: iters >= 1, sink and flops are required");
        return MGENKF_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        mgk_set_error(std::string("mgk_fma_probe: ") + cudaGetErrorString(e));
        return MGENKF_ERR_CUDA;
    }
    const int grid = kCtasPerSm * sms;
    const cudaStream_t s = (cudaStream_t)stream;
    if (fp64)
        k_fma_probe<double><<<grid, kThreads, 0, s>>>(iters, static_cast<double *>(sink));
    else
        k_fma_probe<float><<<grid, kThreads, 0, s>>>(iters, static_cast<float *>(sink));
    mgk::count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        mgk_set_error(std::string("mgk_fma_probe: ") + cudaGetErrorString(e));
        return MGENKF_ERR_CUDA;
    }
    *flops = 2.0 * kChains * (double)iters * grid * kThreads;
    return MGENKF_OK;
}

extern "C" int32_t mgk_fma_probe_threads(void) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    return kCtasPerSm * sms * kThreads;
}
