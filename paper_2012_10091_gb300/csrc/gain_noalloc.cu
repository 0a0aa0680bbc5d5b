// gain_noalloc.cu -- the ensemble-space gain solve for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: a host application that hands
// every byte of device memory to its own pool up front, a process that runs
// under a fixed device-memory budget where a new driver allocation in the
// middle of a run is not allowed, or code that must not make allocation calls
// that synchronise the device.  For them this entry point computes the same
// T as the handle's analysis (S = I + Y^T Y / sigma^2, its FP64 Cholesky
// factor, T = S^-1 Y^T [D | d*] / sigma^2) using only the caller's inputs and
// outputs plus a fixed scratch array compiled into the library.
//
// The scratch is one file-scope __device__ array (S, L^T and a status word)
// sized for at most kNoAllocMaxMembers members; every GPU that loads the
// library holds it until the process exits.  Host code cannot use the array's
// name as a device address (on the host it names a shadow variable), so the
// first call on each device looks the address up with cudaGetSymbolAddress,
// with that device current, and keeps it.  Every call reuses the same array:
// the status word is cleared at the start of each call and S and L^T are fully
// rewritten, so nothing carries over from the previous call, but two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mgenkf_ops.h"
#include "analysis.h"
#include "common.cuh"

namespace {

constexpr int kNoAllocMaxMembers = 128;
constexpr int kNoAllocMaxDevices = 64;
constexpr size_t kMat = (size_t)kNoAllocMaxMembers * kNoAllocMaxMembers;

// [S (ne x ne) | L^T (ne x ne) | status word], 256 KB + 256 bytes
static __device__ __align__(256) double g_gain_scratch[2 * kMat + 32];

std::mutex g_mu;
double *g_addr[kNoAllocMaxDevices] = {};

// device address of the scratch array on the current device (set up once per device)
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gain_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// true if p is device (or managed) memory of the current device
bool on_current_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // the query's own error, raised just now
        return false;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" mgenkf_status mgk_gain_ensemble_noalloc(const double *Y, const double *Z, int32_t n_members,
                                                   int32_t n_obs, double obs_sigma, double *T,
                                                   int32_t *info, void *stream) {
    mgk_set_error("");
    if (!Y || !Z || !T) {
        mgk_set_error("mgk_gain_ensemble_noalloc: Y, Z and T are required");
        return MGENKF_ERR_INVALID_ARG;
    }
    if (n_members < 2 || n_members > kNoAllocMaxMembers) {
        mgk_set_error("mgk_gain_ensemble_noalloc: n_members must be in [2, " +
                      std::to_string(kNoAllocMaxMembers) + "] (fixed scratch size), got " +
                      std::to_string(n_members));
        return MGENKF_ERR_INVALID_ARG;
    }
    if (n_obs < 1 || !(obs_sigma > 0.0)) {
        mgk_set_error("mgk_gain_ensemble_noalloc: n_obs must be >= 1 and obs_sigma > 0");
        return MGENKF_ERR_INVALID_ARG;
    }
    if (!on_current_device(Y) || !on_current_device(Z) || !on_current_device(T) ||
        (info && !on_current_device(info))) {
        mgk_set_error("mgk_gain_ensemble_noalloc: Y, Z, T (and info, if given) must be device memory "
                      "of the current device");
        return MGENKF_ERR_INVALID_ARG;
    }
    // An error left pending by earlier, unrelated work would be read back by
    // the launch check below and reported as this call's failure: report it
    // now instead, without clearing it, and do nothing.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        mgk_set_error(std::string("mgk_gain_ensemble_noalloc: an earlier CUDA error is pending (not raised by "
                                  "this call): ") + cudaGetErrorString(e));
        return MGENKF_ERR_CUDA;
    }
    double *base = nullptr;
    e = scratch_address(&base);
    if (e != cudaSuccess) {
        mgk_set_error(std::string("mgk_gain_ensemble_noalloc: scratch address: ") + cudaGetErrorString(e));
        return MGENKF_ERR_CUDA;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    const int ne = n_members;
    double *S = base;
    double *Lt = base + kMat;
    int *status = reinterpret_cast<int *>(base + 2 * kMat);
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        const double s2 = obs_sigma * obs_sigma;
        mgk::launch_gemm_nt_f64(Y, ne, Y, ne, Z, ne + 1, n_obs, s2, 1.0, S, T, status, s);
        mgk::launch_cholesky(S, Lt, ne, status, s);
        mgk::launch_chol_solve(S, Lt, ne, T, T, ne + 1, nullptr, 0, status, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, status, sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        mgk_set_error(std::string("mgk_gain_ensemble_noalloc: ") + cudaGetErrorString(e));
        return MGENKF_ERR_CUDA;
    }
    return MGENKF_OK;
}
