// common.cuh -- shared device/host helpers of the MGEnKF GPU library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/mgenkf.h"

namespace mgk {

// ---------------------------------------------------------------------------
// Host: run a set-up step once per device.  Kernel attributes (the dynamic
// shared-memory limit) and occupancy figures belong to one device context, so
// a flag shared by all devices would skip the step on the second device.  The
// step runs with the device current; it is retried on the next call if it
// failed.  Thread-safe.
// ---------------------------------------------------------------------------
constexpr int kMaxDevices = 128;
class OncePerDevice {
  public:
    // index of the current device in [0, kMaxDevices), or -1 on error
    static int current() {
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
        return dev;
    }
    template <class F>
    cudaError_t run(F &&f) {
        const int dev = current();
        if (dev < 0) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lock(mu_);
        if (done_[dev]) return cudaSuccess;
        const cudaError_t e = f(dev);
        if (e == cudaSuccess) done_[dev] = true;
        return e;
    }

  private:
    std::mutex mu_;
    bool done_[kMaxDevices] = {};
};

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (grids are sized from the device query)

__host__ __device__ inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// device status word values (a subset of mgenkf_status)
constexpr int kStatusOk = 0;

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller normals.
// ---------------------------------------------------------------------------
struct U64x4 {
    uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    U64x4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

// Normals n = 4 blk .. 4 blk + 3 of the stream (seed, tag, ctr0): Philox block
// (ctr0, blk, 0, 0) with key (seed, tag); lanes (0, 1) and (2, 3) give one
// Box-Muller pair each, u = ((x >> 11) + 1) 2^-53, z = sqrt(-2 ln u1) (cos, sin)(2 pi u2).
__device__ __forceinline__ void philox_normals4(uint64_t seed, uint64_t tag, uint64_t ctr0, uint64_t blk,
                                                double (&z)[4]) {
    const U64x4 x = philox4x64_10(ctr0, blk, 0, 0, seed, tag);
    const double inv53 = 1.0 / 9007199254740992.0;
#pragma unroll
    for (int pair = 0; pair < 2; ++pair) {
        const double u1 = (double)((x.v[2 * pair] >> 11) + 1) * inv53;
        const double u2 = (double)((x.v[2 * pair + 1] >> 11) + 1) * inv53;
        const double rad = sqrt(-2.0 * log(u1));
        const double th = 6.283185307179586 * u2;
        z[2 * pair] = rad * cos(th);
        z[2 * pair + 1] = rad * sin(th);
    }
}

// The same four normals with the Box-Muller transform evaluated in FP32 on
// the same Philox words (each uniform rounded to FP32 first): within about
// 1e-6 of the FP64 values, without GB300's slow FP64 logarithm and sines.
__device__ __forceinline__ void philox_normals4_f32(uint64_t seed, uint64_t tag, uint64_t ctr0, uint64_t blk,
                                                    double (&z)[4]) {
    const U64x4 x = philox4x64_10(ctr0, blk, 0, 0, seed, tag);
#pragma unroll
    for (int pair = 0; pair < 2; ++pair) {
        const float u1 = __ull2float_rn((x.v[2 * pair] >> 11) + 1) * 0x1p-53f;
        const float u2 = __ull2float_rn((x.v[2 * pair + 1] >> 11) + 1) * 0x1p-53f;
        const float rad = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincosf(6.2831853071795865f * u2, &sn, &cs);
        z[2 * pair] = (double)(rad * cs);
        z[2 * pair + 1] = (double)(rad * sn);
    }
}

constexpr uint64_t kEpsTag = 0x45505300ULL;  // "EPS\0": perturbation stream of the analysis

// ---------------------------------------------------------------------------
// small type helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double to_f64(T x) {
    return (double)x;
}

}  // namespace mgk

namespace mgk {
// number of kernel launches issued by the library (process-wide counter)
void count_launches(int n);
}  // namespace mgk

// error text of the stateless entry points (per host thread)
void mgk_set_error(const std::string &msg);
