// forecast_burgers.cu -- batched SSP-RK3 forecast of periodic viscous Burgers.
//
// Model (Eq. burgers, flux form on a periodic vertex grid x_j = j dx):
//   dt L(u)_j = a (u_{j-1}^2 - u_{j+1}^2) + b (u_{j+1} + u_{j-1} - 2 u_j),
//   a = dt / (4 dx), b = dt nu / dx^2      [= dt (-(F_{j+1}-F_{j-1})/(2dx) + nu D2 u), F = u^2/2]
// Time (SSP-RK3, Shu-Osher form):
//   u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1)); u' = 1/3 u + 2/3 (u2 + dt L(u2)).
//
// GPU design.  One launch advances every grid of the cycle (the Ne coarse
// members, Algorithm 3 step 2, and the fine run, Algorithm 4 step 2) by all
// nsteps of an observation interval:
//   * a grid segment lives in registers for the whole launch: thread t owns P
//     consecutive points, so a member is read from and written to memory once
//     per interval; only the two edge values of each thread go through shared
//     memory at every RK stage (one barrier per stage, double-buffered);
//   * a member grid (<= 4096 points) is one CTA ("whole" CTAs);
//   * a fine grid larger than that is split over a thread-block cluster of cs
//     CTAs ("split" CTAs); the CTA-edge values are read from the neighbouring
//     CTA's shared memory (DSMEM) after a cluster barrier.  This keeps every SM
//     at the same per-step work instead of letting the fine run, r_C times a
//     member, set the pace on a single SM.
#include <cooperative_groups.h>

#include <cstdio>
#include <cstdlib>
#include <string>
#include <type_traits>

#include "common.cuh"
#include "forecast.h"

namespace cg = cooperative_groups;

namespace mgk {

template <typename T>
struct BurgersArgs {
    T *whole;          // n_whole_probs grids of n_whole points
    int n_whole;
    int n_whole_probs;
    int whole_ctas;    // n_whole_probs rounded up to a multiple of cs
    T aw, bw;          // stencil constants on the whole grids
    T *split;          // n_split_probs grids of n_split points, cs CTAs each
    int n_split;
    int n_split_probs;
    int cs;
    T as, bs;
    int nsteps;
};

// One RK stage on the points a thread owns.  v: stage input (overwritten by
// the stage output); u0: state at the start of the step; lft/rgt: old values
// of the neighbouring points outside the thread.  FULL: the thread owns all P
// points (no ragged tail).
// Returns the new value of the thread's last owned point.
template <typename T, int P, bool FULL, int STAGE>
__device__ __forceinline__ T burgers_stage(T (&v)[P], T (&u0)[P], int cnt, T lft, T rgt, T a,
                                           T b) {
    T last = T(0);
    T prev = lft;
    T sq_prev = lft * lft;
    T cur = v[0];
    T sq_cur = cur * cur;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (FULL || k < cnt) {
            T nxt;
            if (k + 1 < P) {
                nxt = (FULL || k + 1 < cnt) ? v[k + 1] : rgt;
            } else {
                nxt = rgt;
            }
            const T sq_nxt = nxt * nxt;
            const T lap = fma(T(-2), cur, prev + nxt);
            const T dtL = fma(a, sq_prev - sq_nxt, b * lap);
            T nv;
            if (STAGE == 0) {
                u0[k] = cur;
                nv = cur + dtL;
            } else if (STAGE == 1) {
                nv = fma(T(0.25), cur + dtL, T(0.75) * u0[k]);
            } else {
                nv = fma(T(2.0 / 3.0), cur + dtL, u0[k] * T(1.0 / 3.0));
            }
            v[k] = nv;
            if (FULL ? k == P - 1 : k == cnt - 1) last = nv;
            prev = cur;
            sq_prev = sq_cur;
            cur = nxt;
            sq_cur = sq_nxt;
        }
    }
    return last;
}

template <typename T, int P>
constexpr int burgers_max_threads() {
    return P >= 16 ? 256 : (P >= 8 ? 512 : 1024);
}

template <typename T, int P>
__global__ void __launch_bounds__(burgers_max_threads<T, P>())
    burgers_rk3_kernel(BurgersArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sh = reinterpret_cast<T *>(smem_raw);  // [2 buffers][first | last][blockDim]
    const int t = threadIdx.x, nt = blockDim.x;
    const int bid = blockIdx.x;

    T *base;
    int npts;
    T a, b;
    bool split;
    int rank = 0;
    if (bid < A.whole_ctas) {
        if (bid >= A.n_whole_probs) return;  // padding CTA of the last cluster
        base = A.whole + (size_t)bid * A.n_whole;
        npts = A.n_whole;
        a = A.aw;
        b = A.bw;
        split = false;
    } else {
        const int q = bid - A.whole_ctas;
        const int prob = q / A.cs;
        rank = q % A.cs;
        npts = A.n_split / A.cs;
        base = A.split + (size_t)prob * A.n_split + (size_t)rank * npts;
        a = A.as;
        b = A.bs;
        split = A.cs > 1;
    }
    const int t_last = (npts - 1) / P;                 // last thread owning points
    const int cnt = min(max(npts - t * P, 0), P);      // points owned by this thread

    T v[P], u0[P];
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = (k < cnt) ? base[t * P + k] : T(0);
    // value of the last owned point, kept in its own register (a runtime
    // index into v[] would move the array to local memory)
    T vlast = cnt > 0 ? base[t * P + cnt - 1] : T(0);

    // one RK stage: publish the thread's edge values, barrier, read the
    // neighbours' edge values (DSMEM across the CTA edges of a split grid),
    // update the owned points.  Buffers alternate so one barrier per stage
    // separates every write from the reads of the previous stage.
    int buf = 0;
    auto stage = [&](auto stage_tag) {
        constexpr int S = decltype(stage_tag)::value;
        T *shf = sh + buf * 2 * nt;
        T *shl = shf + nt;
        if (cnt > 0) {
            shf[t] = v[0];
            shl[t] = vlast;
        }
        if (split) {
            cg::this_cluster().sync();
        } else {
            __syncthreads();
        }
        if (cnt > 0) {
            T lft, rgt;
            if (t > 0) {
                lft = shl[t - 1];
            } else if (split) {
                const int left = (rank + A.cs - 1) % A.cs;
                lft = cg::this_cluster().map_shared_rank(shl, left)[t_last];
            } else {
                lft = shl[t_last];
            }
            if (t < t_last) {
                rgt = shf[t + 1];
            } else if (split) {
                const int right = (rank + 1) % A.cs;
                rgt = cg::this_cluster().map_shared_rank(shf, right)[0];
            } else {
                rgt = shf[0];
            }
            if (cnt == P) {
                vlast = burgers_stage<T, P, true, S>(v, u0, cnt, lft, rgt, a, b);
            } else {
                vlast = burgers_stage<T, P, false, S>(v, u0, cnt, lft, rgt, a, b);
            }
        }
        buf ^= 1;
    };
    for (int step = 0; step < A.nsteps; ++step) {
        stage(std::integral_constant<int, 0>{});
        stage(std::integral_constant<int, 1>{});
        stage(std::integral_constant<int, 2>{});
    }
#pragma unroll
    for (int k = 0; k < P; ++k)
        if (k < cnt) base[t * P + k] = v[k];
    // peers may still read this CTA's shared memory in their last stage
    if (split) cg::this_cluster().sync();
}

static int pow2_ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <typename T, int P>
static cudaError_t launch_burgers_p(const BurgersArgs<T> &A, int maxpts, cudaStream_t stream) {
    int nt = ceil_div(maxpts, P);
    nt = ceil_div(nt, 32) * 32;
    if (nt > burgers_max_threads<T, P>()) return cudaErrorInvalidConfiguration;
    const size_t smem = sizeof(T) * 4 * (size_t)nt;
    const int grid = A.whole_ctas + A.n_split_probs * A.cs;
    if (grid == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    if (A.cs > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = A.cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.numAttrs = 1;
    }
    count_launches(1);
    return cudaLaunchKernelEx(&cfg, burgers_rk3_kernel<T, P>, A);
}

// Points per thread: about 256 threads per CTA, or the MGENKF_BURGERS_PTS
// override (1, 2, 4, 8 or 16).
static int choose_pts(int maxpts) {
    static int env = -1;
    if (env < 0) {
        const char *s = getenv("MGENKF_BURGERS_PTS");
        env = s ? atoi(s) : 0;
    }
    int p = env;
    if (p != 1 && p != 2 && p != 4 && p != 8 && p != 16) {
        p = pow2_ceil(ceil_div(maxpts, 256));
        if (p > 16) p = 16;
    }
    while (p < 16 && ceil_div(maxpts, p) > 1024) p <<= 1;
    return p;
}

template <typename T>
static cudaError_t launch_burgers(BurgersArgs<T> A, cudaStream_t stream) {
    int maxpts = 0;
    if (A.n_whole_probs > 0) maxpts = A.n_whole;
    if (A.n_split_probs > 0) maxpts = max(maxpts, A.n_split / A.cs);
    if (maxpts == 0 || A.nsteps == 0) return cudaSuccess;
    switch (choose_pts(maxpts)) {
        case 1: return launch_burgers_p<T, 1>(A, maxpts, stream);
        case 2: return launch_burgers_p<T, 2>(A, maxpts, stream);
        case 4: return launch_burgers_p<T, 4>(A, maxpts, stream);
        case 8: return launch_burgers_p<T, 8>(A, maxpts, stream);
        default: return launch_burgers_p<T, 16>(A, maxpts, stream);
    }
}

int burgers_split_factor(int n) {
    // CTAs per grid: the smallest power of two cs with n / cs <= 4096 and n % cs == 0
    for (int cs = 1; cs <= 8; cs <<= 1)
        if (n % cs == 0 && n / cs <= kBurgersMaxPtsPerCta) return cs;
    return 0;
}

template <typename T>
cudaError_t burgers_forecast(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                             int n_split_probs, double length, double dt, double nu, int nsteps,
                             cudaStream_t stream) {
    BurgersArgs<T> A = {};
    A.cs = n_split_probs > 0 ? burgers_split_factor(n_split) : 1;
    if (A.cs == 0) return cudaErrorInvalidValue;
    A.whole = whole;
    A.n_whole = n_whole;
    A.n_whole_probs = n_whole_probs;
    A.whole_ctas = ceil_div(n_whole_probs, A.cs) * A.cs;
    if (n_whole_probs > 0) {
        const double dx = length / n_whole;
        A.aw = (T)(dt / (4.0 * dx));
        A.bw = (T)(dt * nu / (dx * dx));
    }
    A.split = split;
    A.n_split = n_split;
    A.n_split_probs = n_split_probs;
    if (n_split_probs > 0) {
        const double dx = length / n_split;
        A.as = (T)(dt / (4.0 * dx));
        A.bs = (T)(dt * nu / (dx * dx));
    }
    A.nsteps = nsteps;
    return launch_burgers<T>(A, stream);
}

template cudaError_t burgers_forecast<float>(float *, int, int, float *, int, int, double, double,
                                             double, int, cudaStream_t);
template cudaError_t burgers_forecast<double>(double *, int, int, double *, int, int, double,
                                              double, double, int, cudaStream_t);

}  // namespace mgk
