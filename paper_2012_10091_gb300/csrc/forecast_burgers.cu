// forecast_burgers.cu -- batched SSP-RK3 forecast of periodic viscous Burgers.
//
// Model (Eq. burgers, flux form on a periodic vertex grid x_j = j dx):
//   dt L(u)_j = a (u_{j-1}^2 - u_{j+1}^2) + b (u_{j+1} - 2 u_j + u_{j-1}),
//   a = dt / (4 dx), b = dt nu / dx^2      [= dt (-(F_{j+1}-F_{j-1})/(2dx) + nu D2 u), F = u^2/2]
// Time (SSP-RK3, Shu-Osher form):
//   u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1)); u' = 1/3 u + 2/3 (u2 + dt L(u2)).
//
// GPU design.  The grids of the cycle (the Ne coarse members, Algorithm 3
// step 2, and the fine run, Algorithm 4 step 2) advance by all nsteps of an
// observation interval inside one kernel pass:
//   * a grid segment lives in registers for the whole launch: thread t owns
//     consecutive points, so a member is read from and written to memory once
//     per interval; only the edge values of each thread go through shared
//     memory (double-buffered);
//   * a member grid (<= 4096 points) is one CTA ("whole" CTAs);
//   * a fine grid larger than that is split over a thread-block cluster of cs
//     CTAs ("split" CTAs); the CTA-edge values are read from the neighbouring
//     CTA's shared memory (DSMEM) after a cluster barrier.  This keeps every SM
//     at about the same per-step work instead of letting the fine run, r_C
//     times a member, set the pace on a single SM;
//   * the FP32 path (burgers_f32x2_kernel) runs the fine run on its own
//     cluster launch and the members in a second launch beside it (see
//     launch_burgers); the generic kernel runs both in one launch.
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

// Stage increments of SSP-RK3 written around the state u0 at the start of the step:
//   k0 = dt L(u0),  u1 = u0 + k0
//   k1 = dt L(u1),  u2 = u0 + (k0 + k1) / 4
//   k2 = dt L(u2),  u' = u0 + (k0 + k1) / 6 + 2/3 k2
// which is the Shu-Osher form u2 = 3/4 u0 + 1/4 (u1 + k1), u' = 1/3 u0 + 2/3 (u2 + k2)
// rearranged.  dt L is formed from neighbour differences (exact in floating
// point for neighbours within a factor 2):
//   dt L_j = a (u_{j-1} - u_{j+1}) (u_{j-1} + u_{j+1}) + b ((u_{j+1} - u_j) + (u_{j-1} - u_j)).
// With the small dt of the fine grid one step changes u by about one FP32 ulp,
// so the FP32 state is carried as a compensated pair (hi, lo): the step
// increment is added with Fast2Sum and its rounding error kept in lo.
template <typename T>
__device__ __forceinline__ T burgers_dtl(T prev, T cur, T nxt, T a, T b) {
    const T lap = (nxt - cur) + (prev - cur);
    const T adv = (prev - nxt) * (prev + nxt);
    return fma(a, adv, b * lap);
}

// One stage on the P points a thread owns.  s: stage input (overwritten by the
// next stage input, or by nothing in the last stage); hi/lo: state at the start
// of the step (updated in the last stage); kk: k0, then k0 + k1.  lft/rgt: stage
// inputs of the neighbouring points outside the thread.  Returns the value the
// thread must publish as its last point for the next stage.
template <typename T, int P, bool FULL, int STAGE>
__device__ __forceinline__ T burgers_stage(T (&s)[P], T (&hi)[P], T (&lo)[P], T (&kk)[P], int cnt,
                                           T lft, T rgt, T a, T b) {
    constexpr bool COMP = sizeof(T) == 4;
    T last = T(0);
    T prev = lft;
    T cur = s[0];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (FULL || k < cnt) {
            T nxt;
            if (k + 1 < P) {
                nxt = (FULL || k + 1 < cnt) ? s[k + 1] : rgt;
            } else {
                nxt = rgt;
            }
            const T kq = burgers_dtl(prev, cur, nxt, a, b);
            T nv;
            if (STAGE == 0) {
                kk[k] = kq;
                nv = hi[k] + kq;
            } else if (STAGE == 1) {
                kk[k] = kk[k] + kq;
                nv = fma(T(0.25), kk[k], hi[k]);
            } else {
                const T d = fma(T(2.0 / 3.0), kq, kk[k] * T(1.0 / 6.0));
                if (COMP) {  // Fast2Sum: hi + (lo + d) = new hi + new lo exactly
                    const T t = lo[k] + d;
                    const T sum = hi[k] + t;
                    lo[k] = t - (sum - hi[k]);
                    hi[k] = sum;
                } else {
                    hi[k] = hi[k] + d;
                }
                nv = hi[k];
            }
            s[k] = nv;
            if (FULL ? k == P - 1 : k == cnt - 1) last = nv;
            prev = cur;
            cur = nxt;
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

    T v[P], hi[P], lo[P], kk[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        v[k] = (k < cnt) ? base[t * P + k] : T(0);
        hi[k] = v[k];
        lo[k] = T(0);
    }
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
                vlast = burgers_stage<T, P, true, S>(v, hi, lo, kk, cnt, lft, rgt, a, b);
            } else {
                vlast = burgers_stage<T, P, false, S>(v, hi, lo, kk, cnt, lft, rgt, a, b);
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
        if (k < cnt) base[t * P + k] = hi[k] + lo[k];
    // peers may still read this CTA's shared memory in their last stage
    if (split) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// FP32 fast path: folded pairs, packed FP32x2 arithmetic, one barrier per step.
//
// A CTA segment of npts points is folded into h = npts/2 pairs (A_j, B_j) =
// (point j, point j + h), held as float2 so that every arithmetic instruction
// (FFMA2 / FADD2 / FMUL2) advances two points.  Thread t owns pairs
// [tQ, tQ + Q) plus a halo of 3 pairs on each side; the three RK stages are
// computed on shrinking ranges (Q+4, Q+2, Q pairs), so the halo is refreshed
// once per time step instead of once per stage.  Folding makes the neighbour
// of pair 0 on the left (B_{h-1}, A_{h-1}) of the left segment/self and the
// neighbour of pair h-1 on the right (B_0, A_0) of self/right segment: the two
// components swap at the fold.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// The folded kernel carries the scaled variable v = a u (a = dt / (4 dx); the
// load and the store convert, see burgers_f32x2_kernel).  In v the stage
// increment a dt L(u)_j needs no multiplication by a:
//   a dt L(u)_j = b (v_{j+1} - 2 v_j + v_{j-1}) + (v_{j-1} - v_{j+1}) (v_{j-1} + v_{j+1})
//              = b (d_{j-1} - d_j) + (d_{j-1} + d_j) (v_{j-1} + v_{j+1}),   d_j = v_j - v_{j+1},
// and the edge difference d_j serves points j and j + 1: six operations per
// point (d_j, the two edge combinations, the neighbour sum, the product and one
// FMA) against eight for the unscaled form.  d_j is exact for neighbours within
// a factor 2, so the diffusion term keeps the accuracy of the difference form.
__device__ __forceinline__ float2 dtl_x2(float2 prev, float2 nxt, float2 dl, float2 dr, float2 cb) {
    const float2 m1 = f2(-1.f);
    const float2 lap = __ffma2_rn(dr, m1, dl);  // d_{j-1} - d_j
    const float2 dif = __fadd2_rn(dl, dr);      // v_{j-1} - v_{j+1}
    return __ffma2_rn(cb, lap, __fmul2_rn(dif, __fadd2_rn(prev, nxt)));
}

__device__ __forceinline__ float2 edge_x2(float2 left, float2 right) {
    return __ffma2_rn(right, f2(-1.f), left);  // left - right
}

// One time step on the pairs a thread holds: hv = hi parts at the start of the
// step (own pairs at [3, Q+3), halo pairs around them), lo = low parts of the
// own pairs, sv = stage inputs, kk = k0 then k0 + k1 (index i-1 for pair i).
// Stage ranges shrink by one pair per side: [1, Q+5), [2, Q+4), [3, Q+3).
// All values are in the scaled variable v.
template <int Q>
__device__ __forceinline__ void step_x2(float2 (&hv)[Q + 6], float2 (&lo)[Q], float2 (&sv)[Q + 6],
                                        float2 (&kk)[Q + 4], float2 cb) {
    const float2 m1 = f2(-1.f);
    // stage 1: k0 = a dt L(u0), v1 = v0 + k0
    {
        float2 dl = edge_x2(hv[0], hv[1]);
#pragma unroll
        for (int i = 1; i < Q + 5; ++i) {
            const float2 dr = edge_x2(hv[i], hv[i + 1]);
            const float2 k0 = dtl_x2(hv[i - 1], hv[i + 1], dl, dr, cb);
            kk[i - 1] = k0;
            sv[i] = __fadd2_rn(hv[i], k0);
            dl = dr;
        }
    }
    // stage 2: k1 = a dt L(u1), v2 = v0 + (k0 + k1) / 4   (in place, previous input kept)
    {
        float2 prev = sv[1];
        float2 dl = edge_x2(sv[1], sv[2]);
#pragma unroll
        for (int i = 2; i < Q + 4; ++i) {
            const float2 cur = sv[i];
            const float2 dr = edge_x2(cur, sv[i + 1]);
            const float2 k1 = dtl_x2(prev, sv[i + 1], dl, dr, cb);
            kk[i - 1] = __fadd2_rn(kk[i - 1], k1);
            sv[i] = __ffma2_rn(f2(0.25f), kk[i - 1], hv[i]);
            prev = cur;
            dl = dr;
        }
    }
    // stage 3: k2 = a dt L(u2), v' = v0 + (k0 + k1)/6 + 2/3 k2, added by Fast2Sum
    {
        float2 prev = sv[2];
        float2 dl = edge_x2(sv[2], sv[3]);
#pragma unroll
        for (int i = 3; i < Q + 3; ++i) {
            const float2 cur = sv[i];
            const float2 dr = edge_x2(cur, sv[i + 1]);
            const float2 k2 = dtl_x2(prev, sv[i + 1], dl, dr, cb);
            // t = lo + (k0 + k1)/6 + 2/3 k2 in two FMAs
            const float2 t = __ffma2_rn(f2(2.0f / 3.0f), k2, __ffma2_rn(f2(1.0f / 6.0f), kk[i - 1], lo[i - 3]));
            const float2 sum = __fadd2_rn(hv[i], t);
            lo[i - 3] = __ffma2_rn(__ffma2_rn(hv[i], m1, sum), m1, t);  // t - (sum - hi)
            hv[i] = sum;
            prev = cur;
            dl = dr;
        }
    }
}

template <int Q>
__global__ void __launch_bounds__(512) burgers_f32x2_kernel(BurgersArgs<float> A) {
    // A launch that follows this one with programmatic serialisation (the
    // members after the fine run, see launch_burgers) may start once every CTA
    // here is resident; before leaving, a CTA waits for the grid it follows
    // (a no-op for a launch that follows none).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sh = reinterpret_cast<float2 *>(smem_raw);  // [2 buffers][first 3 | last 3][blockDim]
    const int t = threadIdx.x, nt = blockDim.x;
    const int bid = blockIdx.x;
    float *base;
    int npts, rank = 0;
    float a, b;
    bool split;
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
    const int h = npts / 2;
    const int te = h / Q;  // threads owning pairs; the others only join the barriers
    const bool active = t < te;
    const float2 cb = f2(b);

    // v = a u as the compensated pair (hi, lo): the rounding error of a u is
    // exact in one FMA
    float2 w[Q + 6], lo[Q], sv[Q + 6], kk[Q + 4];
    if (active) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int j = t * Q + k;
            const float2 u = make_float2(base[j], base[h + j]);
            w[3 + k] = __fmul2_rn(f2(a), u);
            lo[k] = __ffma2_rn(f2(a), u, make_float2(-w[3 + k].x, -w[3 + k].y));
        }
    }
    int buf = 0;
    for (int step = 0; step < A.nsteps; ++step) {
        float2 *F = sh + buf * 6 * nt;  // first3[m] at F[m*nt + t], last3[m] at F[(3+m)*nt + t]
        if (active) {
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                F[m * nt + t] = w[3 + m];
                F[(3 + m) * nt + t] = w[Q + m];
            }
        }
        if (split) {
            cg::this_cluster().sync();
        } else {
            __syncthreads();
        }
        if (active) {
            if (t > 0) {
#pragma unroll
                for (int m = 0; m < 3; ++m) w[m] = F[(3 + m) * nt + t - 1];
            } else {
                const float2 *L = split ? cg::this_cluster().map_shared_rank(F, (rank + A.cs - 1) % A.cs) : F;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float2 r = L[(3 + m) * nt + te - 1], l = F[(3 + m) * nt + te - 1];
                    w[m] = make_float2(r.y, l.x);
                }
            }
            if (t < te - 1) {
#pragma unroll
                for (int m = 0; m < 3; ++m) w[Q + 3 + m] = F[m * nt + t + 1];
            } else {
                const float2 *R = split ? cg::this_cluster().map_shared_rank(F, (rank + 1) % A.cs) : F;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float2 l = F[m * nt], r = R[m * nt];
                    w[Q + 3 + m] = make_float2(l.y, r.x);
                }
            }
            step_x2<Q>(w, lo, sv, kk, cb);
        }
        buf ^= 1;
    }
    if (active) {
        // u = (hi + lo) / a: q = hi / a correctly rounded, its remainder
        // hi - q a exact in one FMA, then the remainder and lo divided and added
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int j = t * Q + k;
            const float qx = __fdiv_rn(w[3 + k].x, a), qy = __fdiv_rn(w[3 + k].y, a);
            const float rx = fmaf(-qx, a, w[3 + k].x), ry = fmaf(-qy, a, w[3 + k].y);
            base[j] = qx + __fdiv_rn(rx + lo[k].x, a);
            base[h + j] = qy + __fdiv_rn(ry + lo[k].y, a);
        }
    }
    if (split) cg::this_cluster().sync();
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Q (pairs per thread) for the folded kernel, or 0 if it does not apply:
// every segment even, h % Q == 0, h / Q <= 512 threads.
static int choose_q(const BurgersArgs<float> &A) {
    static int env = -1;
    if (env < 0) {
        const char *s = getenv("MGENKF_BURGERS_Q");
        env = s ? atoi(s) : 0;
    }
    const int cand[4] = {env, 8, 4, 16};
    for (int c : cand) {
        if (c != 4 && c != 8 && c != 16) continue;
        bool ok = true;
        if (A.n_whole_probs > 0) ok = ok && A.n_whole % (2 * c) == 0 && A.n_whole / (2 * c) <= 512;
        if (A.n_split_probs > 0) {
            const int seg = A.n_split / A.cs;
            ok = ok && A.n_split % A.cs == 0 && seg % (2 * c) == 0 && seg / (2 * c) <= 512;
        }
        if (ok) return c;
    }
    return 0;
}

// The folded kernel works in v = a u: a must keep v and the products of v in
// the normal FP32 range (a = dt / (4 dx) lies far inside this for any usable
// step); other a go to the generic kernel.
static bool fold_scale_ok(const BurgersArgs<float> &A) {
    auto ok = [](float a) { return a >= 0x1p-40f && a <= 0x1p40f; };
    return (A.n_whole_probs == 0 || ok(A.aw)) && (A.n_split_probs == 0 || ok(A.as));
}

template <int Q>
static cudaError_t launch_f32x2(const BurgersArgs<float> &A, cudaStream_t stream, bool follows = false,
                                bool whole_sm = false) {
    int te = 0;
    if (A.n_whole_probs > 0) te = A.n_whole / (2 * Q);
    if (A.n_split_probs > 0) te = max(te, A.n_split / A.cs / (2 * Q));
    const int nt = ceil_div(te, 32) * 32;
    size_t smem = sizeof(float2) * 12 * (size_t)nt;  // <= 48 KB for nt <= 512
    if (whole_sm) {
        // enough shared memory that no other CTA fits beside this one on its SM
        static OncePerDevice attr;
        attr.run([](int) {
            return cudaFuncSetAttribute(burgers_f32x2_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        210 * 1024);
        });
        smem = 210 * 1024;
    }
    const int grid = A.whole_ctas + A.n_split_probs * A.cs;
    if (grid == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[2];
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    if (A.cs > 1) {
        attr[cfg.numAttrs].id = cudaLaunchAttributeClusterDimension;
        attr[cfg.numAttrs].val.clusterDim.x = A.cs;
        attr[cfg.numAttrs].val.clusterDim.y = 1;
        attr[cfg.numAttrs].val.clusterDim.z = 1;
        ++cfg.numAttrs;
    }
    if (follows) {  // may start while the previous launch on the stream runs (see the kernel)
        attr[cfg.numAttrs].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[cfg.numAttrs].val.programmaticStreamSerializationAllowed = 1;
        ++cfg.numAttrs;
    }
    count_launches(1);
    return cudaLaunchKernelEx(&cfg, burgers_f32x2_kernel<Q>, A);
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
    if constexpr (std::is_same<T, float>::value) {
        static int off = -1;
        if (off < 0) off = getenv("MGENKF_BURGERS_GENERIC") ? 1 : 0;
        const bool fold = !off && fold_scale_ok(A);
        if (fold && A.nsteps > 0 && A.n_whole_probs > 0 && A.n_split_probs > 0 && A.n_whole % 16 == 0 &&
            A.n_whole / 16 <= 512) {
            // Members and a split fine run: a split grid's step costs its
            // cluster barrier (a 4096-point segment under a cluster barrier
            // steps about a quarter slower than a whole 4096-point grid under its
            // CTA barrier), so the fine run gets segments of at most 2048 points
            // on its own cluster launch, and the members follow it with
            // programmatic serialisation: they start once the fine run's CTAs
            // are resident (the cluster is placed first) and run beside it.
            int cs2 = 0;
            for (int cs = 2; cs <= 8 && !cs2; cs <<= 1)
                if (A.n_split % cs == 0 && A.n_split / cs <= kBurgersMaxPtsPerCta / 2 && (A.n_split / cs) % 8 == 0)
                    cs2 = cs;
            if (cs2) {
                BurgersArgs<float> F = A, W = A;
                F.n_whole_probs = 0;
                F.whole_ctas = 0;
                F.cs = cs2;
                W.n_split_probs = 0;
                W.cs = 1;
                W.whole_ctas = A.n_whole_probs;
                // four pairs per thread on the fine run (256 threads per 2048-point
                // segment: two warps per SM sub-partition instead of one), eight on
                // the members
                cudaError_t e = launch_f32x2<4>(F, stream, false, true);
                if (e != cudaSuccess) return e;
                return launch_f32x2<8>(W, stream, true);
            }
        }
        if (fold && A.nsteps > 0) {
            switch (choose_q(A)) {
                case 4: return launch_f32x2<4>(A, stream);
                case 8: return launch_f32x2<8>(A, stream);
                case 16: return launch_f32x2<16>(A, stream);
                default: break;
            }
        }
    }
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
