// update_tc.cu -- member update and coarse correction on the tensor cores
// (Eq. ensemble_update with K = X Y^T C^-1, written as x^a,(i) = x^f,(i) + X T_i,
// and x^C' - x^C* = X T_ne, Algorithm 4 step 5), with the normalised
// anomalies X of the forecast ensemble (Eq. Ensemble_Anomaly) formed on the way.
//
// D[p][c] = sum_a X[p][a] T[c][a]: M = Nx points (tile 128), N = Ne + 1 padded
// to a multiple of 16 (<= 256), K = Ne padded to 16, BF16 operands, FP32
// accumulation.  One CTA per 128-point tile:
//   * one thread issues the TMA loads of T (K-major, 128-byte swizzle, 64
//     values per swizzle atom) and of the members' 128-point tile ([Ne][128]
//     FP32) and waits on an mbarrier;
//   * warp 0 allocates TMEM for the 128 x N FP32 accumulator;
//   * each thread forms its point's ensemble mean from the member tile (FP32
//     error-free sums over 8 member slices, combined in FP64) and its row of
//     BF16 anomalies (x_i - mean) / sqrt(Ne - 1), written in the 128-byte
//     swizzled K-major layout the MMA reads (the layout TMA would write), so
//     the members are read from HBM once for both the anomalies and the update;
//   * one thread issues K/16 tcgen05.mma (kind::f16, cta_group::1) and commits
//     them to a second mbarrier;
//   * the four warps read their 32 TMEM lanes (tcgen05.ld 32x32b), add
//     D[p][c] into the shared member tile (c < Ne) and store dC[p] = D[p][Ne];
//     one thread writes the member tile back with a TMA store.
// Every mbarrier wait is bounded (about a second of SM clocks); on expiry the
// kernel records MGENKF_ERR_TIMEOUT in the status word, waits (bounded) for its
// own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "analysis.h"
#include "batch_analysis.h"
#include "common.cuh"
#include "tc_common.cuh"
#include "update_tc.h"

namespace mgk {

namespace {

constexpr int kTileM = 128;
constexpr int kAtomK = 64;                        // bf16 values per 128-byte swizzle row
using namespace tc;

}  // namespace

// One 128-point tile (first point m0) of one problem; the tensor maps are
// kernel parameters (__grid_constant__) of the calling kernel.  inv_ne = 1/Ne,
// isq = 1/sqrt(Ne - 1) (host values).
__device__ __forceinline__ void update_tc_tile(const CUtensorMap *map_t, const CUtensorMap *map_m,
                                               float *__restrict__ dC, int nx, int ne, int kblocks, int ntile,
                                               int tmem_cols, long long wait_limit, int *status, int m0,
                                               double inv_ne, double isq) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand buffers
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sa = base;                                        // kblocks x [128][64] bf16 (written here)
    unsigned char *sb = base + (size_t)kblocks * kTileM * 128;       // kblocks x [ntile][64] bf16 (TMA)
    float *sm = reinterpret_cast<float *>(sb + (size_t)kblocks * ntile * 128);  // [ne][128] members (TMA)
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + (size_t)ne * kTileM);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);
    __shared__ int s_fail, s_bad;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        s_fail = *status;  // one read: the whole CTA leaves or none of it
        s_bad = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (s_fail) return;  // s_fail is 0 from here on until the operand wait below
    const uint32_t tx_bytes = (uint32_t)kblocks * ntile * 128 + (uint32_t)ne * kTileM * 4;
    if (tid == 0) {
        mbar_expect_tx(&bars[0], tx_bytes);
        for (int kb = 0; kb < kblocks; ++kb)
            tma_load_2d(sb + (size_t)kb * ntile * 128, map_t, &bars[0], kb * kAtomK, 0);
        tma_load_2d(sm, map_m, &bars[0], m0, 0);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // the operand wait uses the plan's limit (thread 0 decides for the CTA); an
    // expired wait issues no MMA
    if (tid == 0 && !mbar_wait(&bars[0], 0, wait_limit)) s_fail = 1;
    __syncthreads();
    bool ok = s_fail == 0;
    if (ok) {
        mbar_wait(&bars[0], 0);  // complete: each thread's own acquire of the copied tiles
        // ensemble mean of point pl: members i = q, q + 8, ... summed in FP32
        // with their rounding errors (error-free two-sum), the 8 slice sums
        // combined in FP64 in slice order
        const int pl = tid;
        double sum = 0.0;
        for (int q = 0; q < 8; ++q) {
            float sh = 0.f, sl = 0.f;
            for (int i = q; i < ne; i += 8) {
                const float a = sm[i * kTileM + pl];
                const float t = sh + a, bv = t - sh;
                sl += (sh - (t - bv)) + (a - bv);
                sh = t;
            }
            sum += (double)sh + (double)sl;
        }
        // BF16 anomalies, FP32 centring and scaling; K padding is zero.  Row pl
        // of atom kb: 8 granules of 16 bytes, granule g stored at g ^ (pl mod 8)
        const float xbf = (float)(sum * inv_ne), isqf = (float)isq;
        const uint32_t sw = (uint32_t)(pl & 7);
        for (int kb = 0; kb < kblocks; ++kb) {
            unsigned char *row = sa + (size_t)kb * kTileM * 128 + (size_t)pl * 128;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int i0 = kb * kAtomK + g * 8 + 2 * h;
                    const float v0 = i0 < ne ? (sm[i0 * kTileM + pl] - xbf) * isqf : 0.f;
                    const float v1 = i0 + 1 < ne ? (sm[(i0 + 1) * kTileM + pl] - xbf) * isqf : 0.f;
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v0, v1);  // v0 at the lower address
                    w[h] = *reinterpret_cast<const uint32_t *>(&b2);
                }
                *reinterpret_cast<uint4 *>(row + (((uint32_t)g ^ sw) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        // the anomaly rows are read by the MMA (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (ok && tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = idesc_bf16(kTileM, ntile);
        const int ksteps = kblocks * (kAtomK / 16);
        for (int j = 0; j < ksteps; ++j) {
            const int kb = j / (kAtomK / 16), kk = j % (kAtomK / 16);
            const uint64_t adesc = smem_desc_sw128(smem_u32(sa + (size_t)kb * kTileM * 128 + kk * 32));
            const uint64_t bdesc = smem_desc_sw128(smem_u32(sb + (size_t)kb * ntile * 128 + kk * 32));
            mma_bf16(tmem, adesc, bdesc, idesc, j > 0 ? 1u : 0u);
        }
        mma_commit(&bars[1]);
    }
    // the accumulator wait; the CTA goes on only if every thread saw it
    if (ok && !mbar_wait(&bars[1], 0)) s_bad = 1;
    __syncthreads();
    const bool done = ok && s_bad == 0;
    if (!done) {
        if (tid == 0) {
            atomicCAS(status, 0, kStTimeout);
            if (!ok) mbar_wait(&bars[0], 0);  // let our own copies land (default bound) before the CTA exits
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int pl = warp * 32 + lane, p = m0 + pl;
        const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < ntile; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(row + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int c = c0 + q;
                const float v = __uint_as_float(r[q]);
                if (c < ne)
                    sm[c * kTileM + pl] += v;  // rows past nx are clipped by the TMA store
                else if (c == ne && p < nx)
                    dC[p] = v;
            }
        }
        // the member tile goes back with one TMA store (generic-proxy writes
        // made visible to the async proxy first)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) tma_store_2d(map_m, sm, m0, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

__global__ void __launch_bounds__(128) k_update_tc(const __grid_constant__ CUtensorMap map_t,
                                                   const __grid_constant__ CUtensorMap map_m,
                                                   float *__restrict__ dC, int nx, int ne, int kblocks,
                                                   int ntile, int tmem_cols, long long wait_limit, int *status,
                                                   double inv_ne, double isq) {
    update_tc_tile(&map_t, &map_m, dC, nx, ne, kblocks, ntile, tmem_cols, wait_limit, status, blockIdx.x * kTileM,
                   inv_ne, isq);
}

// The update of up to kUpdateGroupMax problems in one launch: their tensor
// maps travel as one parameter block (T and members of the launch's problem q
// at 2 q, 2 q + 1; prob[q] its index in the table); block b works on tile
// map[b].y of the launch's problem map[b].x.
struct UpdateGroupMaps {
    CUtensorMap m[2 * kUpdateGroupMax];
    int prob[kUpdateGroupMax];
};

__global__ void __launch_bounds__(128) k_update_tc_group(const __grid_constant__ UpdateGroupMaps maps,
                                                         const GroupProb *__restrict__ probs,
                                                         const int2 *__restrict__ map) {
    // the problem's scalars are read once per block (every block of the
    // problem reads the same table entry)
    __shared__ float *s_dc;
    __shared__ int *s_status;
    __shared__ int s_nx, s_ne, s_kb, s_nt, s_cols;
    __shared__ long long s_wait;
    __shared__ double s_inv, s_isq;
    const int2 e = map[blockIdx.x];
    if (threadIdx.x == 0) {
        const GroupProb &g = probs[maps.prob[e.x]];
        s_dc = g.dC;
        s_status = g.status;
        s_nx = g.nx;
        s_ne = g.ne;
        s_kb = g.kblocks;
        s_nt = g.ntile;
        s_cols = g.tmem_cols;
        s_wait = g.wait_limit;
        s_inv = g.inv_ne;
        s_isq = g.isq;
    }
    __syncthreads();
    update_tc_tile(&maps.m[2 * e.x], &maps.m[2 * e.x + 1], s_dc, s_nx, s_ne, s_kb, s_nt, s_cols, s_wait, s_status,
                   e.y * kTileM, s_inv, s_isq);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

static bool encode_kmajor(CUtensorMap *m, const __nv_bfloat16 *ptr, int ld, int rows, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)kAtomK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t update_tc_smem(int kblocks, int ntpad, int ne) {
    return 1024 + (size_t)kblocks * (kTileM + ntpad) * 128 + (size_t)ne * kTileM * 4 + 64;
}

size_t update_tc_launch_smem(size_t smem, int tmem_cols) {
    // at most 512 / tmem_cols CTAs may share an SM's 512 TMEM columns: ask for
    // enough shared memory that no more are resident (no CTA ever waits in alloc)
    const size_t per_sm = 228 * 1024;
    const size_t min_smem = per_sm / (size_t)(512 / tmem_cols + 1) + 2048;
    return smem < min_smem ? min_smem : smem;
}

bool update_tc_supported(int ne, int ldx, int ntpad, int nx) {
    // N = ntpad rows of T in one MMA (<= 256), K = ldx (multiple of 16); TMA
    // inner box of 64 values; the member tile box is 128 x ne (ne <= 256) with
    // rows of nx floats (a multiple of 16 bytes); all of it fits shared memory.
    // The anomaly rows hold 64 kblocks >= ne values.
    if (ntpad < 16 || ntpad > 256 || ntpad % 16 || ldx % 16 || ne < 2 || ne > 256 || nx % 4) return false;
    const int kblocks = (ldx + kAtomK - 1) / kAtomK;
    return update_tc_smem(kblocks, ntpad, ne) <= 200 * 1024 && encode_fn() != nullptr;
}

static bool encode_members(CUtensorMap *m, const float *ptr, int nx, int ne) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ne};
    const cuuint64_t strides[1] = {(cuuint64_t)nx * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kTileM, (cuuint32_t)ne};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool update_tc_prepare(UpdateTcPlan *plan, int ldx, int nx, const __nv_bfloat16 *Tt, int ntpad, int ne,
                       const float *members) {
    if (!update_tc_supported(ne, ldx, ntpad, nx)) return false;
    memset(plan, 0, sizeof(*plan));
    plan->kblocks = (ldx + kAtomK - 1) / kAtomK;
    plan->ntile = ntpad;
    int cols = 32;
    while (cols < ntpad) cols <<= 1;
    plan->tmem_cols = cols;
    plan->smem = update_tc_launch_smem(update_tc_smem(plan->kblocks, ntpad, ne), cols);
    plan->nx = nx;
    plan->ne = ne;
    plan->wait_limit = kWaitLimitCycles;
    if (!encode_kmajor(&plan->map_t, Tt, ldx, ntpad, ntpad)) return false;
    if (!encode_members(&plan->map_m, members, nx, ne)) return false;
    plan->members = members;
    plan->ready = true;
    return true;
}

cudaError_t launch_update_tc(const UpdateTcPlan &plan, float *members, float *dC, int *status, cudaStream_t s) {
    static OncePerDevice attr;
    attr.run([](int) { return cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); });
    if (members != plan.members) return cudaErrorInvalidValue;
    count_launches(1);
    const int grid = (plan.nx + kTileM - 1) / kTileM;
    k_update_tc<<<grid, 128, plan.smem, s>>>(plan.map_t, plan.map_m, dC, plan.nx, plan.ne, plan.kblocks, plan.ntile,
                                             plan.tmem_cols, plan.wait_limit, status, 1.0 / plan.ne,
                                             1.0 / std::sqrt((double)(plan.ne - 1)));
    return cudaGetLastError();
}

cudaError_t launch_update_tc_group(const GroupPlan &plan, cudaStream_t s) {
    static OncePerDevice attr;
    cudaError_t e = attr.run(
        [](int) { return cudaFuncSetAttribute(k_update_tc_group, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); });
    if (e != cudaSuccess) return e;
    UpdateGroupMaps maps;
    for (const GroupPlan::UpdateLaunch &L : plan.upd) {
        const int nb = L.map_end - L.map_begin;
        if (nb <= 0) continue;
        memset(&maps, 0, sizeof(maps));
        for (size_t q = 0; q < L.probs.size(); ++q) {
            maps.m[2 * q] = plan.upd_maps[2 * (size_t)L.probs[q]];
            maps.m[2 * q + 1] = plan.upd_maps[2 * (size_t)L.probs[q] + 1];
            maps.prob[q] = L.probs[q];
        }
        count_launches(1);
        k_update_tc_group<<<nb, 128, L.smem, s>>>(maps, plan.d_probs, plan.d_maps + plan.map_off[kGsUpdate] + L.map_begin);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mgk
