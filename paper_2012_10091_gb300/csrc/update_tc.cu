// update_tc.cu -- member update and coarse correction on the tensor cores
// (Eq. ensemble_update with K = X Y^T C^-1, written as x^a,(i) = x^f,(i) + X T_i,
// and x^C' - x^C* = X T_ne, Algorithm 4 step 5).
//
// D[p][c] = sum_a X[p][a] T[c][a]: M = Nx points (tile 128), N = Ne + 1 padded
// to a multiple of 16 (<= 256), K = Ne padded to 16, BF16 operands, FP32
// accumulation.  One CTA per 128-point tile:
//   * one thread issues the TMA loads of the X tile and of T (K-major, 128-byte
//     swizzle, 64 values per swizzle atom) and waits on an mbarrier;
//   * warp 0 allocates TMEM for the 128 x N FP32 accumulator;
//   * one thread issues K/16 tcgen05.mma (kind::f16, cta_group::1) and commits
//     them to a second mbarrier;
//   * the same TMA transaction brings the members' 128-point tile ([Ne][128]
//     FP32), so the epilogue never waits on global loads;
//   * the four warps read their 32 TMEM lanes (tcgen05.ld 32x32b), add
//     D[p][c] into the shared member tile (c < Ne) and store dC[p] = D[p][Ne];
//     one thread writes the member tile back with a TMA store.
// Every mbarrier wait is bounded (about a second of SM clocks); on expiry the
// kernel records MGENKF_ERR_TIMEOUT in the status word, waits (bounded) for its
// own copies, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "analysis.h"
#include "common.cuh"
#include "tc_common.cuh"
#include "update_tc.h"

namespace mgk {

namespace {

constexpr int kTileM = 128;
constexpr int kAtomK = 64;                        // bf16 values per 128-byte swizzle row
using namespace tc;

}  // namespace

__global__ void __launch_bounds__(128) k_update_tc(const __grid_constant__ CUtensorMap map_x,
                                                   const __grid_constant__ CUtensorMap map_t,
                                                   const __grid_constant__ CUtensorMap map_m,
                                                   float *__restrict__ dC, int nx, int ne, int kblocks,
                                                   int ntile, int tmem_cols, long long wait_limit, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand buffers
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sa = base;                                        // kblocks x [128][64] bf16
    unsigned char *sb = base + (size_t)kblocks * kTileM * 128;       // kblocks x [ntile][64] bf16
    float *sm = reinterpret_cast<float *>(sb + (size_t)kblocks * ntile * 128);  // [ne][128] members
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + (size_t)ne * kTileM);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;
    if (tid == 0) {
        s_fail = *status;  // one read: the whole CTA leaves or none of it
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (s_fail) return;  // s_fail is 0 from here on until the TMA wait below
    const uint32_t tx_bytes = (uint32_t)kblocks * (kTileM + ntile) * 128 + (uint32_t)ne * kTileM * 4;
    if (tid == 0) {
        mbar_expect_tx(&bars[0], tx_bytes);
        for (int kb = 0; kb < kblocks; ++kb) {
            tma_load_2d(sa + (size_t)kb * kTileM * 128, &map_x, &bars[0], kb * kAtomK, m0);
            tma_load_2d(sb + (size_t)kb * ntile * 128, &map_t, &bars[0], kb * kAtomK, 0);
        }
        tma_load_2d(sm, &map_m, &bars[0], m0, 0);
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

    if (tid == 0) {
        // the operand wait uses the plan's limit; an expired wait issues no MMA
        if (!mbar_wait(&bars[0], 0, wait_limit)) {
            s_fail = 1;
        } else {
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
    }
    __syncthreads();
    bool ok = s_fail == 0;
    if (ok && !mbar_wait(&bars[1], 0)) ok = false;
    ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the TMEM loads below are warp-collective
    if (!ok) {
        if (tid == 0) {
            atomicCAS(status, 0, kStTimeout);
            mbar_wait(&bars[0], 0);  // let our own copies land (default bound) before the CTA exits
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
        if (tid == 0) tma_store_2d(&map_m, sm, m0, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
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

static size_t update_smem(int kblocks, int ntpad, int ne) {
    return 1024 + (size_t)kblocks * (kTileM + ntpad) * 128 + (size_t)ne * kTileM * 4 + 64;
}

bool update_tc_supported(int ne, int ldx, int ntpad, int nx) {
    // N = ntpad rows of T in one MMA (<= 256), K = ldx (multiple of 16); TMA
    // inner box of 64 values; the member tile box is 128 x ne (ne <= 256) with
    // rows of nx floats (a multiple of 16 bytes); all of it fits shared memory.
    if (ntpad < 16 || ntpad > 256 || ntpad % 16 || ldx % 16 || ne < 2 || ne > 256 || nx % 4) return false;
    const int kblocks = (ldx + kAtomK - 1) / kAtomK;
    return update_smem(kblocks, ntpad, ne) <= 200 * 1024 && encode_fn() != nullptr;
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

bool update_tc_prepare(UpdateTcPlan *plan, const __nv_bfloat16 *X16, int ldx, int nx, const __nv_bfloat16 *Tt,
                       int ntpad, int ne, const float *members) {
    if (!update_tc_supported(ne, ldx, ntpad, nx)) return false;
    memset(plan, 0, sizeof(*plan));
    plan->kblocks = (ldx + kAtomK - 1) / kAtomK;
    plan->ntile = ntpad;
    int cols = 32;
    while (cols < ntpad) cols <<= 1;
    plan->tmem_cols = cols;
    plan->smem = update_smem(plan->kblocks, ntpad, ne);
    // at most 512 / tmem_cols CTAs may share an SM's 512 TMEM columns: ask for
    // enough shared memory that no more are resident (no CTA ever waits in alloc)
    const size_t per_sm = 228 * 1024;
    const size_t min_smem = per_sm / (size_t)(512 / cols + 1) + 2048;
    if (plan->smem < min_smem) plan->smem = min_smem;
    plan->nx = nx;
    plan->ne = ne;
    plan->wait_limit = kWaitLimitCycles;
    if (!encode_kmajor(&plan->map_x, X16, ldx, nx, kTileM)) return false;
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
    k_update_tc<<<grid, 128, plan.smem, s>>>(plan.map_x, plan.map_t, plan.map_m, dC, plan.nx, plan.ne, plan.kblocks,
                                             plan.ntile, plan.tmem_cols, plan.wait_limit, status);
    return cudaGetLastError();
}

}  // namespace mgk
