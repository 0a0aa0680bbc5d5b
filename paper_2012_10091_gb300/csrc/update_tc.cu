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
//   * each thread forms its point's ensemble mean from the member tile (x_ref
//     = member 0's value plus the mean of the exact differences x_i - x_ref,
//     summed in FP32 over 8 member slices) and its row of BF16 anomalies
//     ((x_i - x_ref) - dm) / sqrt(Ne - 1), written in the 128-byte
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

#include <algorithm>
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
constexpr int kUpdateThreads = 256;  // two threads per point of the tile
constexpr int kAtomK = 64;                        // bf16 values per 128-byte swizzle row
using namespace tc;

}  // namespace

// The update of the tiles of up to kUpdateLaunchMax problems: the tensor maps
// and scalars of the launch's problems travel as one parameter block (T and
// members of problem q at m[2 q], m[2 q + 1]); tile k of the launch is tile
// map[k].y of problem map[k].x (map NULL: tile k of problem 0).
struct UpdateLaunchArgs {
    CUtensorMap m[2 * kUpdateLaunchMax];
    UpdateProb p[kUpdateLaunchMax];
    int kbmax, ntmax, nemax, cols;  // shared-memory layout and TMEM columns of the launch
    int nbuf;                       // member buffers (2: the next tile's load overlaps this tile)
};

// Persistent: CTA b works through the tiles [b n / G, (b + 1) n / G) in
// order, one 128-point tile at a time, with two member buffers (one where two
// do not fit shared memory), one anomaly (A) buffer, one T buffer and one TMEM
// accumulator.  Tile k (buffer k & 1):
//   a. thread 0 starts the next tile's member load into the other buffer
//      (free: the previous tile's epilogue has read it; with one buffer the
//      load starts after this tile's epilogue);
//   b. wait for the tile's members (and T when the problem changed);
//   c. the anomalies of the tile into A;
//   d. thread 0 issues the MMAs and commits them; wait for the accumulator;
//   e. thread 0 starts the next problem's T load if the problem changes;
//   f. epilogue: members[c][p] = x[c][p] + D[p][c] from the buffer, stored to
//      HBM directly; dC[p] = D[p][Ne].
// Tiles of a problem whose status word is set are skipped.  Any wait that
// runs out stops the CTA: MGENKF_ERR_TIMEOUT in that problem's status word,
// the copies in flight awaited (default bound), TMEM freed.
__global__ void __launch_bounds__(kUpdateThreads) k_update_tc(const __grid_constant__ UpdateLaunchArgs a,
                                                   const int2 *__restrict__ map, int nent) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand buffers
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sa = base;                                            // kbmax x [128][64] bf16 (written here)
    unsigned char *sb = base + (size_t)a.kbmax * kTileM * 128;           // kbmax x [ntile][64] bf16 (TMA)
    float *smb = reinterpret_cast<float *>(sb + (size_t)a.kbmax * a.ntmax * 128);  // nbuf x [ne][128] members (TMA)
    const size_t bstride = (size_t)a.nemax * kTileM;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smb + a.nbuf * bstride);  // members x2, MMA, T
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
    __shared__ int s_abort, s_next, s_next2, s_tload;
    __shared__ float s_part[4][kTileM];  // slice sums 4..7 of the second thread half
    __shared__ float2 s_ref[kTileM];     // per point: x_ref, mean offset dm

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int e0 = (int)((long long)blockIdx.x * nent / gridDim.x);
    const int e1 = (int)((long long)(blockIdx.x + 1) * nent / gridDim.x);
    auto entry = [&](int k) { return map ? map[k] : make_int2(0, k); };

    // thread 0's view of the copies: the problem whose T is (being) loaded, the
    // status of the last problem looked at; per member barrier (bit b) the
    // parity of its last load and whether that load is outstanding
    int tq = -1, sq = -1, sq_ok = 0, lpar = 0, pend = 0, ntl = 0, pend_t = 0;
    auto next_valid = [&](int k) {
        for (; k < e1; ++k) {
            const int q = entry(k).x;
            if (q != sq) {
                sq = q;
                sq_ok = *(volatile int *)a.p[q].status == 0;
            }
            if (sq_ok) break;
        }
        return k;
    };
    int nld[2] = {0, 0};  // loads issued per member barrier (thread 0)
    auto load_members = [&](int k, int b) {
        const int2 e = entry(k);
        mbar_expect_tx(&bars[b], (uint32_t)a.p[e.x].ne * kTileM * 4);
        tma_load_2d(smb + b * bstride, &a.m[2 * e.x + 1], &bars[b], e.y * kTileM, 0);
        const int n = b ? ++nld[1] : ++nld[0];
        lpar = (lpar & ~(1 << b)) | (((n - 1) & 1) << b);
        pend |= 1 << b;
    };
    auto load_t = [&](int q) {
        const UpdateProb &P = a.p[q];
        mbar_expect_tx(&bars[3], (uint32_t)P.kblocks * P.ntile * 128);
        for (int kb = 0; kb < P.kblocks; ++kb)
            tma_load_2d(sb + (size_t)kb * P.ntile * 128, &a.m[2 * q], &bars[3], kb * kAtomK, 0);
        tq = q;
        pend_t = 1;
        ++ntl;
    };

    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(a.cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // the first tile's copies, and thread 0's bounded wait for them straight
    // after (its limit read before the copies are issued)
    int cur_q = -1;  // the problem of the tile in hand (its status word takes a timeout)
    if (tid == 0) {
        const int k = next_valid(e0);
        s_next = k;
        s_tload = 0;
        if (k < e1) {
            cur_q = entry(k).x;
            const long long lim = a.p[cur_q].wait_limit;
            load_t(entry(k).x);
            s_tload = 1;
            load_members(k, 0);
            if (!(mbar_wait(&bars[0], 0, lim) && mbar_wait(&bars[3], 0, lim))) s_abort = 1;
        }
    }
    __syncthreads();

    const bool two = a.nbuf == 2;
    int k = s_next, it = 0, tph = 0, ph = 0;  // ph bit b: parity of buffer b's next completion
    while (k < e1 && !s_abort) {
        const int b = two ? (it & 1) : 0;
        const int2 e = entry(k);
        const UpdateProb &P = a.p[e.x];
        cur_q = e.x;
        const bool tload = s_tload != 0;
        float *sm = smb + b * bstride;
        // a. the next tile's members into the other buffer
        if (tid == 0) {
            const int nk = next_valid(k + 1);
            s_next2 = nk;
            if (two && nk < e1) load_members(nk, b ^ 1);
        }
        // b. the operands: thread 0 waits with the handle's limit and decides
        // for the CTA (for the first tile it did so when it issued the copies);
        // the others then acquire the completed copies at once
        if (tid == 0 && it > 0) {
            bool ok = mbar_wait(&bars[b], (ph >> b) & 1, P.wait_limit);
            if (ok && tload) ok = mbar_wait(&bars[3], tph & 1, P.wait_limit);
            if (!ok) s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        mbar_wait(&bars[b], (ph >> b) & 1);
        if (tload) mbar_wait(&bars[3], tph & 1);
        if (tid == 0) {
            pend &= ~(1 << b);
            if (tload) pend_t = 0;
        }
        ph ^= 1 << b;
        tph += tload ? 1 : 0;
        const int nk = s_next2;
        // c. anomalies of point pl = tid mod 128: the mean as x_ref + dm,
        // x_ref = member 0's value and dm the mean of the differences
        // x_i - x_ref (exact for members within a factor 2 of each other), the
        // differences summed in FP32 per member slice i = q, q + 8, ... in
        // member order (half h = tid / 128 sums slices 4h .. 4h + 3 as four
        // independent chains), the slices in slice order; then the BF16 rows
        // ((x_i - x_ref) - dm) / sqrt(Ne - 1), K padding zero, granules split
        // between the halves.  The same operations as the CUDA-core anomaly
        // kernel, so both updates see identical operands.  Row pl of atom kb:
        // 8 granules of 16 bytes, granule g stored at g ^ (pl mod 8)
        {
            const int ne = P.ne, pl = tid & (kTileM - 1), half = tid >> 7;
            const float xr = sm[pl];
            float ps[4] = {0.f, 0.f, 0.f, 0.f};
            for (int i0 = 4 * half; i0 < ne; i0 += 8) {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
                    if (i0 + qq < ne) ps[qq] = __fadd_rn(ps[qq], __fsub_rn(sm[(i0 + qq) * kTileM + pl], xr));
            }
            if (half) {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) s_part[qq][pl] = ps[qq];
            }
            __syncthreads();
            if (!half) {
                float D = 0.f;
#pragma unroll
                for (int q = 0; q < 8; ++q) D = __fadd_rn(D, q < 4 ? ps[q] : s_part[q - 4][pl]);
                s_ref[pl] = make_float2(xr, __fmul_rn(D, (float)P.inv_ne));
            }
            __syncthreads();
            const float2 rf = s_ref[pl];
            const float isqf = (float)P.isq;
            const uint32_t sw = (uint32_t)(pl & 7);
            for (int gi = half; gi < P.kblocks * 8; gi += 2) {
                const int kb = gi >> 3, g = gi & 7;
                unsigned char *row = sa + (size_t)kb * kTileM * 128 + (size_t)pl * 128;
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int i0 = gi * 8 + 2 * h;
                    const float v0 =
                        i0 < ne ? __fmul_rn(__fsub_rn(__fsub_rn(sm[i0 * kTileM + pl], rf.x), rf.y), isqf) : 0.f;
                    const float v1 = i0 + 1 < ne
                                         ? __fmul_rn(__fsub_rn(__fsub_rn(sm[(i0 + 1) * kTileM + pl], rf.x), rf.y), isqf)
                                         : 0.f;
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v0, v1);  // v0 at the lower address
                    w[h] = *reinterpret_cast<const uint32_t *>(&b2);
                }
                *reinterpret_cast<uint4 *>(row + (((uint32_t)g ^ sw) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A is read by the MMA (async proxy)
        }
        __syncthreads();
        // d. D = A T^T
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = idesc_bf16(kTileM, P.ntile);
            const int ksteps = P.kblocks * (kAtomK / 16);
            for (int j = 0; j < ksteps; ++j) {
                const int kb = j / (kAtomK / 16), kk = j % (kAtomK / 16);
                const uint64_t adesc = smem_desc_sw128(smem_u32(sa + (size_t)kb * kTileM * 128 + kk * 32));
                const uint64_t bdesc = smem_desc_sw128(smem_u32(sb + (size_t)kb * P.ntile * 128 + kk * 32));
                mma_bf16(tmem, adesc, bdesc, idesc, j > 0 ? 1u : 0u);
            }
            mma_commit(&bars[2]);
        }
        if (!mbar_wait(&bars[2], it & 1)) s_abort = 1;  // default bound
        __syncthreads();
        if (s_abort) break;
        // e. T of the next problem (the MMAs reading T are complete)
        if (tid == 0) {
            s_tload = 0;
            if (nk < e1 && entry(nk).x != tq) {
                load_t(entry(nk).x);
                s_tload = 1;
            }
        }
        // f. epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its points)
        // and the 16-column chunks w / 4, w / 4 + 2, ...
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        {
            const int lq = warp & 3, pl = lq * 32 + lane, p = e.y * kTileM + pl, ne = P.ne, nx = P.nx;
            const uint32_t row = tmem + ((uint32_t)(lq * 32) << 16);
            for (int c0 = (warp >> 2) * 16; c0 < P.ntile; c0 += 32) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
                    : "r"(row + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (p < nx) {
                    float *mp = P.members + (size_t)c0 * nx + p;
                    const float *sp = sm + c0 * kTileM + pl;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int c = c0 + q;
                        const float v = __uint_as_float(r[q]);
                        if (c < ne)
                            mp[(size_t)q * nx] = sp[q * kTileM] + v;
                        else if (c == ne)
                            P.dC[p] = v;
                    }
                }
            }
        }
        // g. TMEM, A and this buffer are free for the next tiles
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (!two && tid == 0 && nk < e1) load_members(nk, 0);
        k = nk;
        ++it;
    }
    __syncthreads();
    if (s_abort && tid == 0) {
        if (cur_q >= 0) atomicCAS(a.p[cur_q].status, 0, kStTimeout);
        // let our own copies land (default bound) before the CTA exits
        for (int i = 0; i < 2; ++i)
            if ((pend >> i) & 1) mbar_wait(&bars[i], (lpar >> i) & 1);
        if (pend_t) mbar_wait(&bars[3], (ntl - 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.cols) : "memory");
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

size_t update_tc_smem(int kblocks, int ntpad, int ne, int nbuf) {
    // alignment slack, A, T, the member tiles, barriers and the TMEM slot
    return 1024 + (size_t)kblocks * (kTileM + ntpad) * 128 + (size_t)nbuf * ne * kTileM * 4 + 64;
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
    return update_tc_smem(kblocks, ntpad, ne, 1) <= 200 * 1024 && encode_fn() != nullptr;
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
    plan->smem = update_tc_launch_smem(update_tc_smem(plan->kblocks, ntpad, ne, 1), cols);
    plan->nx = nx;
    plan->ne = ne;
    plan->wait_limit = kWaitLimitCycles;
    if (!encode_kmajor(&plan->map_t, Tt, ldx, ntpad, ntpad)) return false;
    if (!encode_members(&plan->map_m, members, nx, ne)) return false;
    plan->members = members;
    plan->ready = true;
    return true;
}

// one launch of the persistent update over `nent` tiles of the problems
// args.p[0 .. nprob) (maps filled); its layout from their largest sizes
static cudaError_t update_launch(UpdateLaunchArgs &args, int nprob, const int2 *map, int nent, cudaStream_t s) {
    static OncePerDevice attr;
    cudaError_t e =
        attr.run([](int) { return cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); });
    if (e != cudaSuccess) return e;
    if (nent <= 0) return cudaSuccess;
    int kbmax = 1, ntmax = 16, nemax = 2;
    for (int q = 0; q < nprob; ++q) {
        kbmax = std::max(kbmax, args.p[q].kblocks);
        ntmax = std::max(ntmax, args.p[q].ntile);
        nemax = std::max(nemax, args.p[q].ne);
    }
    int cols = 32;
    while (cols < ntmax) cols <<= 1;
    args.kbmax = kbmax;
    args.ntmax = ntmax;
    args.nemax = nemax;
    args.cols = cols;
    args.nbuf = update_tc_smem(kbmax, ntmax, nemax, 2) <= 200 * 1024 ? 2 : 1;
    const size_t smem = update_tc_launch_smem(update_tc_smem(kbmax, ntmax, nemax, args.nbuf), cols);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    int dev = 0, sms = kNumSMs;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // CTAs per SM: 228 KB of shared memory per SM, 1 KB of it reserved per CTA
    // besides the kernel's static shared memory; 8 warps per CTA
    cudaFuncAttributes fa;
    const size_t stat = cudaFuncGetAttributes(&fa, k_update_tc) == cudaSuccess ? fa.sharedSizeBytes : 8192;
    const int per_sm = std::max(1, std::min(8, (int)((size_t)228 * 1024 / (smem + stat + 1024))));
    const int grid = std::min(nent, std::max(1, sms) * per_sm);
    count_launches(1);
    k_update_tc<<<grid, kUpdateThreads, smem, s>>>(args, map, nent);
    return cudaGetLastError();
}

UpdateProb update_tc_prob(const UpdateTcPlan &plan, float *dC, int *status) {
    UpdateProb p;
    p.members = const_cast<float *>(plan.members);
    p.dC = dC;
    p.status = status;
    p.nx = plan.nx;
    p.ne = plan.ne;
    p.kblocks = plan.kblocks;
    p.ntile = plan.ntile;
    p.wait_limit = plan.wait_limit;
    p.inv_ne = 1.0 / plan.ne;
    p.isq = 1.0 / std::sqrt((double)(plan.ne - 1));
    return p;
}

cudaError_t launch_update_tc(const UpdateTcPlan &plan, float *members, float *dC, int *status, cudaStream_t s) {
    if (members != plan.members) return cudaErrorInvalidValue;
    UpdateLaunchArgs args;
    memset(&args, 0, sizeof(args));
    args.m[0] = plan.map_t;
    args.m[1] = plan.map_m;
    args.p[0] = update_tc_prob(plan, dC, status);
    return update_launch(args, 1, nullptr, (plan.nx + kTileM - 1) / kTileM, s);
}

cudaError_t launch_update_tc_group(const GroupPlan &plan, cudaStream_t s) {
    UpdateLaunchArgs args;
    for (const GroupPlan::UpdateLaunch &L : plan.upd) {
        memset(&args, 0, sizeof(args));
        const int np = (int)L.probs.size();
        if (np > kUpdateLaunchMax) return cudaErrorInvalidValue;
        for (int q = 0; q < np; ++q) {
            const int j = L.probs[q];
            args.m[2 * q] = plan.upd_maps[2 * (size_t)j];
            args.m[2 * q + 1] = plan.upd_maps[2 * (size_t)j + 1];
            args.p[q] = plan.upd_probs[j];
        }
        cudaError_t e = update_launch(args, np, plan.d_maps + plan.map_off[kGsUpdate] + L.map_begin,
                                      L.map_end - L.map_begin, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mgk
