// conv_tc.cu -- the 3x3 periodic convolutions of the learned correction on the
// tensor cores (tcgen05), as an implicit GEMM with no im2col copy.
//
// Activations are stored in channel groups of 8 ("C8"): element (b, i, p) of a
// C-channel n x n map sits at ((b C/8 + i/8) n^2 + p) 8 + i % 8, so the 8
// channels of one group at one pixel are 16 contiguous bytes.
//
// A CTA computes ROWS output rows x 128 pixels x COUT channels of one sample:
//   * the input block (ROWS + 2 rows x 130 pixels, periodic wrap) is copied to
//     shared memory as one plane per channel group with pixels 16 bytes apart.
//     That is the no-swizzle K-major operand layout (a core matrix = 8 pixels x
//     8 channels = 128 contiguous bytes; the next 8 pixels 128 bytes on, the
//     next 8 channels one plane on), so the A operand of tap (dy, dx) for
//     output row r is the same planes with the start moved to pixel
//     (r + dy, dx): nine taps, nine start addresses, no copies;
//   * the packed weights [tap][group][COUT][8] (k_pack_conv_weights) are the
//     B operands in the same layout;
//   * one thread issues ROWS x 9 x CIN/16 MMAs (M = 128 pixels, N = COUT,
//     K = 16 channels), each output row accumulating in its own TMEM columns,
//     and commits them to an mbarrier;
//   * the four warps read back their 32 TMEM lanes (pixels), add the bias,
//     apply the ReLU and store BF16 C8 (hidden layers) or FP32 planes
//     (the last layer, read by the pixel shuffle).
// CIN = 8 is padded to K = 16 with a zero plane and zero weights.  Rows and
// pixels past the map's edge are computed from wrapped inputs and not stored.
// The mbarrier wait is bounded; on expiry the kernel records
// MGENKF_ERR_TIMEOUT in the status word, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "conv_tc.h"
#include "tc_common.cuh"

namespace mgk {

namespace {

constexpr int kPix = 128;        // output pixels per MMA (M)
constexpr int kRowW = 136;       // smem pixels per input row (130 used)
constexpr int kConvRows = 4;     // output rows per CTA

template <int CIN, int COUT>
struct ConvTcShape {
    static constexpr int CGI = CIN / 8;                 // input channel groups held in global memory
    static constexpr int CGK = CIN < 16 ? 2 : CIN / 8;  // channel groups of K (padded to 16 channels)
    static constexpr int PLANE = (kConvRows + 2) * kRowW * 16;  // bytes per channel-group plane
    static constexpr int IN_BYTES = CGK * PLANE;
    static constexpr int W_BYTES = 9 * CGK * COUT * 16;
    static constexpr int COLS_USED = kConvRows * COUT;
    static constexpr int TMEM_COLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128 : 256;
    static_assert(COLS_USED <= 256, "accumulators of one CTA fit 256 TMEM columns");
    static_assert(COUT % 16 == 0 && COUT >= 16 && COUT <= 256, "N of an M = 128 MMA");
    static_assert(CIN == 8 || CIN % 16 == 0, "channel groups of 8, K steps of 16");
    // at most 512 / TMEM_COLS CTAs may share an SM's TMEM: ask for enough
    // shared memory that no more are resident, so no CTA waits in alloc
    static constexpr int MIN_SMEM = 228 * 1024 / (512 / TMEM_COLS + 1) + 2048;
    static constexpr int NEED = 1024 + IN_BYTES + W_BYTES + 64;
    static constexpr int SMEM = NEED > MIN_SMEM ? NEED : MIN_SMEM;
};

__device__ __forceinline__ int wrap_c8(int v, int n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

__device__ __forceinline__ void cp_async16_cg(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_u32(smem)), "l"(gmem) : "memory");
}

}  // namespace

// packed[t][g][o][j] = W[o][8g + j][t] (0 past CIN), W in [COUT][CIN][9] order
__global__ void k_pack_conv_weights(const __nv_bfloat16 *__restrict__ W, int cin, int cout, int cgk,
                                    __nv_bfloat16 *__restrict__ packed) {
    const int total = 9 * cgk * cout * 8;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int j = e % 8, o = (e / 8) % cout, g = (e / (8 * cout)) % cgk, t = e / (8 * cout * cgk);
        const int ch = 8 * g + j;
        packed[e] = ch < cin ? W[((size_t)o * cin + ch) * 9 + t] : __float2bfloat16(0.f);
    }
}

template <int CIN, int COUT, bool RELU, bool OUT_BF16>
__global__ void __launch_bounds__(128) k_conv_fwd_tc(const __nv_bfloat16 *__restrict__ in,
                                                     const __nv_bfloat16 *__restrict__ wp,
                                                     const float *__restrict__ bias, void *__restrict__ out, int n,
                                                     int *status) {
    using S = ConvTcShape<CIN, COUT>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sin = base;                  // CGK planes of (ROWS + 2) x kRowW pixels x 16 bytes
    unsigned char *sw = base + S::IN_BYTES;     // [9][CGK][COUT][8] bf16
    uint64_t *bar = reinterpret_cast<uint64_t *>(sw + S::W_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z, x0 = blockIdx.x * kPix, y0 = blockIdx.y * kConvRows;
    const size_t pl = (size_t)n * n;
    if (tid == 0) {
        s_fail = status ? *status : 0;  // one read: the whole CTA leaves or none of it
        tc::mbar_init(bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (s_fail) return;
    // input block: plane g, row r (map row y0 - 1 + r), pixel j (map column x0 - 1 + j)
    constexpr int IN_CHUNKS = S::CGI * (kConvRows + 2) * (kPix + 2);
    const __nv_bfloat16 *inb = in + (size_t)b * S::CGI * pl * 8;
    for (int e = tid; e < IN_CHUNKS; e += 128) {
        const int j = e % (kPix + 2), r = (e / (kPix + 2)) % (kConvRows + 2), g = e / ((kPix + 2) * (kConvRows + 2));
        const int gy = wrap_c8(y0 - 1 + r, n), gx = wrap_c8(x0 - 1 + j, n);
        cp_async16_cg(sin + g * S::PLANE + (r * kRowW + j) * 16, inb + ((size_t)g * pl + (size_t)gy * n + gx) * 8);
    }
    if (S::CGK > S::CGI) {  // zero planes of the K padding
        for (int e = tid; e < (S::CGK - S::CGI) * (kConvRows + 2) * kRowW; e += 128)
            reinterpret_cast<uint4 *>(sin + S::CGI * S::PLANE)[e] = make_uint4(0, 0, 0, 0);
    }
    for (int e = tid; e < S::W_BYTES / 16; e += 128) cp_async16_cg(sw + e * 16, wp + (size_t)e * 8);
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    // generic-proxy writes of shared memory, then read by the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) tc::tmem_alloc(tmem_slot, S::TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const int rows = min(kConvRows, n - y0);

    if (tid == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16(kPix, COUT);
        const uint32_t a0 = tc::smem_u32(sin), b0 = tc::smem_u32(sw);
        for (int r = 0; r < rows; ++r) {
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3, dx = t % 3;
#pragma unroll
                for (int s = 0; s < S::CGK / 2; ++s) {
                    const uint64_t ad = tc::smem_desc_interleave(
                        a0 + (uint32_t)(2 * s * S::PLANE + ((r + dy) * kRowW + dx) * 16), S::PLANE, 128);
                    const uint64_t bd =
                        tc::smem_desc_interleave(b0 + (uint32_t)((t * S::CGK + 2 * s) * COUT * 16), COUT * 16, 128);
                    tc::mma_bf16(tmem + (uint32_t)(r * COUT), ad, bd, idesc, (t | s) ? 1u : 0u);
                }
            }
        }
        tc::mma_commit(bar);
    }
    __syncthreads();
    // warp-uniform: the TMEM loads below are warp-collective
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(bar, 0));
    if (!ok) {
        if (lane == 0 && status) atomicCAS(status, 0, tc::kStTimeout);
    } else {
        tc::fence_after_sync();
        const int x = x0 + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int r = 0; r < rows; ++r) {
            const size_t p = (size_t)(y0 + r) * n + x;
#pragma unroll
            for (int c0 = 0; c0 < COUT; c0 += 16) {
                float v[16];
                tc::tmem_ld16(lane_base + (uint32_t)(r * COUT + c0), v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    v[q] += __ldg(bias + c0 + q);
                    if (RELU) v[q] = fmaxf(v[q], 0.f);
                }
                if (x < n) {
                    if (OUT_BF16) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            uint4 pk;
                            uint32_t *w = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const __nv_bfloat162 two = __floats2bfloat162_rn(v[8 * h + 2 * q], v[8 * h + 2 * q + 1]);
                                w[q] = *reinterpret_cast<const uint32_t *>(&two);
                            }
                            const int g = (c0 >> 3) + h;
                            reinterpret_cast<uint4 *>(out)[((size_t)b * (COUT / 8) + g) * pl + p] = pk;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            reinterpret_cast<float *>(out)[((size_t)b * COUT + c0 + q) * pl + p] = v[q];
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

template <int CIN, int COUT, bool RELU, bool OUT_BF16>
cudaError_t launch_conv_fwd_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *wp, const float *bias, void *out, int n,
                               int batch, int *status, cudaStream_t s) {
    using S = ConvTcShape<CIN, COUT>;
    static OncePerDevice attr;
    attr.run([](int) {
        return cudaFuncSetAttribute(k_conv_fwd_tc<CIN, COUT, RELU, OUT_BF16>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    });
    count_launches(1);
    const dim3 grid(ceil_div(n, kPix), ceil_div(n, kConvRows), batch);
    k_conv_fwd_tc<CIN, COUT, RELU, OUT_BF16><<<grid, 128, S::SMEM, s>>>(in, wp, bias, out, n, status);
    return cudaGetLastError();
}

int conv_packed_elems(int cin, int cout) { return 9 * (cin < 16 ? 2 : cin / 8) * cout * 8; }

cudaError_t launch_pack_conv_weights(const __nv_bfloat16 *W, int cin, int cout, __nv_bfloat16 *packed,
                                     cudaStream_t s) {
    count_launches(1);
    k_pack_conv_weights<<<ceil_div(conv_packed_elems(cin, cout), 256), 256, 0, s>>>(W, cin, cout,
                                                                                  cin < 16 ? 2 : cin / 8, packed);
    return cudaGetLastError();
}

template cudaError_t launch_conv_fwd_tc<8, 32, true, true>(const __nv_bfloat16 *, const __nv_bfloat16 *,
                                                           const float *, void *, int, int, int *, cudaStream_t);
template cudaError_t launch_conv_fwd_tc<32, 32, true, true>(const __nv_bfloat16 *, const __nv_bfloat16 *,
                                                            const float *, void *, int, int, int *, cudaStream_t);
template cudaError_t launch_conv_fwd_tc<32, 64, false, false>(const __nv_bfloat16 *, const __nv_bfloat16 *,
                                                              const float *, void *, int, int, int *, cudaStream_t);

}  // namespace mgk
