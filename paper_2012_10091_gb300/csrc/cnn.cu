// cnn.cu -- learned correction of the prolongation (residual CNN over Pi_F).
//
// Network: the 8 coarse channels [dC, x^C*] (normalised with fixed per-channel
// mean and scale) go through three 3x3 convolutions with periodic padding,
// 8 -> 32 -> 32 -> 64 channels, ReLU after the first two; the 64 output
// channels are pixel-shuffled by 4 into 4 fine channels, scaled per channel,
// and added to Pi_F(dC):
//   dF = Pi_F(dC) + s_out[c] * z3[16 c + 4 sy + sx][y][x]   at fine (4y + sy, 4x + sx).
// Training minimises mean(((dF - target) / s_out)^2) with Adam on FP32 master
// weights; the forward and backward passes use BF16 weights and activations
// with FP32 accumulation.
//
// Activations a0 (8 channels), a1, a2 (32) are BF16 in channel groups of 8
// ("C8": element (b, i, p) at ((b C/8 + i/8) n^2 + p) 8 + i % 8); z3 and the
// gradients are FP32 planes [b][c][p].
//
// Kernels:
//   k_cnn_input       normalised BF16 input, C8
//   k_conv_fwd_tc     the three forward convolutions on the tensor cores
//                     (conv_tc.cu: implicit GEMM, TMEM accumulators)
//   k_cnn_out_grad    residual, loss partials and dz3 through the shuffle
//   (one CTA per 16 x 16 pixel tile of one sample from here on)
//   k_conv_bwd_data   adjoint convolution, ReLU mask of the input
//   k_conv_bwd_weight per-tile partial dW, db; k_reduce_partials sums tiles in order
//   k_adam            Adam step on FP32 master weights, BF16 copy; the packed
//                     tensor-core copy of the weights follows every change
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mgenkf_ops.h"
#include "analysis.h"
#include "common.cuh"
#include "conv_tc.h"

namespace mgk {

constexpr int kT = 16;                    // pixel tile side
constexpr int kTH = kT + 2;               // with halo
constexpr int kCnnParams = 32 * 8 * 9 + 32 + 32 * 32 * 9 + 32 + 64 * 32 * 9 + 64;  // 30080

struct CnnLayer {
    int cin, cout;
    size_t w_off, b_off;  // offsets into the parameter vector
};
static const CnnLayer kLayers[3] = {{8, 32, 0, 2304}, {32, 32, 2336, 11552}, {32, 64, 11584, 30016}};

// element (b, i, p) of a C-channel BF16 activation in the C8 layout
__device__ __forceinline__ size_t c8_at(int b, int i, size_t p, int C, size_t pl) {
    return (((size_t)b * (C / 8) + i / 8) * pl + p) * 8 + (i & 7);
}

__device__ __forceinline__ int wrap(int v, int n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

// ---------------------------------------------------------------------------
__global__ void k_cnn_input(const float *__restrict__ dC, const float *__restrict__ xs, int n, int B,
                            const float *__restrict__ mu, const float *__restrict__ sc,
                            __nv_bfloat16 *__restrict__ a0) {
    const size_t pl = (size_t)n * n, total = (size_t)B * pl;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / pl, k = e % pl;
        uint4 pk;
        uint32_t *w = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = 2 * q + h;
                const float x = c < 4 ? dC[(b * 4 + c) * pl + k] : xs[(b * 4 + c - 4) * pl + k];
                v[h] = (x - mu[c]) / sc[c];
            }
            const __nv_bfloat162 two = __floats2bfloat162_rn(v[0], v[1]);
            w[q] = *reinterpret_cast<const uint32_t *>(&two);
        }
        reinterpret_cast<uint4 *>(a0)[e] = pk;  // C8 with one group: [b][p][8]
    }
}

// din[b][i][p] = (sum_{o,t} W[o][i][t] dout[b][o][p - tap t]) * (mask[b][i][p] > 0)
template <int CIN, int COUT, bool MASK>
__global__ void __launch_bounds__(256) k_conv_bwd_data(const float *__restrict__ dout,
                                                       const __nv_bfloat16 *__restrict__ W,
                                                       const __nv_bfloat16 *__restrict__ mask,
                                                       float *__restrict__ din, int n) {
    extern __shared__ __align__(16) unsigned char sm[];
    float *ds = reinterpret_cast<float *>(sm);                                    // [COUT][kTH][kTH]
    __nv_bfloat16 *ws = reinterpret_cast<__nv_bfloat16 *>(ds + COUT * kTH * kTH);  // [COUT][CIN][9]
    const int b = blockIdx.z, x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
    const size_t pl = (size_t)n * n;
    const float *db = dout + (size_t)b * COUT * pl;
    for (int e = threadIdx.x; e < COUT * kTH * kTH; e += blockDim.x) {
        const int o = e / (kTH * kTH), r = e % (kTH * kTH), ly = r / kTH, lx = r % kTH;
        const int gy = wrap(y0 + ly - 1, n), gx = wrap(x0 + lx - 1, n);
        ds[e] = db[o * pl + (size_t)gy * n + gx];
    }
    for (int e = threadIdx.x; e < COUT * CIN * 9; e += blockDim.x) ws[e] = W[e];
    __syncthreads();
    const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= n || y >= n) return;
    float acc[CIN];
#pragma unroll
    for (int i = 0; i < CIN; ++i) acc[i] = 0.f;
    for (int o = 0; o < COUT; ++o) {
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            // tap t = (dy+1)*3 + (dx+1): in[p] feeds out[p - (dy, dx)]
            const int dy = t / 3 - 1, dx = t % 3 - 1;
            const float v = ds[(o * kTH + ty - dy + 1) * kTH + tx - dx + 1];
#pragma unroll
            for (int i = 0; i < CIN; ++i) acc[i] = fmaf(__bfloat162float(ws[(o * CIN + i) * 9 + t]), v, acc[i]);
        }
    }
    const size_t p = (size_t)y * n + x;
#pragma unroll
    for (int i = 0; i < CIN; ++i) {
        float v = acc[i];
        if (MASK && !(__bfloat162float(mask[c8_at(b, i, p, CIN, pl)]) > 0.f)) v = 0.f;
        din[((size_t)b * CIN + i) * pl + p] = v;
    }
}

// per-tile partial sums: part[tile][(o*CIN + i)*9 + t] = sum_p dout[o][p] in[i][p + tap t],
// part[tile][COUT*CIN*9 + o] = sum_p dout[o][p]
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv_bwd_weight(const __nv_bfloat16 *__restrict__ in,
                                                         const float *__restrict__ dout,
                                                         float *__restrict__ part, int n) {
    extern __shared__ __align__(16) unsigned char sm[];
    float *xs = reinterpret_cast<float *>(sm);  // [CIN][kTH][kTH]
    float *ds = xs + CIN * kTH * kTH;           // [COUT][kT][kT]
    const int b = blockIdx.z, x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
    const size_t pl = (size_t)n * n;
    for (int e = threadIdx.x; e < CIN * kTH * kTH; e += blockDim.x) {
        const int i = e / (kTH * kTH), r = e % (kTH * kTH), ly = r / kTH, lx = r % kTH;
        const int gy = wrap(y0 + ly - 1, n), gx = wrap(x0 + lx - 1, n);
        xs[e] = __bfloat162float(in[c8_at(b, i, (size_t)gy * n + gx, CIN, pl)]);
    }
    for (int e = threadIdx.x; e < COUT * kT * kT; e += blockDim.x) {
        const int o = e / (kT * kT), r = e % (kT * kT), ly = r / kT, lx = r % kT;
        const int y = y0 + ly, x = x0 + lx;
        ds[e] = (y < n && x < n) ? dout[((size_t)b * COUT + o) * pl + (size_t)y * n + x] : 0.f;
    }
    __syncthreads();
    const int tiles = gridDim.x * gridDim.y;
    float *pt = part + ((size_t)b * tiles + blockIdx.y * gridDim.x + blockIdx.x) * (COUT * CIN * 9 + COUT);
    for (int q = threadIdx.x; q < COUT * CIN; q += blockDim.x) {
        const int o = q / CIN, i = q % CIN;
        float acc[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[t] = 0.f;
        for (int ly = 0; ly < kT; ++ly)
            for (int lx = 0; lx < kT; ++lx) {
                const float d = ds[(o * kT + ly) * kT + lx];
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[t] = fmaf(d, xs[(i * kTH + ly + t / 3) * kTH + lx + t % 3], acc[t]);
            }
#pragma unroll
        for (int t = 0; t < 9; ++t) pt[(size_t)q * 9 + t] = acc[t];
    }
    for (int o = threadIdx.x; o < COUT; o += blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < kT * kT; ++k) s += ds[o * kT * kT + k];
        pt[COUT * CIN * 9 + o] = s;
    }
}

__global__ void k_reduce_partials(const float *__restrict__ part, int nparts, int len, float *__restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int q = 0; q < nparts; ++q) s += part[(size_t)q * len + e];
        out[e] = s;
    }
}

// residual through the pixel shuffle; with a target: loss partials and dz3
__global__ void k_cnn_out_grad(const float *__restrict__ z3, int n, int B, const float *__restrict__ s_out,
                               const float *__restrict__ tres, float *__restrict__ res, int accumulate,
                               float *__restrict__ dz3, float *__restrict__ loss_part, float inv_count) {
    const int nf = 4 * n;
    const size_t pf = (size_t)nf * nf, pl = (size_t)n * n, total = (size_t)B * 4 * pf;
    float lsum = 0.f;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / (4 * pf), r = e % (4 * pf);
        const int c = (int)(r / pf);
        const size_t k = r % pf;
        const int fy = (int)(k / nf), fx = (int)(k % nf);
        const int ch = 16 * c + 4 * (fy & 3) + (fx & 3);
        const size_t zi = ((size_t)b * 64 + ch) * pl + (size_t)(fy >> 2) * n + (fx >> 2);
        const float v = s_out[c] * z3[zi];
        if (res) res[e] = accumulate ? res[e] + v : v;
        if (tres) {
            const float d = (v - tres[e]) / s_out[c];
            lsum += d * d;
            dz3[zi] = 2.f * d * inv_count;
        }
    }
    if (tres) {
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
        __shared__ float red[8];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.f;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
            loss_part[blockIdx.x] = s * inv_count;
        }
    }
}

__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, __nv_bfloat16 *__restrict__ w16, int len, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        const float wi = w[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[e] = wi;
        w16[e] = __float2bfloat16(wi);
    }
}

__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, int len) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x)
        b[e] = __float2bfloat16(a[e]);
}

__global__ void k_sub_prolong(const float *__restrict__ target, float *__restrict__ tres, size_t len) {
    // tres already holds -Pi_F(dC); tres = target - Pi_F(dC)
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
        tres[e] += target[e];
}

__global__ void k_zero_fill(float *__restrict__ a, size_t len) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
        a[e] = 0.f;
}

__global__ void k_negate(float *__restrict__ a, size_t len) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
        a[e] = -a[e];
}

}  // namespace mgk

// ===========================================================================
// C ABI: the learned-correction object
// ===========================================================================
using namespace mgk;

struct mgk_cnn {
    int nc, bmax;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // FP32 master, Adam, grads
    __nv_bfloat16 *w16 = nullptr;
    float *stats = nullptr;  // mu_in[8], s_in[8], s_out[4]
    __nv_bfloat16 *a0 = nullptr, *a1 = nullptr, *a2 = nullptr;
    float *z3 = nullptr, *d3 = nullptr, *d2 = nullptr, *d1 = nullptr, *tres = nullptr, *res = nullptr;
    float *part = nullptr, *loss_part = nullptr;
    __nv_bfloat16 *wp = nullptr;  // tensor-core copies of the three layers' weights (conv_tc.cu)
    int *zero_status = nullptr;  // an always-zero status word for the shared prolongation kernel
    int *status = nullptr;       // MGENKF_ERR_TIMEOUT from a tensor-core wait, sticky
    int step = 0;
    std::string err;
};

static int tiles_of(int n) { return (n + kT - 1) / kT; }

// packed tensor-core weights: layer l starts at wp_off(l) elements (16-byte aligned)
static int wp_off(int l) {
    int o = 0;
    for (int q = 0; q < l; ++q) o += conv_packed_elems(kLayers[q].cin, kLayers[q].cout);
    return o;
}
static int wp_elems() { return wp_off(3); }

static void pack_weights(mgk_cnn *c, cudaStream_t s) {
    for (int l = 0; l < 3; ++l)
        launch_pack_conv_weights(c->w16 + kLayers[l].w_off, kLayers[l].cin, kLayers[l].cout, c->wp + wp_off(l), s);
}

template <int CIN, int COUT>
static size_t smem_bwd_data() { return sizeof(float) * COUT * kTH * kTH + sizeof(__nv_bfloat16) * COUT * CIN * 9; }
template <int CIN, int COUT>
static size_t smem_bwd_w() { return sizeof(float) * (CIN * kTH * kTH + COUT * kT * kT); }

static void set_smem_attrs() {
    static OncePerDevice once;
    once.run([](int) {
        const int b = 200 * 1024;
        cudaError_t e = cudaFuncSetAttribute(k_conv_bwd_data<32, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_bwd_data<32, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_bwd_weight<32, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_bwd_weight<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_bwd_weight<8, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        return e;
    });
}

static void cnn_free(mgk_cnn *c) {
    void *ptrs[] = {c->w, c->m, c->v, c->g, c->w16, c->stats, c->a0, c->a1, c->a2, c->z3, c->d3,
                    c->d2, c->d1, c->tres, c->res, c->part, c->loss_part, c->wp, c->zero_status, c->status};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

extern "C" mgenkf_status mgk_cnn_create(int32_t n_coarse, int32_t batch_max, mgk_cnn_t *out) {
    if (!out) return MGENKF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_coarse < 1 || n_coarse > 1024 || batch_max < 1 || batch_max > 256) {
        mgk_set_error("mgk_cnn_create: n_coarse must be in [1, 1024] and batch_max in [1, 256]");
        return MGENKF_ERR_INVALID_ARG;
    }
    mgk_cnn *c = new mgk_cnn();
    c->nc = n_coarse;
    c->bmax = batch_max;
    const size_t pl = (size_t)n_coarse * n_coarse, B = batch_max;
    const size_t tiles = (size_t)tiles_of(n_coarse) * tiles_of(n_coarse) * B;
    const size_t plen = (size_t)64 * 32 * 9 + 64;  // largest layer's partial
    struct A {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&c->w, kCnnParams * sizeof(float)},   {(void **)&c->m, kCnnParams * sizeof(float)},
        {(void **)&c->v, kCnnParams * sizeof(float)},   {(void **)&c->g, kCnnParams * sizeof(float)},
        {(void **)&c->w16, kCnnParams * 2},             {(void **)&c->stats, 20 * sizeof(float)},
        {(void **)&c->a0, B * 8 * pl * 2},              {(void **)&c->a1, B * 32 * pl * 2},
        {(void **)&c->a2, B * 32 * pl * 2},             {(void **)&c->z3, B * 64 * pl * 4},
        {(void **)&c->d3, B * 64 * pl * 4},             {(void **)&c->d2, B * 32 * pl * 4},
        {(void **)&c->d1, B * 32 * pl * 4},             {(void **)&c->tres, B * 4 * 16 * pl * 4},
        {(void **)&c->res, B * 4 * 16 * pl * 4},        {(void **)&c->part, tiles * plen * 4},
        {(void **)&c->loss_part, 4096 * sizeof(float)},  {(void **)&c->zero_status, sizeof(int)},
        {(void **)&c->wp, (size_t)wp_elems() * 2},         {(void **)&c->status, sizeof(int)},
    };
    for (auto &a : allocs) {
        if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            mgk_set_error("mgk_cnn_create: device allocation failed");
            cnn_free(c);
            delete c;
            return MGENKF_ERR_OOM;
        }
    }
    cudaMemset(c->w, 0, kCnnParams * sizeof(float));
    cudaMemset(c->m, 0, kCnnParams * sizeof(float));
    cudaMemset(c->v, 0, kCnnParams * sizeof(float));
    cudaMemset(c->w16, 0, kCnnParams * 2);
    cudaMemset(c->zero_status, 0, sizeof(int));
    cudaMemset(c->status, 0, sizeof(int));
    cudaMemset(c->wp, 0, (size_t)wp_elems() * 2);
    const float st[20] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    cudaMemcpy(c->stats, st, sizeof(st), cudaMemcpyHostToDevice);
    set_smem_attrs();
    if (cudaDeviceSynchronize() != cudaSuccess) {
        mgk_set_error("mgk_cnn_create: CUDA error during set-up");
        cnn_free(c);
        delete c;
        return MGENKF_ERR_CUDA;
    }
    *out = c;
    return MGENKF_OK;
}

extern "C" int32_t mgk_cnn_coarse_size(mgk_cnn_t c) { return c ? c->nc : 0; }

extern "C" mgenkf_status mgk_cnn_destroy(mgk_cnn_t c) {
    if (!c) return MGENKF_OK;
    cudaDeviceSynchronize();
    cnn_free(c);
    delete c;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgk_cnn_set_params(mgk_cnn_t c, const float *params, const float *stats) {
    if (!c) return MGENKF_ERR_INVALID_ARG;
    if (params) {
        if (cudaMemcpy(c->w, params, kCnnParams * sizeof(float), cudaMemcpyDefault) != cudaSuccess) return MGENKF_ERR_CUDA;
        cudaMemset(c->m, 0, kCnnParams * sizeof(float));
        cudaMemset(c->v, 0, kCnnParams * sizeof(float));
        c->step = 0;
        count_launches(1);
        k_to_bf16<<<64, 256>>>(c->w, c->w16, kCnnParams);
        pack_weights(c, 0);
    }
    if (stats && cudaMemcpy(c->stats, stats, 20 * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
        return MGENKF_ERR_CUDA;
    return cudaDeviceSynchronize() == cudaSuccess ? MGENKF_OK : MGENKF_ERR_CUDA;
}

extern "C" mgenkf_status mgk_cnn_get_params(mgk_cnn_t c, float *params, float *grads) {
    if (!c) return MGENKF_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return MGENKF_ERR_CUDA;  // training launches on any stream
    int st = 0;
    if (cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MGENKF_ERR_CUDA;
    if (st) {
        mgk_set_error("mgk_cnn: a tensor-core wait expired in an earlier call");
        return (mgenkf_status)st;
    }
    if (params && cudaMemcpy(params, c->w, kCnnParams * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
        return MGENKF_ERR_CUDA;
    if (grads && cudaMemcpy(grads, c->g, kCnnParams * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
        return MGENKF_ERR_CUDA;
    return MGENKF_OK;
}

// forward of B samples; fills c->z3 (and c->a0..a2)
static void cnn_forward_impl(mgk_cnn *c, const float *dC, const float *xs, int B, int *status, cudaStream_t s) {
    const int n = c->nc;
    const float *mu = c->stats, *sc = c->stats + 8;
    count_launches(1);
    k_cnn_input<<<256, 256, 0, s>>>(dC, xs, n, B, mu, sc, c->a0);
    launch_conv_fwd_tc<8, 32, true, true>(c->a0, c->wp + wp_off(0), c->w + kLayers[0].b_off, c->a1, n, B, status, s);
    launch_conv_fwd_tc<32, 32, true, true>(c->a1, c->wp + wp_off(1), c->w + kLayers[1].b_off, c->a2, n, B, status, s);
    launch_conv_fwd_tc<32, 64, false, false>(c->a2, c->wp + wp_off(2), c->w + kLayers[2].b_off, c->z3, n, B, status,
                                             s);
}

namespace mgk {
mgenkf_status cnn_forward_status(mgk_cnn_t c, const float *dC, const float *xstar, int batch, float *residual,
                                 int accumulate, int *status, cudaStream_t s) {
    if (!c || !dC || !xstar || !residual || batch < 1 || batch > c->bmax) return MGENKF_ERR_INVALID_ARG;
    cnn_forward_impl(c, dC, xstar, batch, status, s);
    count_launches(1);
    k_cnn_out_grad<<<512, 256, 0, s>>>(c->z3, c->nc, batch, c->stats + 16, nullptr, residual, accumulate, nullptr,
                                       nullptr, 0.f);
    return cudaGetLastError() == cudaSuccess ? MGENKF_OK : MGENKF_ERR_CUDA;
}
}  // namespace mgk

extern "C" mgenkf_status mgk_cnn_forward(mgk_cnn_t c, const float *dC, const float *xstar, int32_t batch,
                                         float *residual, int32_t accumulate, void *stream) {
    if (!c) return MGENKF_ERR_INVALID_ARG;
    return cnn_forward_status(c, dC, xstar, batch, residual, accumulate, c->status, (cudaStream_t)stream);
}

extern "C" mgenkf_status mgk_cnn_loss_grad(mgk_cnn_t c, const float *dC, const float *xstar, const float *target,
                                           int32_t batch, float *loss_out, void *stream) {
    if (!c || !dC || !xstar || !target || batch < 1 || batch > c->bmax) return MGENKF_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    const int n = c->nc, B = batch;
    const size_t pl = (size_t)n * n, fine = (size_t)B * 4 * 16 * pl;
    // target residual over Pi_F(dC): tres = target - Pi_F(dC)
    ProlongWeights pw;
    for (int m = 0; m < 4; ++m) {
        const double sv = m / 4.0;
        pw.w[m][0] = -sv * (sv - 1.0) * (sv - 2.0) / 6.0;
        pw.w[m][1] = (sv + 1.0) * (sv - 1.0) * (sv - 2.0) / 2.0;
        pw.w[m][2] = -(sv + 1.0) * sv * (sv - 2.0) / 2.0;
        pw.w[m][3] = (sv + 1.0) * sv * (sv - 1.0) / 6.0;
    }
    count_launches(2);
    k_zero_fill<<<512, 256, 0, s>>>(c->tres, fine);
    for (int b = 0; b < B; ++b)
        launch_prolong_add<float>(c->tres + (size_t)b * 4 * 16 * pl, dC + (size_t)b * 4 * pl, 2, 4, n, 4, pw,
                                  c->zero_status, s);
    k_negate<<<512, 256, 0, s>>>(c->tres, fine);
    count_launches(1);
    k_sub_prolong<<<512, 256, 0, s>>>(target, c->tres, fine);
    cnn_forward_impl(c, dC, xstar, B, c->status, s);
    count_launches(1);
    const float inv_count = 1.f / (float)fine;
    k_cnn_out_grad<<<512, 256, 0, s>>>(c->z3, n, B, c->stats + 16, c->tres, c->res, 0, c->d3, c->loss_part,
                                       inv_count);
    const dim3 grid(tiles_of(n), tiles_of(n), B);
    const int nparts = tiles_of(n) * tiles_of(n) * B;
    // layer 3: dW3, db3 and d(a2) masked by a2 > 0
    count_launches(9);
    k_conv_bwd_weight<32, 64><<<grid, 256, smem_bwd_w<32, 64>(), s>>>(c->a2, c->d3, c->part, n);
    k_reduce_partials<<<128, 256, 0, s>>>(c->part, nparts, 64 * 32 * 9 + 64, c->g + kLayers[2].w_off);
    k_conv_bwd_data<32, 64, true><<<grid, 256, smem_bwd_data<32, 64>(), s>>>(c->d3, c->w16 + kLayers[2].w_off,
                                                                            c->a2, c->d2, n);
    // layer 2
    k_conv_bwd_weight<32, 32><<<grid, 256, smem_bwd_w<32, 32>(), s>>>(c->a1, c->d2, c->part, n);
    k_reduce_partials<<<128, 256, 0, s>>>(c->part, nparts, 32 * 32 * 9 + 32, c->g + kLayers[1].w_off);
    k_conv_bwd_data<32, 32, true><<<grid, 256, smem_bwd_data<32, 32>(), s>>>(c->d2, c->w16 + kLayers[1].w_off,
                                                                            c->a1, c->d1, n);
    // layer 1 (no input gradient)
    k_conv_bwd_weight<8, 32><<<grid, 256, smem_bwd_w<8, 32>(), s>>>(c->a0, c->d1, c->part, n);
    k_reduce_partials<<<128, 256, 0, s>>>(c->part, nparts, 32 * 8 * 9 + 32, c->g + kLayers[0].w_off);
    k_reduce_partials<<<1, 256, 0, s>>>(c->loss_part, 512, 1, c->loss_part + 1024);
    if (loss_out) {
        if (cudaMemcpyAsync(loss_out, c->loss_part + 1024, sizeof(float), cudaMemcpyDefault, s) != cudaSuccess)
            return MGENKF_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? MGENKF_OK : MGENKF_ERR_CUDA;
}

extern "C" mgenkf_status mgk_cnn_adam_step(mgk_cnn_t c, float lr, void *stream) {
    if (!c || !(lr > 0.f)) return MGENKF_ERR_INVALID_ARG;
    c->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)c->step), c2 = 1.f - powf(b2, (float)c->step);
    count_launches(1);
    k_adam<<<128, 256, 0, (cudaStream_t)stream>>>(c->w, c->m, c->v, c->g, c->w16, kCnnParams, lr, b1, b2, 1e-8f, c1, c2);
    pack_weights(c, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? MGENKF_OK : MGENKF_ERR_CUDA;
}
