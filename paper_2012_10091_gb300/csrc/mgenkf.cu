// mgenkf.cu -- host implementation of the C ABI declared in include/mgenkf.h
// and include/mgenkf_ops.h.  Owns the device buffers of one MGEnKF run and
// sequences the kernels of a cycle (Algorithm 4) on the handle's stream.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mgenkf.h"
#include "../../include/mgenkf_ops.h"
#include "analysis.h"
#include "batch_analysis.h"
#include "common.cuh"
#include "forecast.h"
#include "forecast_ns2d.h"
#include "update_tc.h"

using namespace mgk;

static thread_local std::string g_ops_error;
static std::atomic<uint64_t> g_launches{0};
void mgk::count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
void mgk_set_error(const std::string &msg) { g_ops_error = msg; }

struct mgenkf_ctx {
    mgenkf_config cfg;
    int dim, V, nf, nc, r, ne, ny, taps;
    size_t nx, nxf, cpl;
    bool mixed, direct;
    cudaStream_t stream;
    int device;
    uint64_t cycle;
    std::string err;

    void *fine = nullptr, *members = nullptr, *xstar = nullptr, *dC = nullptr;
    int32_t *tap_idx = nullptr;
    double *tap_w = nullptr;
    float *tap_wh = nullptr, *tap_wl = nullptr;  // mixed precision: the weights split into FP32 pairs
    ProlongWeights pw;
    double *yf = nullptr, *yo = nullptr, *ybar = nullptr, *eps = nullptr, *Y = nullptr, *Z = nullptr;
    double *X64 = nullptr;
    __nv_bfloat16 *X16 = nullptr, *Tt = nullptr;
    int ldx = 0, ntpad = 0;
    double *S = nullptr, *Lt = nullptr, *Bt = nullptr;  // ensemble form: S (ne x ne), T in Bt
    double *C = nullptr, *Ct = nullptr, *W = nullptr;   // direct form
    double *Tm = nullptr;                               // T, (ne+1) x ne (points at Bt or own buffer)
    double *truth_d = nullptr, *rmse_part = nullptr, *rmse_d = nullptr, *scratch = nullptr;
    void *ns_scratch = nullptr;  // NS-2D stage buffers
    void *fine_prev = nullptr;   // fine state one model step before the end of the last forecast
    void *fine_tmp = nullptr;    // output of the final fine iteration
    double alpha = 0.0;          // relaxation of the final fine iteration (0: none)
    bool record_prev = false;    // forecasts record fine_prev (regularisation enabled)
    bool have_prev = false;      // fine_prev belongs to the current fine state
    bool recentre = false;       // re-centre the forecast ensemble on x^C* before each analysis
    double filter_sigma = 0.0;   // NS: sixth-order filter after every model step (0: off)
    double *gemm_part = nullptr; // split-K partial sums of the gain GEMMs
    DfOperands df;               // mixed precision, ensemble form: double-FP32 copies of Y and Z
    UpdateTcPlan tc;             // tensor-core member update (mixed precision)
    mgk_cnn_t cnn = nullptr;     // learned correction added by prolong_correct (not owned)
    size_t scratch_n = 0;
    int *status = nullptr;
    uint64_t *cycle_d = nullptr;  // analysis counter on the device (keys the perturbation stream)
    // mgenkf_cycle with a host truth: its copy runs on cstream beside the forecast
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_prev = nullptr, ev_truth = nullptr;
    // mixed NS-2D forecast: a column-march choice per grid (members, fine run;
    // ns2d_march_layout), or -1 for both (the 2-D tile kernel), the device
    // table of the two groups for it, the fine run's stream and the events
    // that fork it from and join it to the handle's stream
    int fc_choice[2] = {-1, -1};
    int fc_units[2] = {0, 0};
    NsGroup<float> *d_fc = nullptr;
    cudaStream_t fstream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
#define H_FAIL(code, msg)      \
    do {                       \
        h->err = (msg);        \
        return (code);         \
    } while (0)

#define H_CUDA(call)                                                                 \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
            return e_ == cudaErrorMemoryAllocation ? MGENKF_ERR_OOM : MGENKF_ERR_CUDA; \
        }                                                                            \
    } while (0)

#define H_LAUNCHED()                                                             \
    do {                                                                         \
        cudaError_t e_ = cudaGetLastError();                                     \
        if (e_ != cudaSuccess) {                                                 \
            h->err = std::string("kernel launch: ") + cudaGetErrorString(e_);    \
            return MGENKF_ERR_CUDA;                                              \
        }                                                                        \
    } while (0)

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// closed-form weights of the 4-point Lagrange interpolant on nodes -1, 0, 1, 2
static void cubic_weights(double s, double w[4]) {
    w[0] = -s * (s - 1.0) * (s - 2.0) / 6.0;
    w[1] = (s + 1.0) * (s - 1.0) * (s - 2.0) / 2.0;
    w[2] = -(s + 1.0) * s * (s - 2.0) / 2.0;
    w[3] = (s + 1.0) * s * (s - 1.0) / 6.0;
}

static size_t tsize(const mgenkf_ctx *h) { return h->mixed ? sizeof(float) : sizeof(double); }

template <typename P>
static mgenkf_status dalloc(mgenkf_ctx *h, P **p, size_t bytes) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e);
        return MGENKF_ERR_OOM;
    }
    *p = (P *)q;
    return MGENKF_OK;
}

#define H_ALLOC(ptr, bytes)                                    \
    do {                                                       \
        mgenkf_status s_ = dalloc(h, &(ptr), (bytes));         \
        if (s_ != MGENKF_OK) return s_;                        \
    } while (0)

static void free_all(mgenkf_ctx *h) {
    void *ptrs[] = {h->fine, h->members, h->xstar, h->dC, h->tap_idx, h->tap_w, h->tap_wh, h->tap_wl, h->yf, h->yo,
                    h->ybar, h->eps, h->Y, h->Z, h->X64, h->X16, h->Tt, h->S, h->Lt, h->Bt, h->C,
                    h->Ct, h->W, h->truth_d, h->rmse_part, h->rmse_d, h->scratch, h->status,
                    h->ns_scratch, h->gemm_part, h->cycle_d, h->fine_prev, h->fine_tmp,
                    h->df.Yh, h->df.Yl, h->df.Zh, h->df.Zl, h->d_fc};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->Tm && h->Tm != h->Bt) cudaFree(h->Tm);
    if (h->cstream) cudaStreamDestroy(h->cstream);
    if (h->ev_prev) cudaEventDestroy(h->ev_prev);
    if (h->ev_truth) cudaEventDestroy(h->ev_truth);
    if (h->fstream) cudaStreamDestroy(h->fstream);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
}

// copy n doubles from a host or device pointer into device buffer dst (FP64)
static mgenkf_status upload_f64(mgenkf_ctx *h, double *dst, const double *src, size_t n) {
    H_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, h->stream));
    return MGENKF_OK;
}

static mgenkf_status ensure_scratch(mgenkf_ctx *h, size_t n) {
    if (h->scratch_n >= n) return MGENKF_OK;
    if (h->scratch) cudaFree(h->scratch);
    h->scratch = nullptr;
    h->scratch_n = 0;
    H_ALLOC(h->scratch, n * sizeof(double));
    h->scratch_n = n;
    return MGENKF_OK;
}

// load n FP64 values (host or device) into a state buffer of the handle's type
static mgenkf_status load_state(mgenkf_ctx *h, void *dst, const double *src, size_t n) {
    if (!h->mixed) return upload_f64(h, (double *)dst, src, n);
    const double *dsrc = src;
    if (!is_device_ptr(src)) {
        mgenkf_status st = ensure_scratch(h, n);
        if (st) return st;
        H_CUDA(cudaMemcpyAsync(h->scratch, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        dsrc = h->scratch;
    }
    launch_convert<double, float>(dsrc, (float *)dst, n, h->stream);
    H_LAUNCHED();
    return MGENKF_OK;
}

// copy a state buffer out as FP64 into a host or device pointer (syncs for host)
static mgenkf_status store_state(mgenkf_ctx *h, double *dst, const void *src, size_t n) {
    const bool dev = is_device_ptr(dst);
    double *target = dst;
    if (!dev) {
        mgenkf_status st = ensure_scratch(h, n);
        if (st) return st;
        target = h->scratch;
    }
    if (h->mixed)
        launch_convert<float, double>((const float *)src, target, n, h->stream);
    else
        launch_convert<double, double>((const double *)src, target, n, h->stream);
    H_LAUNCHED();
    if (!dev) {
        H_CUDA(cudaMemcpyAsync(dst, target, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        H_CUDA(cudaStreamSynchronize(h->stream));
    }
    return MGENKF_OK;
}

static mgenkf_status copy_out_f64(mgenkf_ctx *h, double *dst, const double *src, size_t n) {
    H_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, h->stream));
    if (!is_device_ptr(dst)) H_CUDA(cudaStreamSynchronize(h->stream));
    return MGENKF_OK;
}

// ---------------------------------------------------------------------------
// create / destroy
// ---------------------------------------------------------------------------
static mgenkf_status validate(mgenkf_ctx *h, const mgenkf_config *c, const int32_t *obs_index,
                              const int32_t *obs_var) {
    if (c->model != MGENKF_BURGERS1D && c->model != MGENKF_NS2D) H_FAIL(MGENKF_ERR_INVALID_ARG, "model must be MGENKF_BURGERS1D or MGENKF_NS2D");
    if (c->ratio < 1 || c->ratio > kMaxRatio) H_FAIL(MGENKF_ERR_INVALID_ARG, "ratio must be in [1, 16]");
    if (c->n_fine < 4 || c->n_fine % c->ratio != 0) H_FAIL(MGENKF_ERR_INVALID_ARG, "n_fine must be >= 4 and a multiple of ratio");
    if (c->n_fine / c->ratio < 4) H_FAIL(MGENKF_ERR_INVALID_ARG, "coarse grid needs >= 4 points per side (4-point stencils)");
    if (c->n_members < 2) H_FAIL(MGENKF_ERR_INVALID_ARG, "n_members must be >= 2");
    if (c->n_obs < 1) H_FAIL(MGENKF_ERR_INVALID_ARG, "n_obs must be >= 1");
    if (c->precision != MGENKF_FP64 && c->precision != MGENKF_MIXED) H_FAIL(MGENKF_ERR_INVALID_ARG, "precision must be MGENKF_FP64 or MGENKF_MIXED");
    if (c->gain_form != MGENKF_GAIN_ENSEMBLE && c->gain_form != MGENKF_GAIN_DIRECT) H_FAIL(MGENKF_ERR_INVALID_ARG, "gain_form must be ENSEMBLE or DIRECT");
    if (c->prolong != MGENKF_PROLONG_LAGRANGE4) H_FAIL(MGENKF_ERR_UNSUPPORTED, "only MGENKF_PROLONG_LAGRANGE4 is built");
    if (!(c->dt > 0.0) || !(c->length > 0.0) || !(c->nu >= 0.0)) H_FAIL(MGENKF_ERR_INVALID_ARG, "dt and length must be > 0, nu >= 0");
    if (!(c->obs_sigma >= 0.0) || !std::isfinite(c->obs_sigma)) H_FAIL(MGENKF_ERR_INVALID_ARG, "obs_sigma must be finite and >= 0");
    if (c->gain_form == MGENKF_GAIN_ENSEMBLE && !(c->obs_sigma > 0.0)) H_FAIL(MGENKF_ERR_INVALID_ARG, "the ensemble-space gain needs obs_sigma > 0 (R^-1)");
    if (!obs_index || !obs_var) H_FAIL(MGENKF_ERR_INVALID_ARG, "obs_index and obs_var are required");
    if (c->n_members > 512) H_FAIL(MGENKF_ERR_INVALID_ARG, "n_members must be <= 512");
    if (c->gain_form == MGENKF_GAIN_DIRECT && c->n_obs > 2048) H_FAIL(MGENKF_ERR_INVALID_ARG, "direct gain form supports n_obs <= 2048");
    const int dim = c->model == MGENKF_BURGERS1D ? 1 : 2;
    const int V = c->model == MGENKF_BURGERS1D ? 1 : 4;
    const long long nfp = dim == 1 ? (long long)c->n_fine : (long long)c->n_fine * c->n_fine;
    for (int j = 0; j < c->n_obs; ++j) {
        if (obs_index[j] < 0 || obs_index[j] >= nfp) H_FAIL(MGENKF_ERR_INVALID_ARG, "obs_index[" + std::to_string(j) + "] out of the fine grid");
        if (obs_var[j] < 0 || obs_var[j] >= V) H_FAIL(MGENKF_ERR_INVALID_ARG, "obs_var[" + std::to_string(j) + "] out of range");
    }
    if (c->model == MGENKF_BURGERS1D) {
        if (c->n_fine / c->ratio > kBurgersMaxPtsPerCta) H_FAIL(MGENKF_ERR_INVALID_ARG, "Burgers coarse grid must have <= 4096 points (one CTA per member)");
        if (burgers_split_factor(c->n_fine) == 0) H_FAIL(MGENKF_ERR_INVALID_ARG, "Burgers fine grid must split into <= 8 CTAs of <= 4096 points");
    } else {
        const char *why = ns2d_check_size(c->n_fine / c->ratio, c->n_fine);
        if (why) H_FAIL(MGENKF_ERR_INVALID_ARG, why);
    }
    return MGENKF_OK;
}

static mgenkf_status upload_fc_table(mgenkf_ctx *h);

static mgenkf_status create_impl(mgenkf_ctx *h, const mgenkf_config *cfg, const int32_t *obs_index,
                                 const int32_t *obs_var) {
    mgenkf_status st = validate(h, cfg, obs_index, obs_var);
    if (st) return st;
    h->cfg = *cfg;
    h->dim = cfg->model == MGENKF_BURGERS1D ? 1 : 2;
    h->V = cfg->model == MGENKF_BURGERS1D ? 1 : 4;
    h->nf = cfg->n_fine;
    h->r = cfg->ratio;
    h->nc = h->nf / h->r;
    h->ne = cfg->n_members;
    h->ny = cfg->n_obs;
    h->taps = h->dim == 1 ? 4 : 16;
    h->cpl = h->dim == 1 ? (size_t)h->nc : (size_t)h->nc * h->nc;
    h->nx = (size_t)h->V * h->cpl;
    h->nxf = (size_t)h->V * (h->dim == 1 ? (size_t)h->nf : (size_t)h->nf * h->nf);
    h->mixed = cfg->precision == MGENKF_MIXED;
    h->direct = cfg->gain_form == MGENKF_GAIN_DIRECT;
    h->cycle = 0;
    H_CUDA(cudaGetDevice(&h->device));

    const size_t ts = tsize(h), ne = h->ne, ny = h->ny, nx = h->nx;
    H_ALLOC(h->fine, h->nxf * ts);
    H_ALLOC(h->fine_prev, h->nxf * ts);
    H_ALLOC(h->fine_tmp, h->nxf * ts);
    H_ALLOC(h->members, ne * nx * ts);
    H_ALLOC(h->xstar, nx * ts);
    H_ALLOC(h->dC, nx * ts);
    H_ALLOC(h->tap_idx, ny * h->taps * sizeof(int32_t));
    H_ALLOC(h->tap_w, ny * h->taps * sizeof(double));
    H_ALLOC(h->yf, (ne + 1) * ny * sizeof(double));
    H_ALLOC(h->yo, ny * sizeof(double));
    H_ALLOC(h->ybar, ny * sizeof(double));
    H_ALLOC(h->eps, ne * ny * sizeof(double));
    H_ALLOC(h->Y, ne * ny * sizeof(double));
    H_ALLOC(h->Z, (ne + 1) * ny * sizeof(double));
    h->ldx = (int)((ne + 15) / 16 * 16);
    h->ntpad = (int)((ne + 1 + 15) / 16 * 16);
    if (h->mixed && !h->direct) {
        H_ALLOC(h->df.Yh, ne * ny * sizeof(float));
        H_ALLOC(h->df.Yl, ne * ny * sizeof(float));
        H_ALLOC(h->df.Zh, (ne + 1) * ny * sizeof(float));
        H_ALLOC(h->df.Zl, (ne + 1) * ny * sizeof(float));
    }
    if (h->mixed) {
        H_ALLOC(h->X16, nx * h->ldx * sizeof(__nv_bfloat16));
        H_ALLOC(h->Tt, (size_t)h->ntpad * h->ldx * sizeof(__nv_bfloat16));
        H_CUDA(cudaMemsetAsync(h->X16, 0, nx * h->ldx * sizeof(__nv_bfloat16), h->stream));
        H_CUDA(cudaMemsetAsync(h->Tt, 0, (size_t)h->ntpad * h->ldx * sizeof(__nv_bfloat16), h->stream));
    } else {
        H_ALLOC(h->X64, ne * nx * sizeof(double));
    }
    if (h->direct) {
        H_ALLOC(h->C, ny * ny * sizeof(double));
        H_ALLOC(h->Ct, ny * ny * sizeof(double));
        H_ALLOC(h->W, (ne + 1) * ny * sizeof(double));
        H_ALLOC(h->Tm, (ne + 1) * ne * sizeof(double));
    } else {
        H_ALLOC(h->S, ne * ne * sizeof(double));
        H_ALLOC(h->Lt, ne * ne * sizeof(double));
        H_ALLOC(h->Bt, (ne + 1) * ne * sizeof(double));
        h->Tm = h->Bt;
    }
    if (cfg->model == MGENKF_NS2D)
        H_ALLOC(h->ns_scratch, ns2d_scratch_elems(h->nc, h->ne, h->nf, 1) * ts);
    {
        const size_t p1 = (size_t)gemm_nt_splits((int)ne, (int)ne, (int)ne + 1, (int)ny) * ne * (2 * ne + 1);
        const size_t p2 = (size_t)gemm_nt_splits((int)ne, 0, (int)ne + 1, (int)ny) * ne * (ne + 1);
        H_ALLOC(h->gemm_part, std::max(p1, p2) * sizeof(double));
    }
    H_ALLOC(h->rmse_part, (size_t)kRmseBlocks * h->V * 2 * sizeof(double));
    H_ALLOC(h->rmse_d, 4 * sizeof(double));
    H_ALLOC(h->status, sizeof(int));
    H_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    H_ALLOC(h->cycle_d, sizeof(uint64_t));
    H_CUDA(cudaMemsetAsync(h->cycle_d, 0, sizeof(uint64_t), h->stream));
    H_CUDA(cudaMemsetAsync(h->fine, 0, h->nxf * ts, h->stream));
    H_CUDA(cudaMemsetAsync(h->members, 0, ne * nx * ts, h->stream));
    H_CUDA(cudaMemsetAsync(h->dC, 0, nx * ts, h->stream));

    // observation operator H^C = H^F Pi_F: Lagrange taps at each observed fine node
    std::vector<int32_t> tidx(ny * h->taps);
    std::vector<double> tw(ny * h->taps);
    for (size_t j = 0; j < ny; ++j) {
        const int f = obs_index[j];
        const size_t plane = (size_t)obs_var[j] * h->cpl;
        if (h->dim == 1) {
            const int J = f / h->r;
            double w[4];
            cubic_weights((double)(f % h->r) / h->r, w);
            for (int t = 0; t < 4; ++t) {
                tidx[j * 4 + t] = (int32_t)(plane + (J - 1 + t + h->nc) % h->nc);
                tw[j * 4 + t] = w[t];
            }
        } else {
            const int fy = f / h->nf, fx = f % h->nf;
            const int Jy = fy / h->r, Jx = fx / h->r;
            double wy[4], wx[4];
            cubic_weights((double)(fy % h->r) / h->r, wy);
            cubic_weights((double)(fx % h->r) / h->r, wx);
            for (int ty = 0; ty < 4; ++ty)
                for (int tx = 0; tx < 4; ++tx) {
                    const size_t yy = (size_t)((Jy - 1 + ty + h->nc) % h->nc);
                    const size_t xx = (size_t)((Jx - 1 + tx + h->nc) % h->nc);
                    tidx[j * 16 + ty * 4 + tx] = (int32_t)(plane + yy * h->nc + xx);
                    tw[j * 16 + ty * 4 + tx] = wy[ty] * wx[tx];
                }
        }
    }
    H_CUDA(cudaMemcpyAsync(h->tap_idx, tidx.data(), tidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    H_CUDA(cudaMemcpyAsync(h->tap_w, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (h->mixed) {
        // w = hi + lo: hi the weight rounded to FP32, lo the remainder (exact in
        // FP64) rounded to FP32
        std::vector<float> whi(tw.size()), wlo(tw.size());
        for (size_t q = 0; q < tw.size(); ++q) {
            whi[q] = (float)tw[q];
            wlo[q] = (float)(tw[q] - (double)whi[q]);
        }
        H_ALLOC(h->tap_wh, tw.size() * sizeof(float));
        H_ALLOC(h->tap_wl, tw.size() * sizeof(float));
        H_CUDA(cudaMemcpyAsync(h->tap_wh, whi.data(), whi.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        H_CUDA(cudaMemcpyAsync(h->tap_wl, wlo.data(), wlo.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        H_CUDA(cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
    }
    for (int m = 0; m < h->r; ++m) cubic_weights((double)m / h->r, h->pw.w[m]);
    // mixed precision: the member update runs on the tensor cores when the
    // shapes allow (N = Ne + 1 <= 256); MGENKF_UPDATE=simt selects the
    // CUDA-core kernel instead (used to cross-check the two)
    h->tc.ready = false;
    if (h->mixed) {
        const char *sel = getenv("MGENKF_UPDATE");
        if (!(sel && strcmp(sel, "simt") == 0))
            update_tc_prepare(&h->tc, h->ldx, (int)h->nx, h->Tt, h->ntpad, h->ne, (const float *)h->members);
    }
    if (h->mixed && cfg->model == MGENKF_NS2D) {
        H_ALLOC(h->d_fc, 2 * sizeof(NsGroup<float>));
        H_CUDA(cudaStreamCreateWithFlags(&h->fstream, cudaStreamNonBlocking));
        H_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        H_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        int sms = 0;
        H_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
        h->fc_choice[0] = ns2d_default_choice(h->nc, h->ne, sms);
        h->fc_choice[1] = ns2d_default_choice(h->nf, 1, sms);
        mgenkf_status st = upload_fc_table(h);
        if (st) return st;
    }
    H_CUDA(cudaStreamSynchronize(h->stream));
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_create(const mgenkf_config *cfg, const int32_t *obs_index,
                                       const int32_t *obs_var, void *cuda_stream, mgenkf_handle *out) {
    if (!out) return MGENKF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg) return MGENKF_ERR_INVALID_ARG;
    mgenkf_ctx *h = new mgenkf_ctx();
    h->stream = (cudaStream_t)cuda_stream;
    mgenkf_status st = create_impl(h, cfg, obs_index, obs_var);
    if (st != MGENKF_OK) {
        mgk_set_error(h->err);
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_destroy(mgenkf_handle h) {
    if (!h) return MGENKF_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return MGENKF_OK;
}

extern "C" const char *mgenkf_last_error(mgenkf_handle h) {
    if (!h) return g_ops_error.c_str();
    return h->err.c_str();
}

// ---------------------------------------------------------------------------
// state
// ---------------------------------------------------------------------------
extern "C" mgenkf_status mgenkf_set_state(mgenkf_handle h, const double *fine, const double *members) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    if (h->mixed) {  // one scratch size for both conversions (no reallocation between them)
        mgenkf_status st = ensure_scratch(h, std::max(h->nxf, (size_t)h->ne * h->nx));
        if (st) return st;
    }
    if (fine) {
        mgenkf_status st = load_state(h, h->fine, fine, h->nxf);
        if (st) return st;
    }
    if (members) {
        mgenkf_status st = load_state(h, h->members, members, (size_t)h->ne * h->nx);
        if (st) return st;
    }
    h->cycle = 0;
    h->have_prev = false;
    H_CUDA(cudaMemsetAsync(h->cycle_d, 0, sizeof(uint64_t), h->stream));
    H_CUDA(cudaStreamSynchronize(h->stream));
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_get_state(mgenkf_handle h, double *fine, double *members) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    {
        mgenkf_status st = ensure_scratch(h, std::max(h->nxf, (size_t)h->ne * h->nx));
        if (st) return st;
    }
    if (fine) {
        mgenkf_status st = store_state(h, fine, h->fine, h->nxf);
        if (st) return st;
    }
    if (members) {
        mgenkf_status st = store_state(h, members, h->members, (size_t)h->ne * h->nx);
        if (st) return st;
    }
    return MGENKF_OK;
}

// the two groups (members, fine run) of one handle, scratch laid out as in
// ns2d_forecast_scratch
static void handle_groups(const mgenkf_ctx *h, NsGroup<float> g[2]) {
    const size_t sz0 = (size_t)4 * h->nc * h->nc * h->ne, sz1 = (size_t)4 * h->nf * h->nf;
    float *sc = (float *)h->ns_scratch;
    const int ns[2] = {h->nc, h->nf}, np[2] = {h->ne, 1};
    float *u0[2] = {(float *)h->members, (float *)h->fine};
    float *s1[2] = {sc, sc + 2 * sz0}, *s2[2] = {sc + sz0, sc + 2 * sz0 + sz1};
    for (int k = 0; k < 2; ++k) {
        g[k] = {};
        g[k].u0 = u0[k];
        g[k].s1 = s1[k];
        g[k].s2 = s2[k];
        g[k].n = ns[k];
        g[k].nprob = np[k];
        const double hh = h->cfg.length / ns[k];
        g[k].inv_h = (float)(1.0 / hh);
        g[k].inv_2h = (float)(1.0 / (2.0 * hh));
        g[k].dt = (float)h->cfg.dt;
    }
}

// the handle's forecast table for its current choices (synchronous)
static mgenkf_status upload_fc_table(mgenkf_ctx *h) {
    NsGroup<float> g[2];
    handle_groups(h, g);
    for (int k = 0; k < 2; ++k) {
        h->fc_units[k] = 0;
        if (h->fc_choice[k] < 0) continue;
        int bands = 0, segs = 0, threads = 0;
        ns2d_march_layout(g[k].n, h->fc_choice[k], &bands, &segs, &threads);
        g[k].tx = bands;
        g[k].ty = segs;
        g[k].tile_begin = 0;
        h->fc_units[k] = bands * segs * g[k].nprob;
    }
    H_CUDA(cudaMemcpyAsync(h->d_fc, g, sizeof(g), cudaMemcpyHostToDevice, h->stream));
    H_CUDA(cudaStreamSynchronize(h->stream));
    return MGENKF_OK;
}

// ---------------------------------------------------------------------------
// the cycle
// ---------------------------------------------------------------------------
static mgenkf_status advance_impl(mgenkf_ctx *h, int nsteps);

static mgenkf_status forecast_impl(mgenkf_ctx *h, int nsteps) {
    if (nsteps < 0) H_FAIL(MGENKF_ERR_INVALID_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return MGENKF_OK;
    if (!h->record_prev) return advance_impl(h, nsteps);
    // regularisation enabled: keep the fine state one step before the end
    mgenkf_status st = advance_impl(h, nsteps - 1);
    if (st) return st;
    H_CUDA(cudaMemcpyAsync(h->fine_prev, h->fine, h->nxf * tsize(h), cudaMemcpyDeviceToDevice, h->stream));
    st = advance_impl(h, 1);
    if (st == MGENKF_OK) h->have_prev = true;
    return st;
}

// nsteps FP32 NS-2D steps with the column march: the members on the handle's
// stream, the fine run beside them on its own stream (forked and joined by
// events, so the call is ordered on the handle's stream as a whole)
static cudaError_t march_forecast(mgenkf_ctx *h, int nsteps) {
    const mgenkf_config &c = h->cfg;
    cudaError_t e = cudaEventRecord(h->ev_fork, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->fstream, h->ev_fork, 0);
    if (e == cudaSuccess)
        e = ns2d_forecast_table(h->d_fc + 1, 1, h->fc_units[1], h->nf, nsteps, c.gamma, c.nu, c.prandtl,
                                h->fc_choice[1], h->fstream);
    if (e == cudaSuccess)
        e = ns2d_forecast_table(h->d_fc, 1, h->fc_units[0], h->nc, nsteps, c.gamma, c.nu, c.prandtl,
                                h->fc_choice[0], h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->fstream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    return e;
}

static mgenkf_status advance_impl(mgenkf_ctx *h, int nsteps) {
    if (nsteps == 0) return MGENKF_OK;
    const mgenkf_config &c = h->cfg;
    cudaError_t e;
    if (c.model == MGENKF_BURGERS1D) {
        if (h->mixed)
            e = burgers_forecast<float>((float *)h->members, h->nc, h->ne, (float *)h->fine, h->nf, 1,
                                        c.length, c.dt, c.nu, nsteps, h->stream);
        else
            e = burgers_forecast<double>((double *)h->members, h->nc, h->ne, (double *)h->fine, h->nf, 1,
                                         c.length, c.dt, c.nu, nsteps, h->stream);
    } else {
        // with the filter the model step is an RK3 step followed by the filter
        // of every grid (the stage buffers are free in between)
        const int chunk = h->filter_sigma > 0.0 ? 1 : nsteps;
        e = cudaSuccess;
        for (int done = 0; done < nsteps && e == cudaSuccess; done += chunk) {
            if (h->mixed) {
                if (h->fc_choice[0] >= 0)
                    e = march_forecast(h, chunk);
                else
                    e = ns2d_forecast_scratch<float>((float *)h->members, h->nc, h->ne, (float *)h->fine, h->nf,
                                                     1, c.length, c.dt, c.nu, c.gamma, c.prandtl, chunk,
                                                     (float *)h->ns_scratch, h->stream);
                if (e == cudaSuccess && h->filter_sigma > 0.0)
                    e = launch_ns2d_filter6<float>((float *)h->members, (float *)h->ns_scratch, h->nc, h->ne,
                                                   h->filter_sigma, h->stream);
                if (e == cudaSuccess && h->filter_sigma > 0.0)
                    e = launch_ns2d_filter6<float>((float *)h->fine, (float *)h->ns_scratch, h->nf, 1,
                                                   h->filter_sigma, h->stream);
            } else {
                e = ns2d_forecast_scratch<double>((double *)h->members, h->nc, h->ne, (double *)h->fine, h->nf, 1,
                                                  c.length, c.dt, c.nu, c.gamma, c.prandtl, chunk,
                                                  (double *)h->ns_scratch, h->stream);
                if (e == cudaSuccess && h->filter_sigma > 0.0)
                    e = launch_ns2d_filter6<double>((double *)h->members, (double *)h->ns_scratch, h->nc, h->ne,
                                                    h->filter_sigma, h->stream);
                if (e == cudaSuccess && h->filter_sigma > 0.0)
                    e = launch_ns2d_filter6<double>((double *)h->fine, (double *)h->ns_scratch, h->nf, 1,
                                                    h->filter_sigma, h->stream);
            }
        }
    }
    if (e != cudaSuccess) H_FAIL(MGENKF_ERR_CUDA, std::string("forecast launch: ") + cudaGetErrorString(e));
    H_LAUNCHED();
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_forecast(mgenkf_handle h, int32_t nsteps) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    return forecast_impl(h, nsteps);
}

static bool has_fc_choice(const mgenkf_ctx *h) { return h->mixed && h->cfg.model == MGENKF_NS2D; }

extern "C" mgenkf_status mgenkf_get_forecast_choice(mgenkf_handle h, int32_t *members, int32_t *fine) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    if (members) *members = h->fc_choice[0];
    if (fine) *fine = h->fc_choice[1];
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_set_forecast_choice(mgenkf_handle h, int32_t members, int32_t fine) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    if (!has_fc_choice(h)) H_FAIL(MGENKF_ERR_INVALID_ARG, "forecast choices exist for mixed-precision NS-2D handles");
    const bool tile = members == -1 && fine == -1;
    const bool march = members >= 0 && members < kNsTileShapes && fine >= 0 && fine < kNsTileShapes;
    if (!tile && !march) H_FAIL(MGENKF_ERR_INVALID_ARG, "forecast choice out of range (each in [0, 16), or both -1)");
    H_CUDA(cudaStreamSynchronize(h->stream));  // launches in flight read the old table
    h->fc_choice[0] = members;
    h->fc_choice[1] = fine;
    return upload_fc_table(h);
}

// `reps` timings (after one warm-up) of kHandleProbeSteps model steps (one
// observation interval of the workloads), written to the stage buffers, of the
// handle's grids with the current choices: the members (which & 1) on the
// handle's stream, the fine run (which & 2) on its own; the fastest
// repetition's milliseconds in *ms (a few tens of microseconds per step, so
// the minimum, not the sum, keeps a stray slow repetition from deciding)
static constexpr int kHandleProbeSteps = 10;
static mgenkf_status probe_handle(mgenkf_ctx *h, int which, int reps, cudaEvent_t t0, cudaEvent_t t1, float *ms) {
    const mgenkf_config &c = h->cfg;
    mgenkf_status st = upload_fc_table(h);
    if (st) return st;
    *ms = 0.f;
    for (int r = 0; r <= reps; ++r) {
        H_CUDA(cudaEventRecord(t0, h->stream));
        H_CUDA(cudaEventRecord(h->ev_fork, h->stream));
        H_CUDA(cudaStreamWaitEvent(h->fstream, h->ev_fork, 0));
        for (int i = 0; i < kHandleProbeSteps; ++i) {
            if (which & 2)
                H_CUDA(ns2d_probe_step(h->d_fc + 1, 1, h->fc_units[1], h->nf, c.gamma, c.nu, c.prandtl,
                                       h->fc_choice[1], h->fstream));
            if (which & 1)
                H_CUDA(ns2d_probe_step(h->d_fc, 1, h->fc_units[0], h->nc, c.gamma, c.nu, c.prandtl,
                                       h->fc_choice[0], h->stream));
        }
        H_CUDA(cudaEventRecord(h->ev_join, h->fstream));
        H_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
        H_CUDA(cudaEventRecord(t1, h->stream));
        H_CUDA(cudaEventSynchronize(t1));
        float t = 0.f;
        H_CUDA(cudaEventElapsedTime(&t, t0, t1));
        if (r) *ms = r == 1 ? t : std::min(*ms, t);
    }
    return MGENKF_OK;
}

static mgenkf_status forecast_autotune_impl(mgenkf_ctx *h, int reps, cudaEvent_t t0, cudaEvent_t t1) {
    const int start[2] = {h->fc_choice[0] >= 0 ? h->fc_choice[0] : 0, h->fc_choice[1] >= 0 ? h->fc_choice[1] : 0};
    float alone[2] = {0.f, 0.f};
    int best[2] = {start[0], start[1]};
    // each grid alone
    for (int k = 0; k < 2; ++k) {
        float tbest = 1e30f;
        for (int sh = 0; sh < kNsTileShapes; ++sh) {
            h->fc_choice[0] = k == 0 ? sh : start[0];
            h->fc_choice[1] = k == 1 ? sh : start[1];
            float ms = 0.f;
            mgenkf_status st = probe_handle(h, 1 << k, reps, t0, t1, &ms);
            if (st) return st;
            if (ms < tbest) {
                tbest = ms;
                best[k] = sh;
            }
        }
        alone[k] = tbest;
    }
    // both at once, the slower grid first
    const int order[2] = {alone[0] >= alone[1] ? 0 : 1, alone[0] >= alone[1] ? 1 : 0};
    for (int k : order) {
        float tbest = 1e30f;
        int pick = best[k];
        for (int sh = 0; sh < kNsTileShapes; ++sh) {
            h->fc_choice[k] = sh;
            h->fc_choice[1 - k] = best[1 - k];
            float ms = 0.f;
            mgenkf_status st = probe_handle(h, 3, reps, t0, t1, &ms);
            if (st) return st;
            if (ms < tbest) {
                tbest = ms;
                pick = sh;
            }
        }
        best[k] = pick;
    }
    h->fc_choice[0] = best[0];
    h->fc_choice[1] = best[1];
    return upload_fc_table(h);
}

extern "C" mgenkf_status mgenkf_forecast_autotune(mgenkf_handle h, int32_t reps) {
    if (!h || reps < 1) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    if (!has_fc_choice(h)) return MGENKF_OK;
    H_CUDA(cudaStreamSynchronize(h->stream));
    const int keep[2] = {h->fc_choice[0], h->fc_choice[1]};
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    H_CUDA(cudaEventCreate(&t0));
    mgenkf_status st = MGENKF_OK;
    if (cudaEventCreate(&t1) != cudaSuccess) {
        h->err = "cudaEventCreate failed";
        st = MGENKF_ERR_CUDA;
    }
    if (st == MGENKF_OK) st = forecast_autotune_impl(h, reps, t0, t1);
    if (st != MGENKF_OK) {  // keep the choices the handle had
        cudaStreamSynchronize(h->stream);
        cudaStreamSynchronize(h->fstream);
        h->fc_choice[0] = keep[0];
        h->fc_choice[1] = keep[1];
        const std::string why = h->err;
        upload_fc_table(h);
        h->err = why;
    }
    cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return st;
}

template <typename T>
static void analyse_kernels(mgenkf_ctx *h, int gen_eps) {
    const cudaStream_t s = h->stream;
    const int ne = h->ne, ny = h->ny;
    const size_t nx = h->nx;
    T *members = (T *)h->members, *xstar = (T *)h->xstar, *dC = (T *)h->dC;
    launch_restrict<T>((const T *)h->fine, xstar, h->dim, h->V, h->nc, h->r, s);
    if (h->recentre) launch_recentre<T>(members, nx, ne, xstar, h->status, s);
    launch_obs_apply<T>(members, xstar, nx, ne, ny, h->taps, h->tap_idx, h->tap_w, h->yf, s, h->tap_wh, h->tap_wl);
    launch_obs_mean(h->yf, h->yo, ne, ny, h->ybar, h->Z, h->status, s, h->df.Zh, h->df.Zl);
    launch_obs_perturb(h->yf, h->ybar, h->yo, h->eps, gen_eps, h->cfg.seed, h->cycle_d,
                       h->cfg.obs_sigma, ne, ny, h->Y, h->Z, s, h->df);
    // the tensor-core update forms the BF16 anomalies itself from the members it reads
    if (!(h->mixed && h->tc.ready)) launch_ens_anom<T>(members, nx, ne, h->X64, h->X16, h->status, s);
    const double s2 = h->cfg.obs_sigma * h->cfg.obs_sigma;
    if (!h->direct) {
        // S = I + Y^T R^-1 Y (ne x ne) and B = Y^T R^-1 [D | d*]; T = S^-1 B
        // (mixed precision: the products in double-FP32 arithmetic)
        if (h->df.Yh)
            launch_gemm_df(h->df, ne, ny, s2, h->S, h->Bt, h->status, s, h->gemm_part);
        else
            launch_gemm_nt_f64(h->Y, ne, h->Y, ne, h->Z, ne + 1, ny, s2, 1.0, h->S, h->Bt, h->status, s,
                               h->gemm_part);
        launch_cholesky(h->S, h->Lt, ne, h->status, s);
        launch_chol_solve(h->S, h->Lt, ne, h->Bt, h->Bt, ne + 1, h->mixed ? h->Tt : nullptr, h->ldx,
                          h->status, s);
    } else {
        // C = Y Y^T + R (ny x ny), W = C^-1 [D | d*], T = Y^T W
        launch_gemm_tn_f64(h->Y, ne, ny, s2, h->C, h->status, s);
        launch_cholesky(h->C, h->Ct, ny, h->status, s);
        launch_chol_solve(h->C, h->Ct, ny, h->Z, h->W, ne + 1, nullptr, 0, h->status, s);
        launch_gemm_nt_f64(h->Y, ne, nullptr, 0, h->W, ne + 1, ny, 1.0, 0.0, nullptr, h->Tm, h->status, s,
                           h->gemm_part);
        if (h->mixed) launch_tt_bf16(h->Tm, h->Tt, ne, h->ldx, h->status, s);
    }
    if (h->mixed && h->tc.ready)
        launch_update_tc(h->tc, (float *)members, (float *)dC, h->status, s);
    else if (h->mixed)
        launch_update_bf16((float *)members, (float *)dC, h->X16, h->Tt, h->ldx, nx, ne, h->status, s);
    else
        launch_update_f64<T>(members, dC, h->X64, h->Tm, nx, ne, h->status, s);
    launch_bump_counter(h->cycle_d, s);
}

static mgenkf_status analyse_impl(mgenkf_ctx *h, const double *y_obs, const double *eps) {
    if (!y_obs) H_FAIL(MGENKF_ERR_INVALID_ARG, "y_obs is required");
    const bool ydev = is_device_ptr(y_obs);
    if (!ydev) {
        for (int j = 0; j < h->ny; ++j)
            if (!std::isfinite(y_obs[j])) H_FAIL(MGENKF_ERR_NONFINITE, "y_obs[" + std::to_string(j) + "] is not finite");
    }
    H_CUDA(cudaMemsetAsync(h->dC, 0, h->nx * tsize(h), h->stream));
    H_CUDA(cudaMemcpyAsync(h->yo, y_obs, h->ny * sizeof(double), cudaMemcpyDefault, h->stream));
    if (eps) H_CUDA(cudaMemcpyAsync(h->eps, eps, (size_t)h->ne * h->ny * sizeof(double), cudaMemcpyDefault, h->stream));
    if (h->mixed)
        analyse_kernels<float>(h, eps ? 0 : 2);  // FP32 Box-Muller on the mixed path
    else
        analyse_kernels<double>(h, eps ? 0 : 1);
    H_LAUNCHED();
    h->cycle += 1;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_analyse(mgenkf_handle h, const double *y_obs, const double *eps) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    return analyse_impl(h, y_obs, eps);
}

static mgenkf_status prolong_impl(mgenkf_ctx *h) {
    if (h->mixed)
        launch_prolong_add<float>((float *)h->fine, (const float *)h->dC, h->dim, h->V, h->nc, h->r, h->pw, h->status, h->stream);
    else
        launch_prolong_add<double>((double *)h->fine, (const double *)h->dC, h->dim, h->V, h->nc, h->r, h->pw, h->status, h->stream);
    H_LAUNCHED();
    if (h->cnn) {
        mgenkf_status st = cnn_forward_status(h->cnn, (const float *)h->dC, (const float *)h->xstar, 1,
                                              (float *)h->fine, 1, h->status, h->stream);
        if (st) H_FAIL(st, std::string("learned correction: ") + mgk_last_error());
    }
    if (h->alpha > 0.0 && h->have_prev) {
        // final fine iteration (Algorithm 4 step 6), out of place, then back
        const mgenkf_config &c = h->cfg;
        if (h->mixed)
            launch_fine_residual<float>(c.model, (const float *)h->fine, (const float *)h->fine_prev, h->nf, c.length,
                                        c.nu, c.gamma, c.prandtl, c.dt, h->alpha, (float *)h->fine_tmp, nullptr,
                                        h->status, h->stream);
        else
            launch_fine_residual<double>(c.model, (const double *)h->fine, (const double *)h->fine_prev, h->nf,
                                         c.length, c.nu, c.gamma, c.prandtl, c.dt, h->alpha, (double *)h->fine_tmp,
                                         nullptr, h->status, h->stream);
        H_LAUNCHED();
        H_CUDA(cudaMemcpyAsync(h->fine, h->fine_tmp, h->nxf * tsize(h), cudaMemcpyDeviceToDevice, h->stream));
    }
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_set_recentre(mgenkf_handle h, int32_t on) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    h->recentre = on != 0;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_set_filter(mgenkf_handle h, double sigma) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    if (h->cfg.model != MGENKF_NS2D) H_FAIL(MGENKF_ERR_INVALID_ARG, "the sixth-order filter belongs to the NS-2D model");
    if (!(sigma >= 0.0 && sigma <= 1.0)) H_FAIL(MGENKF_ERR_INVALID_ARG, "filter strength sigma must be in [0, 1]");
    if (sigma > 0.0 && (h->nc < 8 || h->nf < 8)) H_FAIL(MGENKF_ERR_INVALID_ARG, "the 7-point filter needs >= 8 points per side");
    h->filter_sigma = sigma;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_set_regularisation(mgenkf_handle h, double alpha) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    if (!(alpha <= 1.0) || !std::isfinite(alpha)) H_FAIL(MGENKF_ERR_INVALID_ARG, "alpha must be finite and <= 1");
    h->record_prev = alpha >= 0.0;
    h->alpha = alpha > 0.0 ? alpha : 0.0;
    if (!h->record_prev) h->have_prev = false;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_set_prolong_cnn(mgenkf_handle h, void *cnn) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    if (cnn && (h->cfg.model != MGENKF_NS2D || !h->mixed || h->r != 4))
        H_FAIL(MGENKF_ERR_INVALID_ARG, "the learned correction needs an NS-2D, mixed-precision handle with ratio 4");
    if (cnn && mgk_cnn_coarse_size((mgk_cnn_t)cnn) != h->nc)
        H_FAIL(MGENKF_ERR_INVALID_ARG, "the learned correction was built for another coarse size");
    h->cnn = (mgk_cnn_t)cnn;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_prolong_correct(mgenkf_handle h) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    return prolong_impl(h);
}

static mgenkf_status rmse_impl(mgenkf_ctx *h, const double *truth, double *out) {
    if (!truth || !out) H_FAIL(MGENKF_ERR_INVALID_ARG, "truth_fine and out are required");
    const double *t = truth;
    if (!is_device_ptr(truth)) {
        if (!h->truth_d) H_ALLOC(h->truth_d, h->nxf * sizeof(double));
        H_CUDA(cudaMemcpyAsync(h->truth_d, truth, h->nxf * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        t = h->truth_d;
    }
    const size_t npts = h->nxf / h->V;
    if (h->mixed)
        launch_rmse<float>((const float *)h->fine, t, h->V, npts, h->rmse_part, kRmseBlocks, h->rmse_d, h->stream);
    else
        launch_rmse<double>((const double *)h->fine, t, h->V, npts, h->rmse_part, kRmseBlocks, h->rmse_d, h->stream);
    H_LAUNCHED();
    return copy_out_f64(h, out, h->rmse_d, h->V);
}

extern "C" mgenkf_status mgenkf_rmse(mgenkf_handle h, const double *truth_fine, double *out) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    return rmse_impl(h, truth_fine, out);
}

// A host truth is copied on a side stream while the forecast runs (after the
// previous work on the handle's stream, which may still read the buffer), and
// the RMSE waits for that copy.
static mgenkf_status stage_truth(mgenkf_ctx *h, const double *truth) {
    if (!h->truth_d) H_ALLOC(h->truth_d, h->nxf * sizeof(double));
    if (!h->cstream) {
        H_CUDA(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
        H_CUDA(cudaEventCreateWithFlags(&h->ev_prev, cudaEventDisableTiming));
        H_CUDA(cudaEventCreateWithFlags(&h->ev_truth, cudaEventDisableTiming));
    }
    H_CUDA(cudaEventRecord(h->ev_prev, h->stream));
    H_CUDA(cudaStreamWaitEvent(h->cstream, h->ev_prev, 0));
    H_CUDA(cudaMemcpyAsync(h->truth_d, truth, h->nxf * sizeof(double), cudaMemcpyHostToDevice, h->cstream));
    H_CUDA(cudaEventRecord(h->ev_truth, h->cstream));
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_cycle(mgenkf_handle h, int32_t nsteps, const double *y_obs,
                                      const double *truth_fine, double *rmse_out) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    if (truth_fine && !rmse_out) H_FAIL(MGENKF_ERR_INVALID_ARG, "rmse_out is required with truth_fine");
    const bool staged = truth_fine && !is_device_ptr(truth_fine);
    mgenkf_status st = staged ? stage_truth(h, truth_fine) : MGENKF_OK;
    if (st == MGENKF_OK) st = forecast_impl(h, nsteps);
    if (st == MGENKF_OK) st = analyse_impl(h, y_obs, nullptr);
    if (st == MGENKF_OK) st = prolong_impl(h);
    if (st == MGENKF_OK && truth_fine) {
        if (staged) {
            const cudaError_t e = cudaStreamWaitEvent(h->stream, h->ev_truth, 0);
            if (e != cudaSuccess) {
                h->err = std::string("truth copy: ") + cudaGetErrorString(e);
                st = MGENKF_ERR_CUDA;
            } else
                st = rmse_impl(h, h->truth_d, rmse_out);
        } else {
            st = rmse_impl(h, truth_fine, rmse_out);
        }
    }
    // the caller's truth buffer is free again when this returns
    if (staged && h->cstream) cudaStreamSynchronize(h->cstream);
    return st;
}

extern "C" mgenkf_status mgenkf_get_field(mgenkf_handle h, int32_t field, double *out, size_t count) {
    if (!h || !out) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    const size_t ne = h->ne, ny = h->ny;
    switch (field) {
        case MGENKF_FIELD_XSTAR:
            if (count < h->nx) H_FAIL(MGENKF_ERR_INVALID_ARG, "count too small");
            return store_state(h, out, h->xstar, h->nx);
        case MGENKF_FIELD_DC:
            if (count < h->nx) H_FAIL(MGENKF_ERR_INVALID_ARG, "count too small");
            return store_state(h, out, h->dC, h->nx);
        case MGENKF_FIELD_YF:
            if (count < (ne + 1) * ny) H_FAIL(MGENKF_ERR_INVALID_ARG, "count too small");
            return copy_out_f64(h, out, h->yf, (ne + 1) * ny);
        case MGENKF_FIELD_T:
            if (count < (ne + 1) * ne) H_FAIL(MGENKF_ERR_INVALID_ARG, "count too small");
            return copy_out_f64(h, out, h->Tm, (ne + 1) * ne);
        case MGENKF_FIELD_EPS:
            if (count < ne * ny) H_FAIL(MGENKF_ERR_INVALID_ARG, "count too small");
            return copy_out_f64(h, out, h->eps, ne * ny);
        case MGENKF_FIELD_GAMMA: {
            if (count < h->nxf) H_FAIL(MGENKF_ERR_INVALID_ARG, "count too small");
            if (!h->have_prev)
                H_FAIL(MGENKF_ERR_INVALID_ARG, "no recorded previous fine state: enable mgenkf_set_regularisation "
                                               "and run a forecast first");
            mgenkf_status st = ensure_scratch(h, h->nxf);
            if (st) return st;
            const mgenkf_config &c = h->cfg;
            if (h->mixed)
                launch_fine_residual<float>(c.model, (const float *)h->fine, (const float *)h->fine_prev, h->nf,
                                            c.length, c.nu, c.gamma, c.prandtl, c.dt, 0.0, nullptr, h->scratch,
                                            nullptr, h->stream);
            else
                launch_fine_residual<double>(c.model, (const double *)h->fine, (const double *)h->fine_prev, h->nf,
                                             c.length, c.nu, c.gamma, c.prandtl, c.dt, 0.0, nullptr, h->scratch,
                                             nullptr, h->stream);
            H_LAUNCHED();
            return copy_out_f64(h, out, h->scratch, h->nxf);
        }
        case MGENKF_FIELD_GAMMA_NORM: {
            if (count < h->nxf) H_FAIL(MGENKF_ERR_INVALID_ARG, "count too small");
            if (!h->have_prev)
                H_FAIL(MGENKF_ERR_INVALID_ARG, "no recorded previous fine state: enable mgenkf_set_regularisation "
                                               "and run a forecast first");
            mgenkf_status st = ensure_scratch(h, h->nxf);
            if (st) return st;
            const mgenkf_config &c = h->cfg;
            const size_t plane = h->nxf / h->V;
            if (h->mixed) {
                launch_fine_residual<float>(c.model, (const float *)h->fine, (const float *)h->fine_prev, h->nf,
                                            c.length, c.nu, c.gamma, c.prandtl, c.dt, 0.0, nullptr, h->scratch,
                                            nullptr, h->stream);
                launch_gamma_norm<float>((const float *)h->fine, (const float *)h->fine_prev, h->V, plane, c.dt,
                                         h->scratch, h->stream);
            } else {
                launch_fine_residual<double>(c.model, (const double *)h->fine, (const double *)h->fine_prev, h->nf,
                                             c.length, c.nu, c.gamma, c.prandtl, c.dt, 0.0, nullptr, h->scratch,
                                             nullptr, h->stream);
                launch_gamma_norm<double>((const double *)h->fine, (const double *)h->fine_prev, h->V, plane, c.dt,
                                          h->scratch, h->stream);
            }
            H_LAUNCHED();
            return copy_out_f64(h, out, h->scratch, h->nxf);
        }
        case MGENKF_FIELD_RATE: {
            if (count < h->nxf) H_FAIL(MGENKF_ERR_INVALID_ARG, "count too small");
            if (!h->have_prev)
                H_FAIL(MGENKF_ERR_INVALID_ARG, "no recorded previous fine state: enable mgenkf_set_regularisation "
                                               "and run a forecast first");
            mgenkf_status st = ensure_scratch(h, h->nxf);
            if (st) return st;
            if (h->mixed)
                launch_state_rate<float>((const float *)h->fine, (const float *)h->fine_prev, h->nxf, h->cfg.dt,
                                         h->scratch, h->stream);
            else
                launch_state_rate<double>((const double *)h->fine, (const double *)h->fine_prev, h->nxf, h->cfg.dt,
                                          h->scratch, h->stream);
            H_LAUNCHED();
            return copy_out_f64(h, out, h->scratch, h->nxf);
        }
        default:
            H_FAIL(MGENKF_ERR_INVALID_ARG, "unknown field");
    }
}

extern "C" mgenkf_status mgenkf_set_wait_limit(mgenkf_handle h, int64_t cycles) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    if (cycles < 0) H_FAIL(MGENKF_ERR_INVALID_ARG, "the wait limit is a number of cycles >= 0");
    h->tc.wait_limit = cycles > 0 ? cycles : 0;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_sync(mgenkf_handle h) {
    if (!h) return MGENKF_ERR_INVALID_ARG;
    H_CUDA(cudaStreamSynchronize(h->stream));
    int st = 0;
    H_CUDA(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        H_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
        H_CUDA(cudaStreamSynchronize(h->stream));
        h->err = st == MGENKF_ERR_NOT_SPD   ? "innovation matrix not SPD: members and fine run left unchanged"
                 : st == MGENKF_ERR_TIMEOUT ? "a bounded device wait ran out: members and fine run left unchanged"
                                            : "non-finite observation: members and fine run left unchanged";
        return (mgenkf_status)st;
    }
    return MGENKF_OK;
}

// ---------------------------------------------------------------------------
// checkpoint
// ---------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];
    int32_t model, n_fine, ratio, n_members, n_obs, precision;
    uint64_t cycle;
};

extern "C" mgenkf_status mgenkf_save(mgenkf_handle h, const char *path) {
    if (!h || !path) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    std::vector<double> fine(h->nxf), mem((size_t)h->ne * h->nx);
    mgenkf_status st = mgenkf_get_state(h, fine.data(), mem.data());
    if (st) return st;
    FILE *f = fopen(path, "wb");
    if (!f) H_FAIL(MGENKF_ERR_INVALID_ARG, std::string("cannot open ") + path);
    CkptHeader hd;
    memcpy(hd.magic, "MGENKF01", 8);
    hd.model = h->cfg.model;
    hd.n_fine = h->nf;
    hd.ratio = h->r;
    hd.n_members = h->ne;
    hd.n_obs = h->ny;
    hd.precision = h->cfg.precision;
    H_CUDA(cudaMemcpy(&hd.cycle, h->cycle_d, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(fine.data(), sizeof(double), fine.size(), f) == fine.size() &&
              fwrite(mem.data(), sizeof(double), mem.size(), f) == mem.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) H_FAIL(MGENKF_ERR_INVALID_ARG, std::string("write failed: ") + path);
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_load(mgenkf_handle h, const char *path) {
    if (!h || !path) return MGENKF_ERR_INVALID_ARG;
    h->err.clear();
    FILE *f = fopen(path, "rb");
    if (!f) H_FAIL(MGENKF_ERR_INVALID_ARG, std::string("cannot open ") + path);
    CkptHeader hd;
    std::vector<double> fine(h->nxf), mem((size_t)h->ne * h->nx);
    bool ok = fread(&hd, sizeof(hd), 1, f) == 1;
    ok = ok && memcmp(hd.magic, "MGENKF01", 8) == 0 && hd.model == h->cfg.model && hd.n_fine == h->nf &&
         hd.ratio == h->r && hd.n_members == h->ne && hd.n_obs == h->ny;
    ok = ok && fread(fine.data(), sizeof(double), fine.size(), f) == fine.size() &&
         fread(mem.data(), sizeof(double), mem.size(), f) == mem.size();
    fclose(f);
    if (!ok) H_FAIL(MGENKF_ERR_INVALID_ARG, std::string("checkpoint does not match this handle: ") + path);
    mgenkf_status st = mgenkf_set_state(h, fine.data(), mem.data());
    if (st) return st;
    h->cycle = hd.cycle;
    // stream-ordered: a plain copy from pageable memory may return before it
    // lands, and the handle's stream need not wait for the legacy stream
    H_CUDA(cudaMemcpyAsync(h->cycle_d, &hd.cycle, sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
    H_CUDA(cudaStreamSynchronize(h->stream));
    return MGENKF_OK;
}

// ---------------------------------------------------------------------------
// stateless entry points (include/mgenkf_ops.h)
// ---------------------------------------------------------------------------
extern "C" mgenkf_status mgk_forecast(int32_t model, int32_t precision, void *state, int32_t nprob,
                                      int32_t n, double length, double dt, double nu, double gamma,
                                      double prandtl, int32_t nsteps, void *stream) {
    g_ops_error.clear();
    if (!state || nprob < 0 || nsteps < 0 || !(dt > 0.0) || !(length > 0.0)) {
        g_ops_error = "invalid state pointer, nprob, nsteps, dt or length";
        return MGENKF_ERR_INVALID_ARG;
    }
    if (precision != MGENKF_FP64 && precision != MGENKF_MIXED) {
        g_ops_error = "precision must be MGENKF_FP64 or MGENKF_MIXED";
        return MGENKF_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (model == MGENKF_BURGERS1D) {
        if (n < 4 || n > 8 * kBurgersMaxPtsPerCta || burgers_split_factor(n) == 0) {
            g_ops_error = "Burgers n must be in [4, 32768] and split into <= 8 CTAs of <= 4096 points";
            return MGENKF_ERR_INVALID_ARG;
        }
        const bool whole = n <= kBurgersMaxPtsPerCta;
        if (precision == MGENKF_MIXED)
            e = whole ? burgers_forecast<float>((float *)state, n, nprob, nullptr, 0, 0, length, dt, nu, nsteps, s)
                      : burgers_forecast<float>(nullptr, 0, 0, (float *)state, n, nprob, length, dt, nu, nsteps, s);
        else
            e = whole ? burgers_forecast<double>((double *)state, n, nprob, nullptr, 0, 0, length, dt, nu, nsteps, s)
                      : burgers_forecast<double>(nullptr, 0, 0, (double *)state, n, nprob, length, dt, nu, nsteps, s);
    } else if (model == MGENKF_NS2D) {
        const char *why = ns2d_check_size(n, n);
        if (why) {
            g_ops_error = why;
            return MGENKF_ERR_INVALID_ARG;
        }
        if (precision == MGENKF_MIXED && (reinterpret_cast<uintptr_t>(state) & 15)) {
            g_ops_error = "NS-2D FP32 states must start on a 16-byte boundary";
            return MGENKF_ERR_INVALID_ARG;
        }
        if (precision == MGENKF_MIXED)
            e = ns2d_forecast<float>((float *)state, n, nprob, nullptr, 0, 0, length, dt, nu, gamma, prandtl, nsteps, s);
        else
            e = ns2d_forecast<double>((double *)state, n, nprob, nullptr, 0, 0, length, dt, nu, gamma, prandtl, nsteps, s);
    } else {
        g_ops_error = "model must be MGENKF_BURGERS1D or MGENKF_NS2D";
        return MGENKF_ERR_INVALID_ARG;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_ops_error = std::string("forecast launch: ") + cudaGetErrorString(e);
        return MGENKF_ERR_CUDA;
    }
    return MGENKF_OK;
}

extern "C" mgenkf_status mgk_normals(uint64_t seed, uint64_t tag, uint64_t ctr0, int64_t count,
                                     double *out, void *stream) {
    g_ops_error.clear();
    if (count < 0 || (count > 0 && !out)) {
        g_ops_error = "count must be >= 0 and out non-NULL";
        return MGENKF_ERR_INVALID_ARG;
    }
    launch_normals(seed, tag, ctr0, count, out, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_ops_error = std::string("normals launch: ") + cudaGetErrorString(e);
        return MGENKF_ERR_CUDA;
    }
    return MGENKF_OK;
}

extern "C" const char *mgk_last_error(void) { return g_ops_error.c_str(); }

extern "C" uint64_t mgk_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

// ===========================================================================
// batched cycles of independent NS-2D handles: one CUDA graph launch per cycle
// ===========================================================================
namespace {
// analysis branches of the captured cycle (problems spread by estimated cost)
constexpr int kMaxBatchStreams = 128;
constexpr int kDefaultBatchBranches = 16;  // measured best for the 96-problem batch (1, 4, 16, 128 tried)
}

struct mgenkf_batch {
    std::vector<mgenkf_ctx *> hs;
    cudaStream_t s0 = nullptr;
    bool own_s0 = false;  // created here when the caller passed the legacy stream
    std::vector<cudaStream_t> aux;
    int nbranch = 1;  // analysis branches (streams aux[0 .. nbranch)); the forecast of grid size k runs on aux[nbranch + k]
    std::vector<int> branch;  // branch of each problem
    std::vector<cudaEvent_t> ev;
    double *obs_stage = nullptr;
    double *innov = nullptr;  // per-problem innovation RMS of the last cycle
    std::vector<size_t> obs_off;
    size_t total_ny = 0;
    std::vector<int> sizes;  // distinct grid sizes of the members and fine runs
    std::vector<int> shape;  // segment choice of the forecast per size (ns2d_seg_rows)
    // per size: device table of its groups, their number and the units of a step launch
    std::vector<NsGroup<float> *> d_groups;
    std::vector<int> ngroups, units;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_nsteps = -1;
    double gamma = 1.4, mu = 1e-3, prandtl = 0.72;
    // grouped analysis: one launch per analysis step over all problems of a
    // part (when every problem fits it; otherwise one chain per problem on the
    // branches).  The problems are split into parts balanced by forecast work:
    // part p + 1's forecast of a grid size starts when part p's has finished,
    // and part p's analysis runs beside part p + 1's forecast.
    bool grouped = false;
    int nparts = 0;                     // parts the plans and part tables were built for
    std::vector<int> part;              // part of each problem
    std::vector<GroupPlan> gplans;      // per part
    std::vector<long long> gplan_wait;  // each handle's update wait limit the plans were built with
    bool ptables_stale = true;          // part tables behind the current forecast choices
    std::vector<NsGroup<float> *> pd_groups;  // [part x sizes]: device tables of the part's groups per size
    std::vector<int> pngroups, punits;
    std::vector<cudaStream_t> pstreams;  // [part x (sizes + 1)]: forecast streams per size, then the analysis stream
    std::vector<cudaEvent_t> pev;        // [part x (sizes + 1)] + 1: forecast done per size, analysis done; start
    std::string err;
};

#define B_FAIL(code, msg) \
    do {                  \
        b->err = (msg);   \
        return (code);    \
    } while (0)
#define B_CUDA(call)                                                         \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);     \
            return MGENKF_ERR_CUDA;                                          \
        }                                                                    \
    } while (0)

static int size_index(const mgenkf_batch *b, int n) {
    for (size_t i = 0; i < b->sizes.size(); ++i)
        if (b->sizes[i] == n) return (int)i;
    return -1;
}


// host tables of groups per grid size (only the size `only_size`, with the
// segment choice `only_shape`, if given)
static void build_tables(mgenkf_batch *b, std::vector<std::vector<NsGroup<float>>> &tab, int only_size,
                         int only_shape) {
    tab.assign(b->sizes.size(), {});
    std::vector<int> units(b->sizes.size(), 0);
    for (mgenkf_ctx *h : b->hs) {
        NsGroup<float> g[2];
        handle_groups(h, g);
        for (int k = 0; k < 2; ++k) {
            const int si = size_index(b, g[k].n);
            int sh = b->shape[si];
            if (only_size > 0) {
                if (g[k].n != only_size) continue;
                sh = only_shape;
            }
            int bands = 0, segs = 0, threads = 0;
            ns2d_march_layout(g[k].n, sh, &bands, &segs, &threads);
            g[k].tx = bands;
            g[k].ty = segs;
            g[k].tile_begin = units[si];
            units[si] += bands * segs * g[k].nprob;
            tab[si].push_back(g[k]);
        }
    }
}

static void free_part_tables(mgenkf_batch *b) {
    for (NsGroup<float> *d : b->pd_groups)
        if (d) cudaFree(d);
    b->pd_groups.clear();
    b->pngroups.clear();
    b->punits.clear();
}

static mgenkf_status upload_tables(mgenkf_batch *b, const std::vector<std::vector<NsGroup<float>>> &tab) {
    // nothing may still read the old tables
    B_CUDA(cudaStreamSynchronize(b->s0));
    for (cudaStream_t s : b->aux) B_CUDA(cudaStreamSynchronize(s));
    for (NsGroup<float> *d : b->d_groups)
        if (d) cudaFree(d);
    const size_t ns = b->sizes.size();
    b->d_groups.assign(ns, nullptr);
    b->ngroups.assign(ns, 0);
    b->units.assign(ns, 0);
    for (size_t k = 0; k < ns; ++k) {
        b->ngroups[k] = (int)tab[k].size();
        if (tab[k].empty()) continue;
        const NsGroup<float> &last = tab[k].back();
        b->units[k] = last.tile_begin + last.tx * last.ty * last.nprob;
        B_CUDA(cudaMalloc(&b->d_groups[k], tab[k].size() * sizeof(NsGroup<float>)));
        // on the batch stream: a plain copy from pageable memory may return
        // before it lands and a non-blocking stream does not wait for it
        B_CUDA(cudaMemcpyAsync(b->d_groups[k], tab[k].data(), tab[k].size() * sizeof(NsGroup<float>),
                               cudaMemcpyHostToDevice, b->s0));
    }
    B_CUDA(cudaStreamSynchronize(b->s0));
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_nsteps = -1;
    b->ptables_stale = true;
    return MGENKF_OK;
}

// device tables of the groups of each (part, grid size), for the current
// forecast choices; nothing may read the old ones (the caller synchronised)
static mgenkf_status upload_part_tables(mgenkf_batch *b) {
    const int ns = (int)b->sizes.size(), np = b->nparts;
    std::vector<std::vector<NsGroup<float>>> tab((size_t)np * ns);
    std::vector<int> units((size_t)np * ns, 0);
    for (size_t j = 0; j < b->hs.size(); ++j) {
        NsGroup<float> g[2];
        handle_groups(b->hs[j], g);
        for (int k = 0; k < 2; ++k) {
            const int si = size_index(b, g[k].n), ti = b->part[j] * ns + si;
            int bands = 0, segs = 0, threads = 0;
            ns2d_march_layout(g[k].n, b->shape[si], &bands, &segs, &threads);
            g[k].tx = bands;
            g[k].ty = segs;
            g[k].tile_begin = units[ti];
            units[ti] += bands * segs * g[k].nprob;
            tab[ti].push_back(g[k]);
        }
    }
    free_part_tables(b);
    b->pd_groups.assign(tab.size(), nullptr);
    b->pngroups.assign(tab.size(), 0);
    b->punits = units;
    for (size_t t = 0; t < tab.size(); ++t) {
        b->pngroups[t] = (int)tab[t].size();
        if (tab[t].empty()) continue;
        B_CUDA(cudaMalloc(&b->pd_groups[t], tab[t].size() * sizeof(NsGroup<float>)));
        B_CUDA(cudaMemcpyAsync(b->pd_groups[t], tab[t].data(), tab[t].size() * sizeof(NsGroup<float>),
                               cudaMemcpyHostToDevice, b->s0));
    }
    B_CUDA(cudaStreamSynchronize(b->s0));
    b->ptables_stale = false;
    return MGENKF_OK;
}

static void batch_free(mgenkf_batch *b) {
    for (GroupPlan &gp : b->gplans) group_plan_free(&gp);
    free_part_tables(b);
    for (cudaStream_t s : b->pstreams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->pev) cudaEventDestroy(e);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (NsGroup<float> *d : b->d_groups)
        if (d) cudaFree(d);
    if (b->obs_stage) cudaFree(b->obs_stage);
    if (b->innov) cudaFree(b->innov);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (cudaStream_t s : b->aux) cudaStreamDestroy(s);
    if (b->own_s0) cudaStreamDestroy(b->s0);
}

extern "C" mgenkf_status mgenkf_batch_create(const mgenkf_handle *handles, int32_t n, void *stream,
                                             mgenkf_batch_t *out) {
    if (!out || !handles || n < 1) return MGENKF_ERR_INVALID_ARG;
    *out = nullptr;
    mgenkf_batch *b = new mgenkf_batch();
    b->s0 = (cudaStream_t)stream;
    auto fail = [&](mgenkf_status st, const std::string &m) {
        mgk_set_error("mgenkf_batch_create: " + m);
        batch_free(b);
        delete b;
        return st;
    };
    for (int i = 0; i < n; ++i) {
        mgenkf_ctx *h = handles[i];
        if (!h) return fail(MGENKF_ERR_INVALID_ARG, "NULL handle");
        if (h->cfg.model != MGENKF_NS2D || !h->mixed)
            return fail(MGENKF_ERR_INVALID_ARG, "batches hold NS-2D mixed-precision handles");
        if (h->record_prev)
            return fail(MGENKF_ERR_INVALID_ARG, "the final fine iteration is not available in batches");
        if (h->filter_sigma > 0.0)
            return fail(MGENKF_ERR_INVALID_ARG, "the sixth-order filter is not available in batches");
        if (i == 0) {
            b->gamma = h->cfg.gamma;
            b->mu = h->cfg.nu;
            b->prandtl = h->cfg.prandtl;
        } else if (h->cfg.gamma != b->gamma || h->cfg.nu != b->mu || h->cfg.prandtl != b->prandtl) {
            return fail(MGENKF_ERR_INVALID_ARG, "all handles of a batch share gamma, mu and Pr");
        }
        for (int j = 0; j < i; ++j)
            if (handles[j] == h) return fail(MGENKF_ERR_INVALID_ARG, "a handle appears twice");
        b->hs.push_back(h);
        b->obs_off.push_back(b->total_ny);
        b->total_ny += h->ny;
        for (int sz : {h->nc, h->nf})
            if (size_index(b, sz) < 0) {
                b->sizes.push_back(sz);
                b->shape.push_back(0);
            }
    }
    if (!b->s0) {
        // the legacy stream cannot be captured: a blocking stream keeps the
        // batch ordered with work the caller issues there
        if (cudaStreamCreate(&b->s0) != cudaSuccess) return fail(MGENKF_ERR_CUDA, "stream");
        b->own_s0 = true;
    }
    if (cudaMalloc(&b->obs_stage, b->total_ny * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->innov, b->hs.size() * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(MGENKF_ERR_OOM, "observation staging buffer");
    }
    // MGENKF_BATCH_STREAMS caps the analysis branches (used to measure how much
    // their concurrency buys)
    int cap = kDefaultBatchBranches;
    if (const char *e = getenv("MGENKF_BATCH_STREAMS")) cap = std::max(1, std::min(kMaxBatchStreams, atoi(e)));
    b->nbranch = std::min(n, cap);
    // longest-processing-time-first: problems in decreasing order of their
    // analysis cost, each onto the least-loaded branch.  Cost: the FP64 FMAs
    // of S and Y^T R^-1 [D | d*] plus the Cholesky's, and the ensemble
    // traffic of the anomalies and update at an eighth of the weight.
    {
        std::vector<double> cost(n);
        std::vector<int> order(n);
        for (int j = 0; j < n; ++j) {
            const mgenkf_ctx *h = b->hs[j];
            const double ne = h->ne, ny = h->ny, nx = (double)h->nx;
            cost[j] = ne * (2 * ne + 1) * ny + ne * ne * ne / 3 + nx * ne / 8;
            order[j] = j;
        }
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        std::vector<double> load(b->nbranch, 0.0);
        b->branch.assign(n, 0);
        for (int j : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            b->branch[j] = k;
            load[k] += cost[j];
        }
    }
    const int nsizes = (int)b->sizes.size();
    const int nstreams = nsizes + b->nbranch;
    for (int k = 0; k < nstreams; ++k) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(MGENKF_ERR_CUDA, "stream");
        b->aux.push_back(s);
    }
    for (int k = 0; k < 2 * nstreams + 2 * nsizes + 2; ++k) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(MGENKF_ERR_CUDA, "event");
        b->ev.push_back(e);
    }
    std::vector<std::vector<NsGroup<float>>> tab;
    build_tables(b, tab, 0, 0);
    if (upload_tables(b, tab) != MGENKF_OK) return fail(MGENKF_ERR_CUDA, b->err);
    *out = b;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_batch_destroy(mgenkf_batch_t b) {
    if (!b) return MGENKF_OK;
    cudaStreamSynchronize(b->s0);
    for (cudaStream_t s : b->aux) cudaStreamSynchronize(s);
    batch_free(b);
    delete b;
    return MGENKF_OK;
}

extern "C" const char *mgenkf_batch_last_error(mgenkf_batch_t b) { return b ? b->err.c_str() : ""; }

// forecast of every handle: one launch sequence per grid size, each on its own
// stream; the event ev[1 + k] marks the end of size k's steps.  join: s0
// waits for all of them (otherwise the analyses wait for their own sizes).
static mgenkf_status batch_forecast(mgenkf_batch *b, int nsteps, bool join) {
    B_CUDA(cudaEventRecord(b->ev[0], b->s0));
    const int ns = (int)b->sizes.size();
    for (int k = 0; k < ns; ++k) {
        cudaStream_t s = b->aux[b->nbranch + k];
        B_CUDA(cudaStreamWaitEvent(s, b->ev[0], 0));
        if (b->units[k]) {
            cudaError_t e = ns2d_forecast_table(b->d_groups[k], b->ngroups[k], b->units[k], b->sizes[k], nsteps,
                                                b->gamma, b->mu, b->prandtl, b->shape[k], s);
            if (e != cudaSuccess) B_FAIL(MGENKF_ERR_CUDA, std::string("batched forecast: ") + cudaGetErrorString(e));
        }
        B_CUDA(cudaEventRecord(b->ev[1 + k], s));
    }
    if (join)
        for (int k = 0; k < ns; ++k) B_CUDA(cudaStreamWaitEvent(b->s0, b->ev[1 + k], 0));
    return MGENKF_OK;
}

// analyses and prolongations of every handle, spread over the auxiliary streams
// Each problem's analysis waits only for the forecasts of its own two grid
// sizes, so analyses of problems whose grids are done run beside the
// remaining forecasts.
static mgenkf_status batch_analyse(mgenkf_batch *b) {
    const int base = 1 + (int)b->sizes.size();
    const int ns = b->nbranch;
    for (int k = 0; k < ns; ++k) B_CUDA(cudaStreamWaitEvent(b->aux[k], b->ev[0], 0));
    for (size_t j = 0; j < b->hs.size(); ++j) {
        mgenkf_ctx *h = b->hs[j];
        cudaStream_t keep = h->stream;
        h->stream = b->aux[b->branch[j]];
        B_CUDA(cudaStreamWaitEvent(h->stream, b->ev[1 + size_index(b, h->nc)], 0));
        B_CUDA(cudaStreamWaitEvent(h->stream, b->ev[1 + size_index(b, h->nf)], 0));
        mgenkf_status st = analyse_impl(h, b->obs_stage + b->obs_off[j], nullptr);
        if (st == MGENKF_OK) {
            launch_innov_rms(h->Z, h->ne, h->ny, b->innov + j, h->stream);
            st = prolong_impl(h);
        }
        h->stream = keep;
        if (st) B_FAIL(st, "problem " + std::to_string(j) + ": " + h->err);
    }
    for (int k = 0; k < ns; ++k) {
        B_CUDA(cudaEventRecord(b->ev[base + 1 + k], b->aux[k]));
        B_CUDA(cudaStreamWaitEvent(b->s0, b->ev[base + 1 + k], 0));
    }
    // every forecast stream joins back too (a size no problem's analysis waited on)
    for (int k = 0; k < (int)b->sizes.size(); ++k) B_CUDA(cudaStreamWaitEvent(b->s0, b->ev[1 + k], 0));
    return MGENKF_OK;
}

// whether handle h runs in the grouped analysis: the ensemble-space gain on the
// tensor-core update, without the re-centring, the learned correction or the
// final fine iteration, at sizes the grouped kernels take
static bool groupable(const mgenkf_ctx *h) {
    return !h->direct && h->df.Yh && !h->recentre && h->tc.ready && !h->cnn && !h->record_prev && h->alpha == 0.0 &&
           h->filter_sigma == 0.0 && group_supported(h->ne, h->ny);
}

// parts of the grouped cycle: MGENKF_BATCH_PARTS, default kDefaultBatchParts,
// at most one per problem
constexpr int kDefaultBatchParts = 2;
constexpr int kMaxBatchParts = 8;

static GroupProb group_prob(const mgenkf_batch *b, size_t j) {
    const mgenkf_ctx *h = b->hs[j];
    GroupProb g;
    memset(&g, 0, sizeof(g));
    g.fine = (float *)h->fine;
    g.members = (float *)h->members;
    g.xstar = (float *)h->xstar;
    g.dC = (float *)h->dC;
    g.tap_idx = h->tap_idx;
    g.tap_w = h->tap_w;
    g.tap_wh = h->tap_wh;
    g.tap_wl = h->tap_wl;
    g.yo_in = b->obs_stage + b->obs_off[j];
    g.yo = h->yo;
    g.yf = h->yf;
    g.ybar = h->ybar;
    g.eps = h->eps;
    g.Y = h->Y;
    g.Z = h->Z;
    g.S = h->S;
    g.Lt = h->Lt;
    g.Bt = h->Bt;
    g.part = h->gemm_part;
    g.df = h->df;
    g.innov = b->innov + j;
    g.Tt = h->Tt;
    g.status = h->status;
    g.cycle = h->cycle_d;
    g.seed = h->cfg.seed;
    g.sigma = h->cfg.obs_sigma;
    g.s2 = h->cfg.obs_sigma * h->cfg.obs_sigma;
    // the same host-side constants as the single-problem launches
    g.inv_ne = 1.0 / h->ne;
    g.isq = 1.0 / std::sqrt((double)(h->ne - 1));
    g.nc = h->nc;
    g.r = h->r;
    g.ne = h->ne;
    g.ny = h->ny;
    g.taps = h->taps;
    g.ldx = h->ldx;
    g.nx = (int)h->nx;
    g.splits = gemm_nt_splits(h->ne, h->ne, h->ne + 1, h->ny);
    g.kchunk = ceil_div(ceil_div(h->ny, g.splits), 32) * 32;
    g.kblocks = h->tc.kblocks;
    g.ntile = h->tc.ntile;
    g.tmem_cols = h->tc.tmem_cols;
    g.wait_limit = h->tc.wait_limit;
    g.pw = h->pw;
    return g;
}

// (Re)build the parts, their grouped plans and part tables when none exist,
// the part count changed or a handle's update wait limit changed, and the
// part tables when the forecast choices changed; b->grouped says whether the
// analyses run grouped.
static mgenkf_status batch_group_prepare(mgenkf_batch *b) {
    const char *env = getenv("MGENKF_BATCH_GROUPED");
    bool want = !(env && strcmp(env, "0") == 0);
    for (const mgenkf_ctx *h : b->hs) want = want && groupable(h);
    if (!want) {
        b->grouped = false;
        return MGENKF_OK;
    }
    int nparts = kDefaultBatchParts;
    if (const char *e = getenv("MGENKF_BATCH_PARTS")) nparts = atoi(e);
    nparts = std::max(1, std::min({nparts, kMaxBatchParts, (int)b->hs.size()}));
    bool fresh = b->nparts == nparts && (int)b->gplans.size() == nparts && b->gplan_wait.size() == b->hs.size();
    for (size_t j = 0; fresh && j < b->hs.size(); ++j) fresh = b->gplan_wait[j] == b->hs[j]->tc.wait_limit;
    if (fresh && b->grouped && !b->ptables_stale) return MGENKF_OK;
    // nothing may still read the old plans and tables
    B_CUDA(cudaStreamSynchronize(b->s0));
    for (cudaStream_t s : b->aux) B_CUDA(cudaStreamSynchronize(s));
    for (cudaStream_t s : b->pstreams) B_CUDA(cudaStreamSynchronize(s));
    if (!fresh) {
        for (GroupPlan &gp : b->gplans) group_plan_free(&gp);
        b->gplans.assign(nparts, GroupPlan());
        b->gplan_wait.clear();
        b->nparts = nparts;
        // parts with equal shares of the forecast work (points of the members
        // and the fine run per step)
        const size_t n = b->hs.size();
        std::vector<double> work(n);
        std::vector<int> order(n);
        for (size_t j = 0; j < n; ++j) {
            const mgenkf_ctx *h = b->hs[j];
            work[j] = (double)h->ne * h->nc * h->nc + (double)h->nf * h->nf;
            order[j] = (int)j;
        }
        b->part.assign(n, 0);
        // MGENKF_BATCH_SPLIT=work: the largest problems first onto the lightest
        // part, whatever their Ne (used to measure the default against it)
        const char *split = getenv("MGENKF_BATCH_SPLIT");
        if (!(split && strcmp(split, "work") == 0)) {
            // by ensemble size: the largest Ne first, each part filled to its
            // share of the forecast work, so the last part (whose analysis
            // follows the last forecast, exposed) holds the problems of the
            // shortest analysis chains (the Cholesky and solve latencies grow
            // with Ne) and the longer ones run beside the last forecast
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
                return b->hs[x]->ne != b->hs[y]->ne ? b->hs[x]->ne > b->hs[y]->ne : work[x] > work[y];
            });
            double total = 0.0, acc = 0.0;
            for (double v : work) total += v;
            int p = 0;
            for (int j : order) {
                b->part[j] = p;
                acc += work[j];
                while (p + 1 < nparts && acc >= total * (p + 1) / nparts) ++p;
            }
        } else {
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
            std::vector<double> load(nparts, 0.0);
            for (int j : order) {
                const int p = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                b->part[j] = p;
                load[p] += work[j];
            }
        }
        b->grouped = true;
        for (int p = 0; p < nparts && b->grouped; ++p) {
            std::vector<GroupProb> probs;
            std::vector<CUtensorMap> maps;
            for (size_t j = 0; j < n; ++j) {
                if (b->part[j] != p) continue;
                probs.push_back(group_prob(b, j));
                maps.push_back(b->hs[j]->tc.map_t);
                maps.push_back(b->hs[j]->tc.map_m);
            }
            b->grouped = !probs.empty() && group_plan_build(&b->gplans[p], probs, maps, b->s0);
        }
        if (!b->grouped) {
            cudaGetLastError();
            for (GroupPlan &gp : b->gplans) group_plan_free(&gp);
            b->gplans.clear();
            b->nparts = 0;
            return MGENKF_OK;
        }
        for (const mgenkf_ctx *h : b->hs) b->gplan_wait.push_back(h->tc.wait_limit);
        // streams and events of the parts
        const size_t need_s = (size_t)nparts * (b->sizes.size() + 1);
        while (b->pstreams.size() < need_s) {
            cudaStream_t st;
            B_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            b->pstreams.push_back(st);
        }
        while (b->pev.size() < need_s + 1) {
            cudaEvent_t ev;
            B_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            b->pev.push_back(ev);
        }
        b->ptables_stale = true;
    }
    if (b->ptables_stale) {
        mgenkf_status st = upload_part_tables(b);
        if (st) return st;
    }
    return MGENKF_OK;
}

// One grouped cycle: for each grid size the parts' forecasts one after the
// other on that size's stream of each part; part p's analysis waits for its own
// forecasts of every size and runs beside part p + 1's.
static mgenkf_status batch_cycle_grouped(mgenkf_batch *b, int nsteps) {
    const int ns = (int)b->sizes.size(), np = b->nparts;
    auto fstream = [&](int p, int k) { return b->pstreams[(size_t)p * (ns + 1) + k]; };
    auto fdone = [&](int p, int k) { return b->pev[(size_t)p * (ns + 1) + k]; };
    cudaEvent_t start = b->pev[(size_t)np * (ns + 1)];
    B_CUDA(cudaEventRecord(start, b->s0));
    for (int p = 0; p < np; ++p)
        for (int k = 0; k < ns; ++k) {
            cudaStream_t s = fstream(p, k);
            B_CUDA(cudaStreamWaitEvent(s, p == 0 ? start : fdone(p - 1, k), 0));
            const size_t t = (size_t)p * ns + k;
            if (b->punits[t]) {
                cudaError_t e = ns2d_forecast_table(b->pd_groups[t], b->pngroups[t], b->punits[t], b->sizes[k],
                                                    nsteps, b->gamma, b->mu, b->prandtl, b->shape[k], s);
                if (e != cudaSuccess)
                    B_FAIL(MGENKF_ERR_CUDA, std::string("batched forecast: ") + cudaGetErrorString(e));
            }
            B_CUDA(cudaEventRecord(fdone(p, k), s));
        }
    for (int p = 0; p < np; ++p) {
        cudaStream_t a = b->pstreams[(size_t)p * (ns + 1) + ns];
        for (int k = 0; k < ns; ++k) B_CUDA(cudaStreamWaitEvent(a, fdone(p, k), 0));
        cudaError_t e = group_analyse(b->gplans[p], a);
        if (e != cudaSuccess) B_FAIL(MGENKF_ERR_CUDA, std::string("grouped analysis: ") + cudaGetErrorString(e));
        cudaEvent_t adone = b->pev[(size_t)p * (ns + 1) + ns];
        B_CUDA(cudaEventRecord(adone, a));
        B_CUDA(cudaStreamWaitEvent(b->s0, adone, 0));
    }
    for (int k = 0; k < ns; ++k) B_CUDA(cudaStreamWaitEvent(b->s0, fdone(np - 1, k), 0));
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_batch_forecast(mgenkf_batch_t b, int32_t nsteps) {
    if (!b || nsteps < 0) return MGENKF_ERR_INVALID_ARG;
    b->err.clear();
    return batch_forecast(b, nsteps, true);
}

extern "C" mgenkf_status mgenkf_batch_cycle(mgenkf_batch_t b, int32_t nsteps, const double *y_obs,
                                            double *innov_out) {
    if (!b || nsteps < 0 || !y_obs) return MGENKF_ERR_INVALID_ARG;
    b->err.clear();
    B_CUDA(cudaMemcpyAsync(b->obs_stage, y_obs, b->total_ny * sizeof(double), cudaMemcpyDefault, b->s0));
    if (!b->exec || b->graph_nsteps != nsteps) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        {
            mgenkf_status st = batch_group_prepare(b);
            if (st) return st;
        }
        B_CUDA(cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeRelaxed));
        mgenkf_status st;
        if (b->grouped) {
            st = batch_cycle_grouped(b, nsteps);
        } else {
            st = batch_forecast(b, nsteps, false);
            if (st == MGENKF_OK) st = batch_analyse(b);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->s0, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) B_FAIL(MGENKF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        b->graph = g;
        B_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
        b->graph_nsteps = nsteps;
    }
    B_CUDA(cudaGraphLaunch(b->exec, b->s0));
    if (innov_out)
        B_CUDA(cudaMemcpyAsync(innov_out, b->innov, b->hs.size() * sizeof(double), cudaMemcpyDefault, b->s0));
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_batch_sync(mgenkf_batch_t b) {
    if (!b) return MGENKF_ERR_INVALID_ARG;
    B_CUDA(cudaStreamSynchronize(b->s0));
    mgenkf_status first = MGENKF_OK;
    for (size_t j = 0; j < b->hs.size(); ++j) {
        mgenkf_status st = mgenkf_sync(b->hs[j]);
        if (st && !first) {
            first = st;
            b->err = "problem " + std::to_string(j) + ": " + b->hs[j]->err;
        }
    }
    return first;
}

// Time one step into the scratch buffers (the states are not touched) of
// every grid size with every segment choice and keep the fastest per size.
constexpr int kJointSteps = 4;  // model steps per stream of one joint probe

// `reps` timings (after one warm-up) of `steps` model steps of every grid size
// at once, each size on its own stream as the forecast runs them, with the
// current choices; the steps write to scratch, the states stay as they are.
// The fastest repetition's milliseconds in *ms.
static mgenkf_status probe_joint(mgenkf_batch *b, int steps, int reps, float *ms) {
    std::vector<std::vector<NsGroup<float>>> tab;
    build_tables(b, tab, 0, 0);
    const int ns = (int)b->sizes.size();
    std::vector<NsGroup<float> *> d(ns, nullptr);
    std::vector<int> units(ns, 0);
    mgenkf_status st = MGENKF_OK;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    auto cuda = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == MGENKF_OK) {
            b->err = std::string("autotune: ") + what + ": " + cudaGetErrorString(e);
            st = MGENKF_ERR_CUDA;
        }
        return st == MGENKF_OK;
    };
    for (int k = 0; k < ns && st == MGENKF_OK; ++k) {
        if (tab[k].empty()) continue;
        const NsGroup<float> &last = tab[k].back();
        units[k] = last.tile_begin + last.tx * last.ty * last.nprob;
        if (cuda(cudaMalloc(&d[k], tab[k].size() * sizeof(NsGroup<float>)), "cudaMalloc"))
            cuda(cudaMemcpyAsync(d[k], tab[k].data(), tab[k].size() * sizeof(NsGroup<float>),
                                 cudaMemcpyHostToDevice, b->s0),
                 "cudaMemcpyAsync");
    }
    cuda(cudaEventCreate(&t0), "cudaEventCreate") && cuda(cudaEventCreate(&t1), "cudaEventCreate");
    *ms = 0.f;
    for (int r = 0; r <= reps && st == MGENKF_OK; ++r) {  // first repetition warms up
        cuda(cudaEventRecord(t0, b->s0), "cudaEventRecord");
        cuda(cudaEventRecord(b->ev[0], b->s0), "cudaEventRecord");
        for (int k = 0; k < ns && st == MGENKF_OK; ++k) {
            cudaStream_t s = b->aux[b->nbranch + k];
            cuda(cudaStreamWaitEvent(s, b->ev[0], 0), "cudaStreamWaitEvent");
            for (int i = 0; i < steps && units[k] && st == MGENKF_OK; ++i)
                cuda(ns2d_probe_step(d[k], (int)tab[k].size(), units[k], b->sizes[k], b->gamma, b->mu, b->prandtl,
                                     b->shape[k], s),
                     "probe step");
            cuda(cudaEventRecord(b->ev[1 + k], s), "cudaEventRecord");
            cuda(cudaStreamWaitEvent(b->s0, b->ev[1 + k], 0), "cudaStreamWaitEvent");
        }
        cuda(cudaEventRecord(t1, b->s0), "cudaEventRecord");
        cuda(cudaEventSynchronize(t1), "cudaEventSynchronize");
        float t = 0.f;
        if (cuda(cudaEventElapsedTime(&t, t0, t1), "cudaEventElapsedTime") && r) *ms = r == 1 ? t : std::min(*ms, t);
    }
    cudaStreamSynchronize(b->s0);
    for (NsGroup<float> *p : d)
        if (p) cudaFree(p);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return st;
}

extern "C" mgenkf_status mgenkf_batch_autotune(mgenkf_batch_t b, int32_t reps) {
    if (!b || reps < 1) return MGENKF_ERR_INVALID_ARG;
    b->err.clear();
    cudaEvent_t t0, t1;
    B_CUDA(cudaEventCreate(&t0));
    B_CUDA(cudaEventCreate(&t1));
    NsGroup<float> *d = nullptr;
    std::vector<float> alone(b->sizes.size(), 0.f);
    for (size_t si = 0; si < b->sizes.size(); ++si) {
        float best = 1e30f;
        int best_shape = 0;
        for (int sh = 0; sh < kNsTileShapes; ++sh) {
            std::vector<std::vector<NsGroup<float>>> tab;
            build_tables(b, tab, b->sizes[si], sh);
            const int ng = (int)tab[si].size();
            if (!ng) continue;
            const NsGroup<float> &last = tab[si].back();
            const int units = last.tile_begin + last.tx * last.ty * last.nprob;
            B_CUDA(cudaMalloc(&d, ng * sizeof(NsGroup<float>)));
            B_CUDA(cudaMemcpyAsync(d, tab[si].data(), ng * sizeof(NsGroup<float>), cudaMemcpyHostToDevice, b->s0));
            float ms = 0.f;
            for (int r = 0; r <= reps; ++r) {  // first repetition warms up
                B_CUDA(cudaEventRecord(t0, b->s0));
                cudaError_t e = ns2d_probe_step(d, ng, units, b->sizes[si], b->gamma, b->mu, b->prandtl, sh, b->s0);
                if (e != cudaSuccess) B_FAIL(MGENKF_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
                B_CUDA(cudaEventRecord(t1, b->s0));
                B_CUDA(cudaEventSynchronize(t1));
                float t = 0.f;
                B_CUDA(cudaEventElapsedTime(&t, t0, t1));
                if (r) ms = r == 1 ? t : std::min(ms, t);
            }
            cudaFree(d);
            d = nullptr;
            if (ms < best) {
                best = ms;
                best_shape = sh;
            }
        }
        b->shape[si] = best_shape;
        alone[si] = best;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    // Alone, a size's last partial wave of CTAs counts in full; in the cycle the
    // sizes step at once and fill each other's tails.  So, size by size (the
    // slowest first), every choice is timed again with all sizes stepping
    // together on their own streams, and the fastest joint choice is kept.
    const int ns = (int)b->sizes.size();
    if (ns > 1) {
        std::vector<int> order(ns);
        for (int k = 0; k < ns; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return alone[x] > alone[y]; });
        for (int si : order) {
            float best = 1e30f;
            int best_shape = b->shape[si];
            for (int sh = 0; sh < kNsTileShapes; ++sh) {
                b->shape[si] = sh;
                float ms = 0.f;
                mgenkf_status st = probe_joint(b, kJointSteps, reps, &ms);
                if (st) return st;
                if (ms < best) {
                    best = ms;
                    best_shape = sh;
                }
            }
            b->shape[si] = best_shape;
        }
    }
    std::vector<std::vector<NsGroup<float>>> tab;
    build_tables(b, tab, 0, 0);
    return upload_tables(b, tab);
}

extern "C" mgenkf_status mgenkf_batch_tiles(mgenkf_batch_t b, int32_t *sizes, int32_t *shapes, int32_t max,
                                            int32_t *count) {
    if (!b || !count) return MGENKF_ERR_INVALID_ARG;
    *count = (int32_t)b->sizes.size();
    for (int32_t i = 0; i < *count && i < max; ++i) {
        if (sizes) sizes[i] = b->sizes[i];
        if (shapes) shapes[i] = b->shape[i];
    }
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_batch_set_tiles(mgenkf_batch_t b, const int32_t *sizes, const int32_t *shapes,
                                                int32_t count) {
    if (!b || (count > 0 && (!sizes || !shapes))) return MGENKF_ERR_INVALID_ARG;
    b->err.clear();
    for (int32_t i = 0; i < count; ++i) {
        if (shapes[i] < 0 || shapes[i] >= kNsTileShapes) B_FAIL(MGENKF_ERR_INVALID_ARG, "segment choice out of range");
        const int si = size_index(b, sizes[i]);
        if (si >= 0) b->shape[si] = shapes[i];
    }
    std::vector<std::vector<NsGroup<float>>> tab;
    build_tables(b, tab, 0, 0);
    return upload_tables(b, tab);
}
