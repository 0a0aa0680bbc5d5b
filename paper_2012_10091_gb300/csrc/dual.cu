// dual.cu -- multigrid Dual EnKF with parameter estimation on the Burgers
// inlet model (Sec. 4: Eqs. burgers and inlet-1D-Burgers; Algorithm 3 with its
// parameter rows, run inside Algorithm 4), FP64.
//
// Model: nodes x_j = j dx; node 0 holds the inlet u0 (1 + theta1 sin(omega t +
// theta2)), the outlet node is extrapolated linearly, the interior follows the
// flux-form central scheme; SSP-RK3 in Shu-Osher form with the inlet set at
// each stage's time.  One CTA advances one grid held in shared memory.
//
// One cycle (mgenkf_dual_cycle):
//   fine forecast with the analysed parameter mean of the previous cycle;
//   parameter forecast theta^f = theta^a + tau (random walk, Philox normals);
//   member forecast with theta^f; perturbed observations; parameter update
//   theta^a = theta^f + Theta T, T = (I + Y^T R^-1 Y)^-1 Y^T R^-1 D (ensemble
//   space, exact R = sigma^2 I); member forecast again from the previous
//   analysis with theta^a; state update x^a = x^f + X T with the same
//   perturbations; fine correction x^F += Pi_F(X T_ne) with d* = y^o - H^C x^C*.
// Projections are open-grid 4-point Lagrange interpolants (one-sided at the
// ends); H^C is the Pi_F row at each observed fine node.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mgenkf.h"
#include "analysis.h"
#include "common.cuh"

namespace mgk {

constexpr uint64_t kThetaTag = 0x54485441ULL;  // "THTA": parameter random walk
constexpr int kDualMaxPts = 1024;               // points per grid (one CTA, one point per thread)

// SSP-RK3 steps of nprob inlet-Burgers grids of n points (one CTA each)
__global__ void __launch_bounds__(1024) k_burgers_inlet(double *__restrict__ u, int n, double dx, double nu,
                                                        double dt, int nsteps, double t0,
                                                        const double *__restrict__ theta, double u0, double omega) {
    extern __shared__ double sh[];
    double *x = sh, *u1 = sh + n, *u2 = sh + 2 * n;
    const int j = threadIdx.x;
    double *g = u + (size_t)blockIdx.x * n;
    const double th1 = theta[2 * blockIdx.x], th2 = theta[2 * blockIdx.x + 1];
    if (j < n) x[j] = g[j];
    const double i2dx = 1.0 / (2.0 * dx), idx2 = 1.0 / (dx * dx);
    auto L = [&](const double *v) {
        const double fp = 0.5 * v[j + 1] * v[j + 1], fm = 0.5 * v[j - 1] * v[j - 1];
        return -(fp - fm) * i2dx + nu * (v[j + 1] - 2.0 * v[j] + v[j - 1]) * idx2;
    };
    auto bc = [&](double *v, double t) {  // after the interior of v is complete
        if (j == 0) v[0] = u0 * (1.0 + th1 * sin(omega * t + th2));
        if (j == n - 1) v[n - 1] = 2.0 * v[n - 2] - v[n - 3];
    };
    const bool in = j > 0 && j < n - 1;
    for (int s = 0; s < nsteps; ++s) {
        const double t = t0 + s * dt;
        __syncthreads();
        if (in) u1[j] = x[j] + dt * L(x);
        __syncthreads();
        bc(u1, t + dt);
        __syncthreads();
        if (in) u2[j] = 0.75 * x[j] + 0.25 * (u1[j] + dt * L(u1));
        __syncthreads();
        bc(u2, t + 0.5 * dt);
        __syncthreads();
        double xn = 0.0;
        if (in) xn = x[j] / 3.0 + 2.0 / 3.0 * (u2[j] + dt * L(u2));
        __syncthreads();  // every read of x in this step is done
        if (in) x[j] = xn;
        __syncthreads();
        bc(x, t + dt);
    }
    __syncthreads();
    if (j < n) g[j] = x[j];
}

// theta^f = theta^a + sqrt(q) tau
__global__ void k_theta_walk(const double *__restrict__ theta, const double *__restrict__ tau, double sq, int count,
                             double *__restrict__ theta_f) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) theta_f[e] = theta[e] + sq * tau[e];
}

// theta^a_i = theta^f_i + sum_a Theta[p][a] T[a][i], Theta the normalised
// parameter anomalies; T column i at Tm[i ne ..]; then (thread 0) the mean
__global__ void k_theta_update(const double *__restrict__ theta_f, const double *__restrict__ Tm, int ne,
                               double *__restrict__ theta_a, double *__restrict__ theta_mean, const int *status) {
    if (*status) return;
    __shared__ double mean[2];
    if (threadIdx.x < 2) {
        double m = 0.0;
        for (int a = 0; a < ne; ++a) m += theta_f[2 * a + threadIdx.x];
        mean[threadIdx.x] = m / ne;
    }
    __syncthreads();
    const double isq = 1.0 / sqrt((double)(ne - 1));
    for (int e = threadIdx.x; e < 2 * ne; e += blockDim.x) {
        const int i = e >> 1, p = e & 1;
        double acc = 0.0;
        for (int a = 0; a < ne; ++a) acc = fma((theta_f[2 * a + p] - mean[p]) * isq, Tm[(size_t)i * ne + a], acc);
        theta_a[e] = theta_f[e] + acc;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double m = 0.0;
        for (int a = 0; a < ne; ++a) m += theta_a[2 * a + threadIdx.x];
        theta_mean[threadIdx.x] = m / ne;
    }
}

// fine += Pi_F(dC) on the open grid: 4 taps from j0[k]
__global__ void k_prolong_open(double *__restrict__ fine, const double *__restrict__ dC, int nf,
                               const int32_t *__restrict__ j0, const double *__restrict__ w, const int *status) {
    if (*status) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    const double *wk = w + 4 * (size_t)k;
    const double *d = dC + j0[k];
    fine[k] += wk[0] * d[0] + wk[1] * d[1] + wk[2] * d[2] + wk[3] * d[3];
}

}  // namespace mgk

using namespace mgk;

struct mgenkf_dual {
    mgenkf_dual_config cfg;
    int nf = 0, nc = 0, ne = 0, ny = 0;
    double t = 0.0;
    uint64_t cycle = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr;  // the fine forecast runs beside the members' forecasts and first analysis
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double *xstar_a = nullptr;   // x^C* stand-in of the parameter analysis (its d* column is not used)
    double *fine = nullptr, *members = nullptr, *prev = nullptr, *theta = nullptr, *theta_f = nullptr;
    double *theta_mean = nullptr, *tau = nullptr, *xstar = nullptr, *dC = nullptr;
    double *yf = nullptr, *yo = nullptr, *ybar = nullptr, *eps = nullptr, *Y = nullptr, *Z = nullptr;
    double *X = nullptr, *S = nullptr, *Lt = nullptr, *Bt = nullptr, *part = nullptr;
    double *tap_w = nullptr, *pro_w = nullptr;
    int32_t *tap_idx = nullptr, *pro_j0 = nullptr;
    uint64_t *cycle_d = nullptr;
    int *status = nullptr;
    std::string err;
};

namespace {

// cubic Lagrange weights through nodes j0 .. j0 + 3 at position s (coarse index units)
void lagrange4(int j0, double s, double w[4]) {
    for (int a = 0; a < 4; ++a) {
        double v = 1.0;
        for (int b = 0; b < 4; ++b)
            if (b != a) v *= (s - (j0 + b)) / (double)(a - b);
        w[a] = v;
    }
}

int open_j0(int k, int r, int nc) {
    int j0 = k / r - 1;
    if (j0 > nc - 4) j0 = nc - 4;
    if (j0 < 0) j0 = 0;
    return j0;
}

void free_dual(mgenkf_dual *d) {
    void *p[] = {d->fine, d->members, d->prev, d->theta, d->theta_f, d->theta_mean, d->tau, d->xstar, d->dC,
                 d->yf, d->yo, d->ybar, d->eps, d->Y, d->Z, d->X, d->S, d->Lt, d->Bt, d->part, d->tap_w,
                 d->pro_w, d->tap_idx, d->pro_j0, d->cycle_d, d->status};
    for (void *q : p)
        if (q) cudaFree(q);
    if (d->xstar_a) cudaFree(d->xstar_a);
    for (cudaEvent_t e : d->ev)
        if (e) cudaEventDestroy(e);
    if (d->aux) cudaStreamDestroy(d->aux);
}

void forecast(mgenkf_dual *d, double *grids, int nprob, int n, const double *theta, int nsteps,
              cudaStream_t s = nullptr) {
    count_launches(1);
    k_burgers_inlet<<<nprob, ((n + 31) / 32) * 32, 3 * n * sizeof(double), s ? s : d->stream>>>(
        grids, n, d->cfg.length / n, d->cfg.nu, d->cfg.dt, nsteps, d->t, theta, d->cfg.u0, d->cfg.omega);
}

// perturbations (generated once per cycle), anomalies and T = S^-1 B (ensemble space)
void gain_solve(mgenkf_dual *d, int gen_eps, const double *xstar) {
    const cudaStream_t s = d->stream;
    const int ne = d->ne, ny = d->ny;
    launch_obs_apply<double>(d->members, xstar, d->nc, ne, ny, 4, d->tap_idx, d->tap_w, d->yf, s);
    launch_obs_mean(d->yf, d->yo, ne, ny, d->ybar, d->Z, d->status, s);
    launch_obs_perturb(d->yf, d->ybar, d->yo, d->eps, gen_eps, d->cfg.seed, d->cycle_d, d->cfg.obs_sigma, ne,
                       ny, d->Y, d->Z, s);
    const double s2 = d->cfg.obs_sigma * d->cfg.obs_sigma;
    launch_gemm_nt_f64(d->Y, ne, d->Y, ne, d->Z, ne + 1, ny, s2, 1.0, d->S, d->Bt, d->status, s, d->part);
    launch_cholesky(d->S, d->Lt, ne, d->status, s);
    launch_chol_solve(d->S, d->Lt, ne, d->Bt, d->Bt, ne + 1, nullptr, 0, d->status, s);
}

}  // namespace

#define D_FAIL(code, msg) \
    do {                  \
        d->err = (msg);   \
        return (code);    \
    } while (0)
#define D_CUDA(x)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) D_FAIL(MGENKF_ERR_CUDA, std::string(cudaGetErrorString(e_))); \
    } while (0)

extern "C" mgenkf_status mgenkf_dual_create(const mgenkf_dual_config *cfg, const int32_t *obs_index,
                                            void *cuda_stream, mgenkf_dual_t *out) {
    if (!cfg || !obs_index || !out) return MGENKF_ERR_INVALID_ARG;
    *out = nullptr;
    const mgenkf_dual_config &c = *cfg;
    if (c.ratio < 1 || c.ratio > 16 || c.n_fine % c.ratio != 0 || c.n_fine > kDualMaxPts ||
        c.n_fine / c.ratio < 8 || c.n_members < 2 || c.n_members > 256 || c.n_obs < 1 ||
        !(c.dt > 0.0) || !(c.length > 0.0) || !(c.nu >= 0.0) || !(c.obs_sigma > 0.0) || !(c.theta_q >= 0.0)) {
        mgk_set_error("mgenkf_dual_create: sizes or parameters out of range");
        return MGENKF_ERR_INVALID_ARG;
    }
    for (int j = 0; j < c.n_obs; ++j)
        if (obs_index[j] < 0 || obs_index[j] >= c.n_fine) {
            mgk_set_error("mgenkf_dual_create: observation index outside the fine grid");
            return MGENKF_ERR_INVALID_ARG;
        }
    mgenkf_dual *d = new mgenkf_dual();
    d->cfg = c;
    d->nf = c.n_fine;
    d->nc = c.n_fine / c.ratio;
    d->ne = c.n_members;
    d->ny = c.n_obs;
    d->stream = (cudaStream_t)cuda_stream;
    const size_t ne = d->ne, ny = d->ny, nc = d->nc, nf = d->nf;
    struct A {
        void **p;
        size_t bytes;
    } al[] = {
        {(void **)&d->fine, nf * 8}, {(void **)&d->members, ne * nc * 8}, {(void **)&d->prev, ne * nc * 8},
        {(void **)&d->theta, 2 * ne * 8}, {(void **)&d->theta_f, 2 * ne * 8}, {(void **)&d->theta_mean, 2 * 8},
        {(void **)&d->tau, 2 * ne * 8 + 32}, {(void **)&d->xstar, nc * 8}, {(void **)&d->dC, nc * 8},
        {(void **)&d->yf, (ne + 1) * ny * 8}, {(void **)&d->yo, ny * 8}, {(void **)&d->ybar, ny * 8},
        {(void **)&d->eps, ne * ny * 8}, {(void **)&d->Y, ne * ny * 8}, {(void **)&d->Z, (ne + 1) * ny * 8},
        {(void **)&d->X, ne * nc * 8}, {(void **)&d->S, ne * ne * 8}, {(void **)&d->Lt, ne * ne * 8},
        {(void **)&d->Bt, (ne + 1) * ne * 8},
        {(void **)&d->part, (size_t)gemm_nt_splits((int)ne, (int)ne, (int)ne + 1, (int)ny) * ne * (2 * ne + 1) * 8},
        {(void **)&d->tap_w, ny * 4 * 8}, {(void **)&d->pro_w, nf * 4 * 8}, {(void **)&d->tap_idx, ny * 4 * 4},
        {(void **)&d->pro_j0, nf * 4}, {(void **)&d->cycle_d, 8}, {(void **)&d->status, 4},
        {(void **)&d->xstar_a, nc * 8},
    };
    for (auto &a : al) {
        if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            free_dual(d);
            delete d;
            mgk_set_error("mgenkf_dual_create: device allocation failed");
            return MGENKF_ERR_OOM;
        }
    }
    // open-grid H^C taps (absolute coarse indices) and Pi_F rows
    std::vector<int32_t> ti(ny * 4), pj(nf);
    std::vector<double> tw(ny * 4), pw(nf * 4);
    for (size_t k = 0; k < nf; ++k) {
        const int j0 = open_j0((int)k, c.ratio, d->nc);
        pj[k] = j0;
        lagrange4(j0, (double)k / c.ratio, &pw[4 * k]);
    }
    for (size_t j = 0; j < ny; ++j) {
        const int k = obs_index[j];
        for (int t = 0; t < 4; ++t) {
            ti[4 * j + t] = pj[k] + t;
            tw[4 * j + t] = pw[4 * (size_t)k + t];
        }
    }
    if (cudaStreamCreateWithFlags(&d->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaMemsetAsync(d->xstar_a, 0, nc * 8, d->stream) != cudaSuccess) {
        cudaGetLastError();
        free_dual(d);
        delete d;
        mgk_set_error("mgenkf_dual_create: stream or event creation failed");
        return MGENKF_ERR_CUDA;
    }
    const uint64_t zero = 0;
    const int zs = 0;
    bool ok = cudaMemcpyAsync(d->tap_idx, ti.data(), ti.size() * 4, cudaMemcpyHostToDevice, d->stream) == cudaSuccess &&
              cudaMemcpyAsync(d->tap_w, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice, d->stream) == cudaSuccess &&
              cudaMemcpyAsync(d->pro_j0, pj.data(), pj.size() * 4, cudaMemcpyHostToDevice, d->stream) == cudaSuccess &&
              cudaMemcpyAsync(d->pro_w, pw.data(), pw.size() * 8, cudaMemcpyHostToDevice, d->stream) == cudaSuccess &&
              cudaMemcpyAsync(d->cycle_d, &zero, 8, cudaMemcpyHostToDevice, d->stream) == cudaSuccess &&
              cudaMemcpyAsync(d->status, &zs, 4, cudaMemcpyHostToDevice, d->stream) == cudaSuccess &&
              cudaStreamSynchronize(d->stream) == cudaSuccess;
    if (!ok) {
        free_dual(d);
        delete d;
        mgk_set_error("mgenkf_dual_create: CUDA error during set-up");
        return MGENKF_ERR_CUDA;
    }
    *out = d;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_dual_set_state(mgenkf_dual_t d, const double *fine, const double *members,
                                               const double *theta, const double *theta_fine, double t0) {
    if (!d || !fine || !members || !theta || !theta_fine) return MGENKF_ERR_INVALID_ARG;
    d->err.clear();
    D_CUDA(cudaMemcpyAsync(d->fine, fine, d->nf * 8, cudaMemcpyDefault, d->stream));
    D_CUDA(cudaMemcpyAsync(d->members, members, (size_t)d->ne * d->nc * 8, cudaMemcpyDefault, d->stream));
    D_CUDA(cudaMemcpyAsync(d->theta, theta, 2 * (size_t)d->ne * 8, cudaMemcpyDefault, d->stream));
    D_CUDA(cudaMemcpyAsync(d->theta_mean, theta_fine, 2 * 8, cudaMemcpyDefault, d->stream));
    D_CUDA(cudaStreamSynchronize(d->stream));
    d->t = t0;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_dual_free_run(mgenkf_dual_t d, int32_t nsteps) {
    if (!d || nsteps < 0) return MGENKF_ERR_INVALID_ARG;
    d->err.clear();
    if (nsteps == 0) return MGENKF_OK;
    forecast(d, d->fine, 1, d->nf, d->theta_mean, nsteps);
    forecast(d, d->members, d->ne, d->nc, d->theta, nsteps);
    D_CUDA(cudaGetLastError());
    d->t += nsteps * d->cfg.dt;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_dual_cycle(mgenkf_dual_t d, int32_t nsteps, const double *y_obs) {
    if (!d || nsteps < 1 || !y_obs) return MGENKF_ERR_INVALID_ARG;
    d->err.clear();
    const cudaStream_t s = d->stream;
    const int ne = d->ne, nc = d->nc;
    D_CUDA(cudaMemcpyAsync(d->yo, y_obs, d->ny * sizeof(double), cudaMemcpyDefault, s));
    // Algorithm 4 step 2: the fine run with the analysed parameter mean, on the
    // auxiliary stream beside the members' forecasts and the parameter analysis
    // (theta_mean is rewritten only after the join below)
    D_CUDA(cudaEventRecord(d->ev[0], s));
    D_CUDA(cudaStreamWaitEvent(d->aux, d->ev[0], 0));
    forecast(d, d->fine, 1, d->nf, d->theta_mean, nsteps, d->aux);
    launch_restrict<double>(d->fine, d->xstar, 1, 1, nc, d->cfg.ratio, d->aux);
    D_CUDA(cudaEventRecord(d->ev[1], d->aux));
    // Algorithm 3 step 2: parameter random walk, members forecast with theta^f
    D_CUDA(cudaMemcpyAsync(d->prev, d->members, (size_t)ne * nc * 8, cudaMemcpyDeviceToDevice, s));
    launch_normals(d->cfg.seed, kThetaTag, d->cycle, 2 * (int64_t)ne, d->tau, s);
    count_launches(1);
    k_theta_walk<<<ceil_div(2 * ne, 256), 256, 0, s>>>(d->theta, d->tau, std::sqrt(d->cfg.theta_q), 2 * ne,
                                                        d->theta_f);
    forecast(d, d->members, ne, nc, d->theta_f, nsteps);
    // steps 3-5: perturbed observations, parameter update theta^a = theta^f + Theta T
    gain_solve(d, 1, d->xstar_a);
    D_CUDA(cudaStreamWaitEvent(s, d->ev[1], 0));  // join: the fine forecast has read theta_mean
    count_launches(1);
    k_theta_update<<<1, 256, 0, s>>>(d->theta_f, d->Bt, ne, d->theta, d->theta_mean, d->status);
    // steps 6-8: members forecast again from the previous analysis with theta^a, state update
    D_CUDA(cudaMemcpyAsync(d->members, d->prev, (size_t)ne * nc * 8, cudaMemcpyDeviceToDevice, s));
    forecast(d, d->members, ne, nc, d->theta, nsteps);
    gain_solve(d, 0, d->xstar);  // the same perturbations
    launch_ens_anom<double>(d->members, nc, ne, d->X, nullptr, d->status, s);
    D_CUDA(cudaMemsetAsync(d->dC, 0, nc * sizeof(double), s));
    launch_update_f64<double>(d->members, d->dC, d->X, d->Bt, nc, ne, d->status, s);
    // Algorithm 4 step 5: x^F += Pi_F(x^C' - x^C*)
    count_launches(1);
    k_prolong_open<<<ceil_div(d->nf, 256), 256, 0, s>>>(d->fine, d->dC, d->nf, d->pro_j0, d->pro_w, d->status);
    launch_bump_counter(d->cycle_d, s);
    D_CUDA(cudaGetLastError());
    d->t += nsteps * d->cfg.dt;
    d->cycle += 1;
    return MGENKF_OK;
}

extern "C" mgenkf_status mgenkf_dual_get_state(mgenkf_dual_t d, double *fine, double *members, double *theta,
                                               double *theta_fine) {
    if (!d) return MGENKF_ERR_INVALID_ARG;
    d->err.clear();
    D_CUDA(cudaStreamSynchronize(d->stream));
    int st = 0;
    D_CUDA(cudaMemcpy(&st, d->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (fine) D_CUDA(cudaMemcpy(fine, d->fine, d->nf * 8, cudaMemcpyDefault));
    if (members) D_CUDA(cudaMemcpy(members, d->members, (size_t)d->ne * d->nc * 8, cudaMemcpyDefault));
    if (theta) D_CUDA(cudaMemcpy(theta, d->theta, 2 * (size_t)d->ne * 8, cudaMemcpyDefault));
    if (theta_fine) D_CUDA(cudaMemcpy(theta_fine, d->theta_mean, 2 * 8, cudaMemcpyDefault));
    if (st) D_FAIL((mgenkf_status)st, "a device-side check failed (non-positive pivot or non-finite observation)");
    return MGENKF_OK;
}

extern "C" const char *mgenkf_dual_last_error(mgenkf_dual_t d) { return d ? d->err.c_str() : ""; }

extern "C" mgenkf_status mgenkf_dual_destroy(mgenkf_dual_t d) {
    if (!d) return MGENKF_OK;
    cudaStreamSynchronize(d->stream);
    free_dual(d);
    delete d;
    return MGENKF_OK;
}
