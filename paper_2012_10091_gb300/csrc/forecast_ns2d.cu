// forecast_ns2d.cu -- batched SSP-RK3 forecast of the 2-D compressible
// Navier-Stokes equations (Eqs. Mass, Momentum, Energy) on periodic grids.
//
// State: 4 planes (rho, rho u, rho v, E) of n x n points, x fastest.  With
// u = (rho u)/rho, v = (rho v)/rho, p = (gamma-1)(E - rho |u|^2 / 2), T = p/rho:
//   dq/dt = -(F_{i+1} - F_{i-1}) / (2h) - (G_{j+1} - G_{j-1}) / (2h)
//           + (Fv_{i+1/2} - Fv_{i-1/2}) / h + (Gv_{j+1/2} - Gv_{j-1/2}) / h
// with nodal inviscid fluxes F = (rho u, rho u u + p, rho u v, (E + p) u),
// G = (rho v, rho v u, rho v v + p, (E + p) v) and face viscous/heat fluxes
// Fv = (0, t_xx, t_xy, t_xx u_f + t_xy v_f + kappa T_x) (normal derivatives
// compact across the face, tangential ones the average of the two central
// differences, face velocities the average of the two nodes), likewise Gv;
// t_xx = mu (4/3 u_x - 2/3 v_y), t_xy = mu (u_y + v_x), kappa = mu gamma /
// ((gamma - 1) Pr).  Every flux telescopes, so the four totals are conserved.
//
// GPU design: one launch per RK stage over every grid of the cycle (Ne members
// and the fine run).  A CTA owns a 32 x 8 tile: it loads the stage input of
// the tile and its one-point halo (periodic wrap) into shared memory, forms the
// primitives once per loaded point, and each thread evaluates the 9-point
// stencil of its point.  Stages: s1 = u0 + k(u0), s2 = u0 + ((s1 - u0) + k(s1))/4,
// u' = u0 + 2/3 ((s2 - u0) + k(s2)), k = dt L (Shu-Osher form rearranged);
// s1 and s2 live in two scratch buffers so a stage never overwrites a value
// another CTA still reads.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "forecast_ns2d.h"

namespace mgk {

constexpr int kNsTx = 32, kNsTy = 8;

template <typename T>
struct NsArgs {
    NsGroup<T> g[2];
    int tiles0;  // tiles of group 0
    T gm1, mu, kappa;
};

// The stencil body is written for a tile shape TX x TY (TX * TY = 256
// threads); the batched path picks the shape per grid size (autotuned).
template <typename T, int STAGE, int TX, int TY>
__device__ __forceinline__ void ns2d_stage_tile(const NsGroup<T> &G, int tile, T gm1, T mu, T kap) {
    constexpr int HX = TX + 2, HY = TY + 2, HALO = HX * HY;
    __shared__ T sq[4][HALO];   // conserved variables of the tile + halo
    __shared__ T spr[4][HALO];  // u, v, p, T
    const int tiles_per_prob = G.tx * G.ty;
    const int prob = tile / tiles_per_prob;
    const int tt = tile % tiles_per_prob;
    const int x0 = (tt % G.tx) * TX, y0 = (tt / G.tx) * TY;
    const int n = G.n;
    const size_t plane = (size_t)n * n;
    T *u0 = G.u0 + (size_t)prob * 4 * plane;
    const T *in = STAGE == 0 ? u0 : (STAGE == 1 ? G.s1 : G.s2) + (size_t)prob * 4 * plane;
    T *out = STAGE == 0 ? G.s1 + (size_t)prob * 4 * plane
                        : (STAGE == 1 ? G.s2 + (size_t)prob * 4 * plane : u0);

    // load the tile and its halo, form the primitives
    for (int e = threadIdx.x; e < HALO; e += blockDim.x) {
        const int ly = e / HX, lx = e % HX;
        int gy = y0 + ly - 1, gx = x0 + lx - 1;  // periodic wrap without integer division
        if (gy < 0) gy += n;
        if (gx < 0) gx += n;
        while (gy >= n) gy -= n;
        while (gx >= n) gx -= n;
        const size_t o = (size_t)gy * n + gx;
        const T rho = in[o], mx = in[plane + o], my = in[2 * plane + o], E = in[3 * plane + o];
        const T rinv = T(1) / rho;  // one division per point
        const T u = mx * rinv, v = my * rinv;
        const T p = gm1 * (E - T(0.5) * rho * (u * u + v * v));
        sq[0][e] = rho;
        sq[1][e] = mx;
        sq[2][e] = my;
        sq[3][e] = E;
        spr[0][e] = u;
        spr[1][e] = v;
        spr[2][e] = p;
        spr[3][e] = p * rinv;
    }
    __syncthreads();
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= n || y >= n) return;
    const int c = (ly + 1) * HX + (lx + 1);
    const int e_ = c + 1, w_ = c - 1, n_ = c + HX, s_ = c - HX;
    const T *U = spr[0], *V = spr[1], *P = spr[2], *TT = spr[3];
    const T ih = G.inv_h, i2h = G.inv_2h;
    const T c43 = T(4.0 / 3.0), c23 = T(2.0 / 3.0), half = T(0.5);
    // inviscid part: central differences of the nodal fluxes
    T r[4];
    {
        const T mxe = sq[1][e_], mxw = sq[1][w_], myn = sq[2][n_], mys = sq[2][s_];
        const T Fe1 = mxe * U[e_] + P[e_], Fw1 = mxw * U[w_] + P[w_];
        const T Fe2 = mxe * V[e_], Fw2 = mxw * V[w_];
        const T Fe3 = (sq[3][e_] + P[e_]) * U[e_], Fw3 = (sq[3][w_] + P[w_]) * U[w_];
        const T Gn1 = myn * U[n_], Gs1 = mys * U[s_];
        const T Gn2 = myn * V[n_] + P[n_], Gs2 = mys * V[s_] + P[s_];
        const T Gn3 = (sq[3][n_] + P[n_]) * V[n_], Gs3 = (sq[3][s_] + P[s_]) * V[s_];
        r[0] = -((mxe - mxw) + (myn - mys)) * i2h;
        r[1] = -((Fe1 - Fw1) + (Gn1 - Gs1)) * i2h;
        r[2] = -((Fe2 - Fw2) + (Gn2 - Gs2)) * i2h;
        r[3] = -((Fe3 - Fw3) + (Gn3 - Gs3)) * i2h;
    }
    // viscous and heat fluxes on the four faces of the node
    T fx[2][3], fy[2][3];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        {   // x-face between columns a = x-1+side and b = a+1
            const int a = side ? c : w_, b = side ? e_ : c;
            const T ux = (U[b] - U[a]) * ih, vx = (V[b] - V[a]) * ih;
            const T uy = half * ((U[a + HX] - U[a - HX]) + (U[b + HX] - U[b - HX])) * i2h;
            const T vy = half * ((V[a + HX] - V[a - HX]) + (V[b + HX] - V[b - HX])) * i2h;
            const T txx = mu * (c43 * ux - c23 * vy), txy = mu * (uy + vx);
            const T uf = half * (U[a] + U[b]), vf = half * (V[a] + V[b]);
            fx[side][0] = txx;
            fx[side][1] = txy;
            fx[side][2] = txx * uf + txy * vf + kap * (TT[b] - TT[a]) * ih;
        }
        {   // y-face between rows a = y-1+side and b = a+1
            const int a = side ? c : s_, b = side ? n_ : c;
            const T uy = (U[b] - U[a]) * ih, vy = (V[b] - V[a]) * ih;
            const T ux = half * ((U[a + 1] - U[a - 1]) + (U[b + 1] - U[b - 1])) * i2h;
            const T vx = half * ((V[a + 1] - V[a - 1]) + (V[b + 1] - V[b - 1])) * i2h;
            const T tyy = mu * (c43 * vy - c23 * ux), txy = mu * (uy + vx);
            const T uf = half * (U[a] + U[b]), vf = half * (V[a] + V[b]);
            fy[side][0] = txy;
            fy[side][1] = tyy;
            fy[side][2] = txy * uf + tyy * vf + kap * (TT[b] - TT[a]) * ih;
        }
    }
    T L[4];
    L[0] = r[0];
#pragma unroll
    for (int k = 1; k < 4; ++k)
        L[k] = r[k] + ((fx[1][k - 1] - fx[0][k - 1]) + (fy[1][k - 1] - fy[0][k - 1])) * ih;

    const size_t o = (size_t)y * n + x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T kq = G.dt * L[k];
        const T s = sq[k][c];
        T res;
        if (STAGE == 0) {
            res = s + kq;
        } else {
            const T base = u0[k * plane + o];
            res = fma(STAGE == 1 ? T(0.25) : T(2.0 / 3.0), (s - base) + kq, base);
        }
        out[k * plane + o] = res;
    }
}

// per-handle launch: two groups (members, fine run) passed by value, 32 x 8 tiles
template <typename T, int STAGE>
__global__ void __launch_bounds__(256) ns2d_stage_kernel(NsArgs<T> A) {
    int tile = blockIdx.x;
    const int gi = tile < A.tiles0 ? 0 : 1;
    if (gi) tile -= A.tiles0;
    const NsGroup<T> G = gi ? A.g[1] : A.g[0];  // no runtime index into the parameter array
    ns2d_stage_tile<T, STAGE, 32, 8>(G, tile, A.gm1, A.mu, A.kappa);
}

// batched launch: a table of groups in device memory, found by binary search
// on the first tile of each group
template <typename T, int STAGE, int TX, int TY>
__global__ void __launch_bounds__(256) ns2d_stage_table_kernel(const NsGroup<T> *__restrict__ groups,
                                                               int ngroups, T gm1, T mu, T kappa) {
    const int tile = blockIdx.x;
    int lo = 0, hi = ngroups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (groups[mid].tile_begin <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    const NsGroup<T> G = groups[lo];
    ns2d_stage_tile<T, STAGE, TX, TY>(G, tile - G.tile_begin, gm1, mu, kappa);
}

const char *ns2d_check_size(int n_whole, int n_split) {
    for (int n : {n_whole, n_split}) {
        if (n < 8 || n > 4096 || n % 8 != 0) return "NS-2D grids need 8 <= n <= 4096 points per side with n % 8 == 0";
    }
    return nullptr;
}

size_t ns2d_scratch_elems(int n_whole, int n_whole_probs, int n_split, int n_split_probs) {
    return 2 * 4 * ((size_t)n_whole * n_whole * n_whole_probs + (size_t)n_split * n_split * n_split_probs);
}

template <typename T>
cudaError_t ns2d_forecast_scratch(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                                  int n_split_probs, double length, double dt, double mu,
                                  double gamma, double prandtl, int nsteps, T *scratch,
                                  cudaStream_t stream) {
    NsArgs<T> A = {};
    const int ns[2] = {n_whole, n_split}, np[2] = {n_whole_probs, n_split_probs};
    T *st[2] = {whole, split};
    T *sc = scratch;
    int tiles[2] = {0, 0};
    for (int g = 0; g < 2; ++g) {
        NsGroup<T> &G = A.g[g];
        G.n = ns[g];
        G.nprob = np[g];
        G.u0 = st[g];
        const size_t sz = (size_t)4 * ns[g] * ns[g] * np[g];
        G.s1 = sc;
        G.s2 = sc + sz;
        sc += 2 * sz;
        if (np[g] > 0) {
            G.tx = ceil_div(ns[g], kNsTx);
            G.ty = ceil_div(ns[g], kNsTy);
            const double h = length / ns[g];
            G.inv_h = (T)(1.0 / h);
            G.inv_2h = (T)(1.0 / (2.0 * h));
            G.dt = (T)dt;
            tiles[g] = G.tx * G.ty * np[g];
        }
    }
    A.tiles0 = tiles[0];
    A.gm1 = (T)(gamma - 1.0);
    A.mu = (T)mu;
    A.kappa = (T)(mu * gamma / ((gamma - 1.0) * prandtl));
    const int grid = tiles[0] + tiles[1];
    if (grid == 0 || nsteps == 0) return cudaSuccess;
    for (int s = 0; s < nsteps; ++s) {
        ns2d_stage_kernel<T, 0><<<grid, 256, 0, stream>>>(A);
        ns2d_stage_kernel<T, 1><<<grid, 256, 0, stream>>>(A);
        ns2d_stage_kernel<T, 2><<<grid, 256, 0, stream>>>(A);
        count_launches(3);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t ns2d_forecast(T *whole, int n_whole, int n_whole_probs, T *split, int n_split,
                          int n_split_probs, double length, double dt, double mu, double gamma,
                          double prandtl, int nsteps, cudaStream_t stream) {
    // stream-ordered scratch for the stateless entry point
    const size_t elems = ns2d_scratch_elems(n_whole, n_whole_probs, n_split, n_split_probs);
    if (elems == 0 || nsteps == 0) return cudaSuccess;
    T *scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&scratch, elems * sizeof(T), stream);
    if (e != cudaSuccess) return e;
    e = ns2d_forecast_scratch<T>(whole, n_whole, n_whole_probs, split, n_split, n_split_probs, length, dt,
                                 mu, gamma, prandtl, nsteps, scratch, stream);
    cudaError_t e2 = cudaFreeAsync(scratch, stream);
    return e != cudaSuccess ? e : e2;
}

int ns2d_tile_x(int shape) { return shape == 1 ? 16 : (shape == 2 ? 64 : 32); }
int ns2d_tile_y(int shape) { return shape == 1 ? 16 : (shape == 2 ? 4 : 8); }

template <typename T, int TX, int TY>
static void launch_table(const NsGroup<T> *groups, int ngroups, int tiles, int nsteps, T gm1, T mu, T kappa,
                         cudaStream_t s) {
    for (int st = 0; st < nsteps; ++st) {
        ns2d_stage_table_kernel<T, 0, TX, TY><<<tiles, 256, 0, s>>>(groups, ngroups, gm1, mu, kappa);
        ns2d_stage_table_kernel<T, 1, TX, TY><<<tiles, 256, 0, s>>>(groups, ngroups, gm1, mu, kappa);
        ns2d_stage_table_kernel<T, 2, TX, TY><<<tiles, 256, 0, s>>>(groups, ngroups, gm1, mu, kappa);
        count_launches(3);
    }
}

template <typename T>
cudaError_t ns2d_forecast_table(const NsGroup<T> *d_groups, int ngroups, int tiles, int shape, int nsteps,
                                double gamma, double mu, double prandtl, cudaStream_t s) {
    if (tiles == 0 || nsteps == 0) return cudaSuccess;
    const T gm1 = (T)(gamma - 1.0), m = (T)mu, kap = (T)(mu * gamma / ((gamma - 1.0) * prandtl));
    if (shape == 1)
        launch_table<T, 16, 16>(d_groups, ngroups, tiles, nsteps, gm1, m, kap, s);
    else if (shape == 2)
        launch_table<T, 64, 4>(d_groups, ngroups, tiles, nsteps, gm1, m, kap, s);
    else
        launch_table<T, 32, 8>(d_groups, ngroups, tiles, nsteps, gm1, m, kap, s);
    return cudaGetLastError();
}

template <typename T, int TX, int TY>
static void launch_probe01(const NsGroup<T> *groups, int ngroups, int tiles, T gm1, T mu, T kappa, cudaStream_t s) {
    ns2d_stage_table_kernel<T, 0, TX, TY><<<tiles, 256, 0, s>>>(groups, ngroups, gm1, mu, kappa);
    ns2d_stage_table_kernel<T, 1, TX, TY><<<tiles, 256, 0, s>>>(groups, ngroups, gm1, mu, kappa);
    count_launches(2);
}

template <typename T>
cudaError_t ns2d_probe_stages01(const NsGroup<T> *d_groups, int ngroups, int tiles, int shape, double gamma,
                                double mu, double prandtl, cudaStream_t s) {
    if (tiles == 0) return cudaSuccess;
    const T gm1 = (T)(gamma - 1.0), m = (T)mu, kap = (T)(mu * gamma / ((gamma - 1.0) * prandtl));
    if (shape == 1)
        launch_probe01<T, 16, 16>(d_groups, ngroups, tiles, gm1, m, kap, s);
    else if (shape == 2)
        launch_probe01<T, 64, 4>(d_groups, ngroups, tiles, gm1, m, kap, s);
    else
        launch_probe01<T, 32, 8>(d_groups, ngroups, tiles, gm1, m, kap, s);
    return cudaGetLastError();
}

#define MGK_NS_INST(T)                                                                            \
    template cudaError_t ns2d_forecast<T>(T *, int, int, T *, int, int, double, double, double,    \
                                          double, double, int, cudaStream_t);                     \
    template cudaError_t ns2d_forecast_scratch<T>(T *, int, int, T *, int, int, double, double,    \
                                                  double, double, double, int, T *, cudaStream_t); \
    template cudaError_t ns2d_forecast_table<T>(const NsGroup<T> *, int, int, int, int, double, double, \
                                                double, cudaStream_t);                                 \
    template cudaError_t ns2d_probe_stages01<T>(const NsGroup<T> *, int, int, int, double, double, double, \
                                                cudaStream_t);
MGK_NS_INST(float)
MGK_NS_INST(double)
#undef MGK_NS_INST

}  // namespace mgk
