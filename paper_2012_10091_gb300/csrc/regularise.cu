// regularise.cu -- final fine-grid iteration (Algorithm 4 step 6) and the
// conservativity residual (Eq. Conservativity_rhov) of the fine run.
//
// The last model step of the observation interval is taken in implicit-Euler
// form, Psi(x) = x - dt L(x) = x_prev (x_prev: the fine state one step before
// the analysis time, recorded by the forecast).  Its residual is
//   Gamma = (x - x_prev) / dt - L(x),
// the paper's conservativity indicator, and the final iteration is one relaxed
// Jacobi (matrix-splitting) sweep from the analysis state (Sec. 3: a single
// iteration, alpha = 0.5):
//   x' = x + alpha D^-1 (x_prev + dt L(x) - x) = x - alpha dt D^-1 Gamma,
// with D the diagonal of dPsi/dx at x:
//   Burgers (central advective flux, no diagonal term): D = 1 + 2 nu dt / dx^2;
//   NS-2D: D = 1 (rho), 1 + dt (14/3) mu / (rho h^2) (rho u, rho v: 8/3 from the
//   compact normal derivative of tau_xx or tau_yy, 2 from tau_xy),
//   1 + dt 4 kappa (gamma - 1) / (rho h^2) (E, heat fluxes through T).
// The residual cancels to O(dt) of the state, so both kernels evaluate it in
// FP64 whatever the storage precision.  One thread per point; the sweep writes
// out of place (the caller copies the result back).
#include <cuda_runtime.h>

#include "analysis.h"
#include "common.cuh"

namespace mgk {

template <typename T>
__global__ void __launch_bounds__(256) k_burgers_residual(const T *__restrict__ x, const T *__restrict__ prev, int n,
                                                          double dx, double nu, double dt, double alpha,
                                                          T *__restrict__ out, double *__restrict__ gamma_out,
                                                          const int *status) {
    if (status && *status) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int im = i == 0 ? n - 1 : i - 1, ip = i == n - 1 ? 0 : i + 1;
    const double um = (double)x[im], u = (double)x[i], up = (double)x[ip];
    const double L = -(0.5 * up * up - 0.5 * um * um) / (2.0 * dx) + nu * (up - 2.0 * u + um) / (dx * dx);
    const double g = (u - (double)prev[i]) / dt - L;
    if (gamma_out) gamma_out[i] = g;
    if (out) {
        const double D = 1.0 + 2.0 * nu * dt / (dx * dx);
        out[i] = (T)(u + alpha * (-dt * g) / D);
    }
}

// conserved and primitive variables of one node, FP64
struct NsNode {
    double rho, mx, my, E, u, v, p, T;
};

template <typename T>
__device__ __forceinline__ NsNode ns_node(const T *q, int n, int x, int y, double gm1) {
    x = x < 0 ? x + n : (x >= n ? x - n : x);
    y = y < 0 ? y + n : (y >= n ? y - n : y);
    const size_t plane = (size_t)n * n, o = (size_t)y * n + x;
    NsNode a;
    a.rho = (double)q[o];
    a.mx = (double)q[plane + o];
    a.my = (double)q[2 * plane + o];
    a.E = (double)q[3 * plane + o];
    // one FP64 division per node (GB300 runs about 2 FP64 FMAs per clock per SM)
    const double ri = 1.0 / a.rho;
    a.u = a.mx * ri;
    a.v = a.my * ri;
    a.p = gm1 * (a.E - 0.5 * a.rho * (a.u * a.u + a.v * a.v));
    a.T = a.p * ri;
    return a;
}

constexpr int kResTile = 16;  // points per side of a CTA's tile (16 x 16 threads)

// Eqs. Mass, Momentum, Energy discretised as the forecast does it: central
// differences of the nodal inviscid fluxes, viscous and heat fluxes on the
// four faces (compact normal derivative, averaged central tangential one).
// A CTA derives the primitives of its 18 x 18 nodes (tile and halo) once, in
// shared memory, then every thread reads its 3 x 3 neighbourhood from there.
template <typename T>
__global__ void __launch_bounds__(256) k_ns2d_residual(const T *__restrict__ q, const T *__restrict__ prev, int n,
                                                       double h, double gamma, double mu, double prandtl,
                                                       double dt, double alpha, T *__restrict__ out,
                                                       double *__restrict__ gamma_out, const int *status) {
    constexpr int HW = kResTile + 2;
    __shared__ NsNode nodes[HW * HW];
    if (status && *status) return;  // set only by earlier launches: the same for the whole CTA
    const double gm1 = gamma - 1.0, kap = mu * gamma / (gm1 * prandtl);
    const double ih = 1.0 / h, i2h = 0.5 / h;
    const int x0 = blockIdx.x * kResTile, y0 = blockIdx.y * kResTile;
    for (int e = threadIdx.x; e < HW * HW; e += blockDim.x) {
        const int ly = e / HW, lx = e - ly * HW;
        nodes[e] = ns_node(q, n, x0 - 1 + lx, y0 - 1 + ly, gm1);
    }
    __syncthreads();
    const int tx = threadIdx.x % kResTile, ty = threadIdx.x / kResTile;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= n || y >= n) return;
    const size_t idx = (size_t)y * n + x;
    // nd(dy, dx): the node at offset (dx, dy) from this thread's point
    auto nd = [&](int dy, int dx) -> const NsNode & { return nodes[(ty + 1 + dy) * HW + tx + 1 + dx]; };
    const NsNode &C = nd(0, 0), &Ee = nd(0, 1), &Ww = nd(0, -1), &Nn = nd(1, 0), &Ss = nd(-1, 0);
    double L[4];
    L[0] = -((Ee.mx - Ww.mx) + (Nn.my - Ss.my)) * i2h;
    L[1] = -(((Ee.mx * Ee.u + Ee.p) - (Ww.mx * Ww.u + Ww.p)) + (Nn.my * Nn.u - Ss.my * Ss.u)) * i2h;
    L[2] = -((Ee.mx * Ee.v - Ww.mx * Ww.v) + ((Nn.my * Nn.v + Nn.p) - (Ss.my * Ss.v + Ss.p))) * i2h;
    L[3] = -(((Ee.E + Ee.p) * Ee.u - (Ww.E + Ww.p) * Ww.u) + ((Nn.E + Nn.p) * Nn.v - (Ss.E + Ss.p) * Ss.v)) * i2h;
    double fx[2][3], fy[2][3];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        {   // x-face between columns a = side - 1 and b = side (offsets from the node)
            const NsNode &a = nd(0, side - 1), &b = nd(0, side);
            const NsNode &an = nd(1, side - 1), &as = nd(-1, side - 1), &bn = nd(1, side), &bs = nd(-1, side);
            const double ux = (b.u - a.u) * ih, vx = (b.v - a.v) * ih;
            const double uy = 0.5 * ((an.u - as.u) + (bn.u - bs.u)) * i2h;
            const double vy = 0.5 * ((an.v - as.v) + (bn.v - bs.v)) * i2h;
            const double txx = mu * (4.0 / 3.0 * ux - 2.0 / 3.0 * vy), txy = mu * (uy + vx);
            const double uf = 0.5 * (a.u + b.u), vf = 0.5 * (a.v + b.v);
            fx[side][0] = txx;
            fx[side][1] = txy;
            fx[side][2] = txx * uf + txy * vf + kap * (b.T - a.T) * ih;
        }
        {   // y-face between rows a = side - 1 and b = side
            const NsNode &a = nd(side - 1, 0), &b = nd(side, 0);
            const NsNode &ae = nd(side - 1, 1), &aw = nd(side - 1, -1), &be = nd(side, 1), &bw = nd(side, -1);
            const double uy = (b.u - a.u) * ih, vy = (b.v - a.v) * ih;
            const double ux = 0.5 * ((ae.u - aw.u) + (be.u - bw.u)) * i2h;
            const double vx = 0.5 * ((ae.v - aw.v) + (be.v - bw.v)) * i2h;
            const double tyy = mu * (4.0 / 3.0 * vy - 2.0 / 3.0 * ux), txy = mu * (uy + vx);
            const double uf = 0.5 * (a.u + b.u), vf = 0.5 * (a.v + b.v);
            fy[side][0] = txy;
            fy[side][1] = tyy;
            fy[side][2] = txy * uf + tyy * vf + kap * (b.T - a.T) * ih;
        }
    }
#pragma unroll
    for (int k = 1; k < 4; ++k) L[k] += ((fx[1][k - 1] - fx[0][k - 1]) + (fy[1][k - 1] - fy[0][k - 1])) * ih;
    const size_t plane = (size_t)n * n;
    const double qc[4] = {C.rho, C.mx, C.my, C.E};
    const double rh2 = C.rho * h * h;
    const double D[4] = {1.0, 1.0 + dt * (14.0 / 3.0) * mu / rh2, 1.0 + dt * (14.0 / 3.0) * mu / rh2,
                         1.0 + dt * 4.0 * kap * gm1 / rh2};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double g = (qc[k] - (double)prev[k * plane + idx]) / dt - L[k];
        if (gamma_out) gamma_out[k * plane + idx] = g;
        if (out) out[k * plane + idx] = (T)(qc[k] + alpha * (-dt * g) / D[k]);
    }
}

// (x - x_prev) / dt in FP64: the time-derivative term of Eq. Conservativity_rhov,
// whose largest magnitude over the grid normalises Gamma (the paper's Gamma*)
template <typename T>
__global__ void k_state_rate(const T *__restrict__ x, const T *__restrict__ prev, size_t count, double inv_dt,
                             double *__restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = ((double)x[i] - (double)prev[i]) * inv_dt;
}

template <typename T>
void launch_state_rate(const T *x, const T *prev, size_t count, double dt, double *out, cudaStream_t s) {
    count_launches(1);
    k_state_rate<T><<<ceil_div((long long)count, 256) < 4096 ? ceil_div((long long)count, 256) : 4096, 256, 0, s>>>(
        x, prev, count, 1.0 / dt, out);
}
template void launch_state_rate<float>(const float *, const float *, size_t, double, double *, cudaStream_t);
template void launch_state_rate<double>(const double *, const double *, size_t, double, double *, cudaStream_t);

// Gamma* = Gamma / C per variable (Sec. 6, the normalisation of the
// conservativity maps): C = max over the plane's points of |x - x_prev| / dt,
// one CTA per variable; a plane that did not change keeps Gamma.
template <typename T>
__global__ void __launch_bounds__(1024) k_gamma_norm(const T *__restrict__ x, const T *__restrict__ prev,
                                                     size_t plane, double inv_dt, double *__restrict__ g) {
    __shared__ double wmax[32];
    const size_t off = (size_t)blockIdx.x * plane;
    double m = 0.0;
    for (size_t i = threadIdx.x; i < plane; i += blockDim.x)
        m = fmax(m, fabs(((double)x[off + i] - (double)prev[off + i]) * inv_dt));
    for (int d = 16; d > 0; d >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, d));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.0;
        for (int d = 16; d > 0; d >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, d));
        if (threadIdx.x == 0) wmax[0] = m;
    }
    __syncthreads();
    const double c = wmax[0] > 0.0 ? wmax[0] : 1.0;
    for (size_t i = threadIdx.x; i < plane; i += blockDim.x) g[off + i] = g[off + i] / c;
}

template <typename T>
void launch_gamma_norm(const T *x, const T *prev, int V, size_t plane, double dt, double *gamma, cudaStream_t s) {
    count_launches(1);
    k_gamma_norm<T><<<V, 1024, 0, s>>>(x, prev, plane, 1.0 / dt, gamma);
}
template void launch_gamma_norm<float>(const float *, const float *, int, size_t, double, double *, cudaStream_t);
template void launch_gamma_norm<double>(const double *, const double *, int, size_t, double, double *, cudaStream_t);

template <typename T>
void launch_fine_residual(int model, const T *x, const T *prev, int n, double length, double nu, double gamma,
                          double prandtl, double dt, double alpha, T *out, double *gamma_out, const int *status,
                          cudaStream_t s) {
    count_launches(1);
    const double h = length / n;
    if (model == 1) {
        k_burgers_residual<T><<<ceil_div(n, 256), 256, 0, s>>>(x, prev, n, h, nu, dt, alpha, out, gamma_out, status);
    } else {
        const dim3 grid(ceil_div(n, kResTile), ceil_div(n, kResTile));
        k_ns2d_residual<T><<<grid, 256, 0, s>>>(x, prev, n, h, gamma, nu, prandtl, dt, alpha, out, gamma_out,
                                                status);
    }
}

template void launch_fine_residual<float>(int, const float *, const float *, int, double, double, double, double,
                                          double, double, float *, double *, const int *, cudaStream_t);
template void launch_fine_residual<double>(int, const double *, const double *, int, double, double, double, double,
                                           double, double, double *, double *, const int *, cudaStream_t);

}  // namespace mgk
