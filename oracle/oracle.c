/*
 * oracle.c -- plain FP64 CPU oracle of the MGEnKF analysis cycle.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library; the GPU library
 * shares no code with it.  Slow and literal on purpose: each routine states
 * the passage of the paper it follows, and uses no blocking, fusion or
 * reordering beyond that passage.  The only parallelism is an OpenMP loop over
 * independent grids (ensemble members), which changes no arithmetic.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP loops below.  Every parallel loop runs over
 * independent problems or members, so no result depends on the count; it is
 * set only to time the oracle on one core and on all of them. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ======================================================================== */
/* Philox4x64-10, from the published definition (Salmon et al., SC'11):      */
/* round: (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),                   */
/*                          hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),                  */
/* key schedule k += (W0, W1) between rounds.  Parity: pinned.               */
/* ======================================================================== */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1 */

static void mul_hilo(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mul_hilo(PHILOX_M0, c0, &hi0, &lo0);
        mul_hilo(PHILOX_M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Box-Muller (1958): z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = ... sin(2 pi u2). */
void orc_normals(uint64_t seed, uint64_t tag, uint64_t ctr0, int64_t count, double *z) {
    const double two_pi = 6.283185307179586;
    const double inv53 = 1.0 / 9007199254740992.0; /* 2^-53 */
    uint64_t key[2] = {seed, tag};
    for (int64_t blk = 0; blk * 4 < count; ++blk) {
        uint64_t ctr[4] = {ctr0, (uint64_t)blk, 0, 0};
        uint64_t x[4];
        orc_philox4x64_10(ctr, key, x);
        double zz[4];
        for (int pair = 0; pair < 2; ++pair) {
            double u1 = (double)((x[2 * pair] >> 11) + 1) * inv53;
            double u2 = (double)((x[2 * pair + 1] >> 11) + 1) * inv53;
            double rad = sqrt(-2.0 * log(u1));
            double th = two_pi * u2;
            zz[2 * pair] = rad * cos(th);
            zz[2 * pair + 1] = rad * sin(th);
        }
        for (int l = 0; l < 4; ++l)
            if (blk * 4 + l < count) z[blk * 4 + l] = zz[l];
    }
}

/* ======================================================================== */
/* Viscous Burgers, Eq. burgers, periodic grid x_j = j dx.                   */
/* Parity: pinned (Fourier amplification factor of the linear flux, Cole-    */
/* Hopf convergence and mass conservation of the nonlinear flux).            */
/* ======================================================================== */
void orc_burgers_rhs(const double *u, int n, double dx, double nu, int flux_kind, double c,
                     double *L) {
    for (int j = 0; j < n; ++j) {
        int jm = (j - 1 + n) % n, jp = (j + 1) % n;
        double Fm, Fp;
        if (flux_kind == 0) {
            Fm = 0.5 * u[jm] * u[jm];
            Fp = 0.5 * u[jp] * u[jp];
        } else {
            Fm = c * u[jm];
            Fp = c * u[jp];
        }
        double adv = -(Fp - Fm) / (2.0 * dx);
        double dif = nu * (u[jp] - 2.0 * u[j] + u[jm]) / (dx * dx);
        L[j] = adv + dif;
    }
}

/* Burgers with an inlet (Sec. 4, Eq. burgers with Eq. inlet-1D-Burgers): nodes
 * x_j = j dx, j = 0..n-1; node 0 holds the Dirichlet inlet value
 * u(0, t) = u0 (1 + theta1 sin(omega t + theta2)), the outlet node n-1 is
 * extrapolated linearly from its two neighbours, the interior nodes follow the
 * flux-form central scheme of orc_burgers_rhs (without wrap-around).  SSP-RK3
 * in Shu-Osher form with the inlet set at each stage's time (t + dt, t + dt/2,
 * t + dt).  theta: nprob x 2 (theta1, theta2), one pair per problem. */
static void inlet_bc(double *u, int n, double t, double u0, double omega, const double *th) {
    u[0] = u0 * (1.0 + th[0] * sin(omega * t + th[1]));
    u[n - 1] = 2.0 * u[n - 2] - u[n - 3];
}

static void inlet_rhs(const double *u, int n, double dx, double nu, double *L) {
    for (int j = 1; j < n - 1; ++j) {
        const double fp = 0.5 * u[j + 1] * u[j + 1], fm = 0.5 * u[j - 1] * u[j - 1];
        L[j] = -(fp - fm) / (2.0 * dx) + nu * (u[j + 1] - 2.0 * u[j] + u[j - 1]) / (dx * dx);
    }
    L[0] = L[n - 1] = 0.0;
}

void orc_burgers_inlet_rk3(double *u, int nprob, int n, double dx, double nu, double dt, int nsteps,
                           double t0, const double *theta, double u0, double omega) {
#pragma omp parallel for schedule(static)
    for (int p = 0; p < nprob; ++p) {
        double *x = u + (size_t)p * n;
        const double *th = theta + 2 * (size_t)p;
        double *u1 = malloc(sizeof(double) * n), *u2 = malloc(sizeof(double) * n), *L = malloc(sizeof(double) * n);
        for (int s = 0; s < nsteps; ++s) {
            const double t = t0 + s * dt;
            inlet_rhs(x, n, dx, nu, L);
            for (int j = 0; j < n; ++j) u1[j] = x[j] + dt * L[j];
            inlet_bc(u1, n, t + dt, u0, omega, th);
            inlet_rhs(u1, n, dx, nu, L);
            for (int j = 0; j < n; ++j) u2[j] = 0.75 * x[j] + 0.25 * (u1[j] + dt * L[j]);
            inlet_bc(u2, n, t + 0.5 * dt, u0, omega, th);
            inlet_rhs(u2, n, dx, nu, L);
            for (int j = 0; j < n; ++j) x[j] = x[j] / 3.0 + 2.0 / 3.0 * (u2[j] + dt * L[j]);
            inlet_bc(x, n, t + dt, u0, omega, th);
        }
        free(u1);
        free(u2);
        free(L);
    }
}

/* SSP-RK3 in Shu-Osher form:
 *   u1 = u + dt L(u);  u2 = 3/4 u + 1/4 (u1 + dt L(u1));
 *   u_new = 1/3 u + 2/3 (u2 + dt L(u2)). */
void orc_burgers_rk3(double *u, int nprob, int n, double dx, double nu, double dt, int nsteps,
                     int flux_kind, double c) {
#pragma omp parallel for schedule(static)
    for (int p = 0; p < nprob; ++p) {
        double *x = u + (size_t)p * n;
        double *u1 = malloc(sizeof(double) * n);
        double *u2 = malloc(sizeof(double) * n);
        double *L = malloc(sizeof(double) * n);
        for (int s = 0; s < nsteps; ++s) {
            orc_burgers_rhs(x, n, dx, nu, flux_kind, c, L);
            for (int j = 0; j < n; ++j) u1[j] = x[j] + dt * L[j];
            orc_burgers_rhs(u1, n, dx, nu, flux_kind, c, L);
            for (int j = 0; j < n; ++j) u2[j] = 0.75 * x[j] + 0.25 * (u1[j] + dt * L[j]);
            orc_burgers_rhs(u2, n, dx, nu, flux_kind, c, L);
            for (int j = 0; j < n; ++j) x[j] = x[j] / 3.0 + 2.0 / 3.0 * (u2[j] + dt * L[j]);
        }
        free(u1);
        free(u2);
        free(L);
    }
}

/* ======================================================================== */
/* Compressible NS, Eqs. Mass, Momentum, Energy (Sec. 6), periodic square.   */
/* Parity: pinned (conservation of the four totals, uniform-state and        */
/* x<->y symmetry invariants, linear acoustic/shear mode decay, the 4 x 4    */
/* discrete symbol of the operator linearised about rest, which fixes the    */
/* 4/3 and -2/3 stress factors, the cross terms and kappa; exact states that */
/* fix the heat flux kappa lap T and the viscous work tau . u).              */
/* ======================================================================== */
#define IDX(y, x) ((size_t)(((y) + n) % n) * n + (size_t)(((x) + n) % n))

void orc_ns2d_rhs(const double *q, int n, double h, double gamma, double mu, double prandtl,
                  double *L) {
    size_t N2 = (size_t)n * n;
    const double *rho = q, *mx = q + N2, *my = q + 2 * N2, *E = q + 3 * N2;
    double *u = malloc(sizeof(double) * N2), *v = malloc(sizeof(double) * N2);
    double *p = malloc(sizeof(double) * N2), *T = malloc(sizeof(double) * N2);
    for (size_t k = 0; k < N2; ++k) {
        u[k] = mx[k] / rho[k];
        v[k] = my[k] / rho[k];
        p[k] = (gamma - 1.0) * (E[k] - 0.5 * rho[k] * (u[k] * u[k] + v[k] * v[k]));
        T[k] = p[k] / rho[k];
    }
    double kappa = mu * gamma / ((gamma - 1.0) * prandtl);
    for (int y = 0; y < n; ++y) {
        for (int x = 0; x < n; ++x) {
            size_t c = IDX(y, x), e = IDX(y, x + 1), w = IDX(y, x - 1);
            size_t nn = IDX(y + 1, x), s = IDX(y - 1, x);
            /* inviscid: nodal fluxes F (x) and G (y), central differences */
            double Fe[4] = {mx[e], mx[e] * u[e] + p[e], mx[e] * v[e], (E[e] + p[e]) * u[e]};
            double Fw[4] = {mx[w], mx[w] * u[w] + p[w], mx[w] * v[w], (E[w] + p[w]) * u[w]};
            double Gn[4] = {my[nn], my[nn] * u[nn], my[nn] * v[nn] + p[nn], (E[nn] + p[nn]) * v[nn]};
            double Gs[4] = {my[s], my[s] * u[s], my[s] * v[s] + p[s], (E[s] + p[s]) * v[s]};
            double r[4];
            for (int k = 0; k < 4; ++k) r[k] = -(Fe[k] - Fw[k]) / (2.0 * h) - (Gn[k] - Gs[k]) / (2.0 * h);
            /* viscous + heat fluxes at the four faces of node (y, x) */
            double Fv[2][4], Gv[2][4];
            for (int side = 0; side < 2; ++side) {
                /* x-face between columns xa = x-1+side and xb = xa+1 */
                int xa = x - 1 + side, xb = xa + 1;
                size_t a = IDX(y, xa), b = IDX(y, xb);
                double ux = (u[b] - u[a]) / h, vx = (v[b] - v[a]) / h;
                double uy = 0.5 * ((u[IDX(y + 1, xa)] - u[IDX(y - 1, xa)]) +
                                   (u[IDX(y + 1, xb)] - u[IDX(y - 1, xb)])) / (2.0 * h);
                double vy = 0.5 * ((v[IDX(y + 1, xa)] - v[IDX(y - 1, xa)]) +
                                   (v[IDX(y + 1, xb)] - v[IDX(y - 1, xb)])) / (2.0 * h);
                double txx = mu * (4.0 / 3.0 * ux - 2.0 / 3.0 * vy);
                double txy = mu * (uy + vx);
                double uf = 0.5 * (u[a] + u[b]), vf = 0.5 * (v[a] + v[b]);
                double Tx = (T[b] - T[a]) / h;
                Fv[side][0] = 0.0;
                Fv[side][1] = txx;
                Fv[side][2] = txy;
                Fv[side][3] = txx * uf + txy * vf + kappa * Tx;
                /* y-face between rows ya = y-1+side and yb = ya+1 */
                int ya = y - 1 + side, yb = ya + 1;
                a = IDX(ya, x);
                b = IDX(yb, x);
                double uy2 = (u[b] - u[a]) / h, vy2 = (v[b] - v[a]) / h;
                double ux2 = 0.5 * ((u[IDX(ya, x + 1)] - u[IDX(ya, x - 1)]) +
                                    (u[IDX(yb, x + 1)] - u[IDX(yb, x - 1)])) / (2.0 * h);
                double vx2 = 0.5 * ((v[IDX(ya, x + 1)] - v[IDX(ya, x - 1)]) +
                                    (v[IDX(yb, x + 1)] - v[IDX(yb, x - 1)])) / (2.0 * h);
                double tyy = mu * (4.0 / 3.0 * vy2 - 2.0 / 3.0 * ux2);
                double txy2 = mu * (uy2 + vx2);
                double uf2 = 0.5 * (u[a] + u[b]), vf2 = 0.5 * (v[a] + v[b]);
                double Ty = (T[b] - T[a]) / h;
                Gv[side][0] = 0.0;
                Gv[side][1] = txy2;
                Gv[side][2] = tyy;
                Gv[side][3] = txy2 * uf2 + tyy * vf2 + kappa * Ty;
            }
            for (int k = 0; k < 4; ++k)
                L[k * N2 + c] = r[k] + (Fv[1][k] - Fv[0][k]) / h + (Gv[1][k] - Gv[0][k]) / h;
        }
    }
    free(u);
    free(v);
    free(p);
    free(T);
}

/* Centred sixth-order explicit filter of the Euler and Navier-Stokes models
 * (Secs. 5 and 6; the paper cites Bogey and Bailly 2004 and prints no
 * coefficients).  Reading: the standard 7-point centred stencil
 *   u_j <- u_j - sigma/64 (-u_{j-3} + 6 u_{j-2} - 15 u_{j-1} + 20 u_j
 *                          - 15 u_{j+1} + 6 u_{j+2} - u_{j+3}),
 * whose transfer function is 1 - sigma sin^6(k h / 2) (exact on Fourier modes,
 * zero-sum stencil: totals conserved), applied along x and then along y to
 * each of the four conserved planes of an n x n periodic grid. */
void orc_ns2d_filter6(double *q, int nprob, int n, double sigma) {
    static const double d[7] = {-1.0, 6.0, -15.0, 20.0, -15.0, 6.0, -1.0};
    const size_t plane = (size_t)n * n;
    double *line = malloc(sizeof(double) * (size_t)n);
    for (size_t pl = 0; pl < (size_t)nprob * 4; ++pl) {
        double *u = q + pl * plane;
        for (int y = 0; y < n; ++y) {          /* along x */
            for (int x = 0; x < n; ++x) line[x] = u[(size_t)y * n + x];
            for (int x = 0; x < n; ++x) {
                double D = 0.0;
                for (int m = -3; m <= 3; ++m) D += d[m + 3] * line[((x + m) % n + n) % n];
                u[(size_t)y * n + x] = line[x] - sigma / 64.0 * D;
            }
        }
        for (int x = 0; x < n; ++x) {          /* along y */
            for (int y = 0; y < n; ++y) line[y] = u[(size_t)y * n + x];
            for (int y = 0; y < n; ++y) {
                double D = 0.0;
                for (int m = -3; m <= 3; ++m) D += d[m + 3] * line[((y + m) % n + n) % n];
                u[(size_t)y * n + x] = line[y] - sigma / 64.0 * D;
            }
        }
    }
    free(line);
}

void orc_ns2d_rk3(double *q, int nprob, int n, double h, double gamma, double mu,
                  double prandtl, double dt, int nsteps) {
    size_t sz = (size_t)4 * n * n;
#pragma omp parallel for schedule(static)
    for (int pb = 0; pb < nprob; ++pb) {
        double *x = q + (size_t)pb * sz;
        double *u1 = malloc(sizeof(double) * sz);
        double *u2 = malloc(sizeof(double) * sz);
        double *L = malloc(sizeof(double) * sz);
        for (int s = 0; s < nsteps; ++s) {
            orc_ns2d_rhs(x, n, h, gamma, mu, prandtl, L);
            for (size_t j = 0; j < sz; ++j) u1[j] = x[j] + dt * L[j];
            orc_ns2d_rhs(u1, n, h, gamma, mu, prandtl, L);
            for (size_t j = 0; j < sz; ++j) u2[j] = 0.75 * x[j] + 0.25 * (u1[j] + dt * L[j]);
            orc_ns2d_rhs(u2, n, h, gamma, mu, prandtl, L);
            for (size_t j = 0; j < sz; ++j) x[j] = x[j] / 3.0 + 2.0 / 3.0 * (u2[j] + dt * L[j]);
        }
        free(u1);
        free(u2);
        free(L);
    }
}
#undef IDX

/* ======================================================================== */
/* Projectors Pi_C and Pi_F: 4th-order Lagrange interpolation (Sec. 2.2).     */
/* Parity: pinned (Pi_C Pi_F = I, exactness on cubics, O(h^4) error).        */
/* ======================================================================== */
void orc_lagrange_weights(int npts, const double *nodes, double s, double *w) {
    for (int k = 0; k < npts; ++k) {
        double num = 1.0, den = 1.0;
        for (int m = 0; m < npts; ++m) {
            if (m == k) continue;
            num *= (s - nodes[m]);
            den *= (nodes[k] - nodes[m]);
        }
        w[k] = num / den;
    }
}

static const double LAG_NODES[4] = {-1.0, 0.0, 1.0, 2.0};

/* interpolate coarse plane xc (nc^dim) at fine node (fy, fx) (fy = 0 in 1-D) */
static double interp_at(const double *xc, int dim, int nc, int r, int fy, int fx) {
    double wx[4], wy[4] = {0.0, 1.0, 0.0, 0.0};
    int Jx = fx / r, Jy = fy / r;
    orc_lagrange_weights(4, LAG_NODES, (double)(fx % r) / r, wx);
    if (dim == 2) orc_lagrange_weights(4, LAG_NODES, (double)(fy % r) / r, wy);
    double acc = 0.0;
    if (dim == 1) {
        for (int t = 0; t < 4; ++t) acc += wx[t] * xc[(Jx - 1 + t + nc) % nc];
        return acc;
    }
    for (int ty = 0; ty < 4; ++ty) {
        int yy = (Jy - 1 + ty + nc) % nc;
        for (int tx = 0; tx < 4; ++tx) {
            int xx = (Jx - 1 + tx + nc) % nc;
            acc += wy[ty] * wx[tx] * xc[(size_t)yy * nc + xx];
        }
    }
    return acc;
}

void orc_restrict(const double *fine, int dim, int V, int nc, int r, double *coarse) {
    int nf = nc * r;
    size_t cpl = dim == 1 ? (size_t)nc : (size_t)nc * nc;
    size_t fpl = dim == 1 ? (size_t)nf : (size_t)nf * nf;
    for (int v = 0; v < V; ++v) {
        if (dim == 1) {
            for (int J = 0; J < nc; ++J) coarse[v * cpl + J] = fine[v * fpl + (size_t)r * J];
        } else {
            for (int Jy = 0; Jy < nc; ++Jy)
                for (int Jx = 0; Jx < nc; ++Jx)
                    coarse[v * cpl + (size_t)Jy * nc + Jx] =
                        fine[v * fpl + (size_t)(r * Jy) * nf + (size_t)r * Jx];
        }
    }
}

void orc_prolong_add(const double *dc, int dim, int V, int nc, int r, double *fine) {
    int nf = nc * r;
    size_t cpl = dim == 1 ? (size_t)nc : (size_t)nc * nc;
    size_t fpl = dim == 1 ? (size_t)nf : (size_t)nf * nf;
    for (int v = 0; v < V; ++v) {
        if (dim == 1) {
            for (int f = 0; f < nf; ++f) fine[v * fpl + f] += interp_at(dc + v * cpl, 1, nc, r, 0, f);
        } else {
            for (int fy = 0; fy < nf; ++fy)
                for (int fx = 0; fx < nf; ++fx)
                    fine[v * fpl + (size_t)fy * nf + fx] += interp_at(dc + v * cpl, 2, nc, r, fy, fx);
        }
    }
}

void orc_obs_coarse(const double *xc, int dim, int V, int nc, int r, int ny,
                    const int32_t *obs_idx, const int32_t *obs_var, double *y) {
    int nf = nc * r;
    size_t cpl = dim == 1 ? (size_t)nc : (size_t)nc * nc;
    (void)V;
    for (int j = 0; j < ny; ++j) {
        int fy = dim == 1 ? 0 : obs_idx[j] / nf;
        int fx = dim == 1 ? obs_idx[j] : obs_idx[j] % nf;
        y[j] = interp_at(xc + (size_t)obs_var[j] * cpl, dim, nc, r, fy, fx);
    }
}

/* ======================================================================== */
/* Cholesky-Banachiewicz and the two triangular solves.                      */
/* ======================================================================== */
int orc_cholesky(double *A, int n) {
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            if (i == j) {
                if (!(s > 0.0) || !isfinite(s)) return i + 1;
                A[(size_t)i * n + i] = sqrt(s);
            } else {
                A[(size_t)i * n + j] = s / A[(size_t)j * n + j];
            }
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) A[(size_t)i * n + j] = 0.0;
    return 0;
}

/* b: nrhs right-hand sides, each contiguous (b[col * n + row]); overwritten
 * by the solution of L L^T x = b. */
void orc_chol_solve(const double *Lf, int n, double *b, int nrhs) {
    for (int c = 0; c < nrhs; ++c) {
        double *x = b + (size_t)c * n;
        for (int i = 0; i < n; ++i) {
            double s = x[i];
            for (int k = 0; k < i; ++k) s -= Lf[(size_t)i * n + k] * x[k];
            x[i] = s / Lf[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = x[i];
            for (int k = i + 1; k < n; ++k) s -= Lf[(size_t)k * n + i] * x[k];
            x[i] = s / Lf[(size_t)i * n + i];
        }
    }
}

/* ======================================================================== */
/* EnKF gain, Sec. 2.1.2 and Algorithm 1 step 6:                              */
/*   K = X Y^T (Y Y^T + R)^-1, X: nx x ne, Y: ny x ne (row-major), R: ny x ny */
/* computed as K = X M^T with M = (Y Y^T + R)^-1 Y.                           */
/* ======================================================================== */
int orc_enkf_gain(int nx, int ne, int ny, const double *X, const double *Y, const double *Rm,
                  double *K) {
    double *C = malloc(sizeof(double) * (size_t)ny * ny);
    for (int a = 0; a < ny; ++a)
        for (int b = 0; b < ny; ++b) {
            double s = 0.0;
            for (int i = 0; i < ne; ++i) s += Y[(size_t)a * ne + i] * Y[(size_t)b * ne + i];
            C[(size_t)a * ny + b] = s + Rm[(size_t)a * ny + b];
        }
    if (orc_cholesky(C, ny) != 0) {
        free(C);
        return 1;
    }
    /* M stored as ne columns of length ny: Mcol[i*ny + j] = M[j][i] */
    double *Mcol = malloc(sizeof(double) * (size_t)ny * ne);
    for (int i = 0; i < ne; ++i)
        for (int j = 0; j < ny; ++j) Mcol[(size_t)i * ny + j] = Y[(size_t)j * ne + i];
    orc_chol_solve(C, ny, Mcol, ne);
    for (int p = 0; p < nx; ++p)
        for (int j = 0; j < ny; ++j) {
            double s = 0.0;
            for (int i = 0; i < ne; ++i) s += X[(size_t)p * ne + i] * Mcol[(size_t)i * ny + j];
            K[(size_t)p * ny + j] = s;
        }
    free(C);
    free(Mcol);
    return 0;
}

/* ======================================================================== */
/* Coarse-mesh analysis (Algorithm 3, state part) and the coarse correction  */
/* of the fine run (Algorithm 4 step 5, first line).                          */
/* Parity: pinned (brute-force gain at n <= 16, KF limit, limits, r = 1).    */
/* ======================================================================== */
int orc_enkf_analyse(int dim, int V, int nc, int r, int ne, int ny, const int32_t *obs_idx,
                     const int32_t *obs_var, const double *yo, const double *eps, double sigma,
                     int gain_form, double *members, const double *xstar, double *dC) {
    size_t nx = (size_t)V * (dim == 1 ? (size_t)nc : (size_t)nc * nc);
    double sq = sqrt((double)(ne - 1));
    /* Algorithm 3 step 2: model counterparts y^f,(i) = H^C(x^f,(i)); and H^C(x*) */
    double *yf = malloc(sizeof(double) * (size_t)ne * ny);
    double *hstar = malloc(sizeof(double) * ny);
    for (int i = 0; i < ne; ++i)
        orc_obs_coarse(members + (size_t)i * nx, dim, V, nc, r, ny, obs_idx, obs_var, yf + (size_t)i * ny);
    orc_obs_coarse(xstar, dim, V, nc, r, ny, obs_idx, obs_var, hstar);
    /* Algorithm 1 step 4: ensemble means of x^f, y^f and eps */
    double *xbar = calloc(nx, sizeof(double));
    double *ybar = calloc(ny, sizeof(double));
    double *ebar = calloc(ny, sizeof(double));
    for (int i = 0; i < ne; ++i) {
        for (size_t p = 0; p < nx; ++p) xbar[p] += members[(size_t)i * nx + p];
        for (int j = 0; j < ny; ++j) {
            ybar[j] += yf[(size_t)i * ny + j];
            ebar[j] += eps[(size_t)i * ny + j];
        }
    }
    for (size_t p = 0; p < nx; ++p) xbar[p] /= ne;
    for (int j = 0; j < ny; ++j) {
        ybar[j] /= ne;
        ebar[j] /= ne;
    }
    /* Algorithm 3 step 7: normalised anomalies X (nx x ne), Y, E (ny x ne) */
    double *X = malloc(sizeof(double) * nx * ne);
    double *Y = malloc(sizeof(double) * (size_t)ny * ne);
    double *Eo = malloc(sizeof(double) * (size_t)ny * ne);
    for (int i = 0; i < ne; ++i) {
        for (size_t p = 0; p < nx; ++p) X[p * ne + i] = (members[(size_t)i * nx + p] - xbar[p]) / sq;
        for (int j = 0; j < ny; ++j) {
            Y[(size_t)j * ne + i] = (yf[(size_t)i * ny + j] - ybar[j]) / sq;
            Eo[(size_t)j * ne + i] = (eps[(size_t)i * ny + j] - ebar[j]) / sq;
        }
    }
    int status = 0;
    if (gain_form == 1) {
        /* Ensemble-space form of the same gain (push-through identity):
         * Y^T (Y Y^T + R)^-1 = (I + Y^T R^-1 Y)^-1 Y^T R^-1,  R = sigma^2 I. */
        double s2 = sigma * sigma;
        double *S = malloc(sizeof(double) * (size_t)ne * ne);
        double *B = malloc(sizeof(double) * (size_t)(ne + 1) * ne); /* column c contiguous */
        for (int a = 0; a < ne; ++a)
            for (int b = 0; b < ne; ++b) {
                double s = 0.0;
                for (int j = 0; j < ny; ++j) s += Y[(size_t)j * ne + a] * Y[(size_t)j * ne + b];
                S[(size_t)a * ne + b] = (a == b ? 1.0 : 0.0) + s / s2;
            }
        for (int c = 0; c <= ne; ++c)
            for (int a = 0; a < ne; ++a) {
                double s = 0.0;
                for (int j = 0; j < ny; ++j) {
                    double d = c < ne ? yo[j] + eps[(size_t)c * ny + j] - yf[(size_t)c * ny + j]
                                      : yo[j] - hstar[j];
                    s += Y[(size_t)j * ne + a] * d;
                }
                B[(size_t)c * ne + a] = s / s2;
            }
        if (orc_cholesky(S, ne) != 0) {
            status = 1;
        } else {
            orc_chol_solve(S, ne, B, ne + 1); /* B <- T, column c = T[:, c] */
            for (int c = 0; c < ne; ++c)
                for (size_t p = 0; p < nx; ++p) {
                    double s = 0.0;
                    for (int a = 0; a < ne; ++a) s += X[p * ne + a] * B[(size_t)c * ne + a];
                    members[(size_t)c * nx + p] += s;
                }
            for (size_t p = 0; p < nx; ++p) {
                double s = 0.0;
                for (int a = 0; a < ne; ++a) s += X[p * ne + a] * B[(size_t)ne * ne + a];
                dC[p] = s;
            }
        }
        free(S);
        free(B);
    } else {
        /* Literal gain (Algorithm 3 step 8) with R = sigma^2 I or R^e = E E^T */
        double *Rm = calloc((size_t)ny * ny, sizeof(double));
        if (gain_form == 2) {
            for (int a = 0; a < ny; ++a)
                for (int b = 0; b < ny; ++b) {
                    double s = 0.0;
                    for (int i = 0; i < ne; ++i) s += Eo[(size_t)a * ne + i] * Eo[(size_t)b * ne + i];
                    Rm[(size_t)a * ny + b] = s;
                }
        } else {
            for (int a = 0; a < ny; ++a) Rm[(size_t)a * ny + a] = sigma * sigma;
        }
        double *K = malloc(sizeof(double) * nx * ny);
        if (orc_enkf_gain((int)nx, ne, ny, X, Y, Rm, K) != 0) {
            status = 1;
        } else {
            /* x^a,(i) = x^f,(i) + K (y^o + eps^(i) - y^f,(i)) */
            for (int i = 0; i < ne; ++i)
                for (size_t p = 0; p < nx; ++p) {
                    double s = 0.0;
                    for (int j = 0; j < ny; ++j)
                        s += K[p * ny + j] * (yo[j] + eps[(size_t)i * ny + j] - yf[(size_t)i * ny + j]);
                    members[(size_t)i * nx + p] += s;
                }
            /* x^C' - x^C* = K (y^o - H^C(x^C*)) */
            for (size_t p = 0; p < nx; ++p) {
                double s = 0.0;
                for (int j = 0; j < ny; ++j) s += K[p * ny + j] * (yo[j] - hstar[j]);
                dC[p] = s;
            }
        }
        free(K);
        free(Rm);
    }
    free(yf);
    free(hstar);
    free(xbar);
    free(ybar);
    free(ebar);
    free(X);
    free(Y);
    free(Eo);
    return status;
}

/* ======================================================================== */
/* Learned correction: periodic 3x3 convolutions and pixel shuffle.          */
/* Parity: pinned (library convolution with wrap padding, library pixel      */
/* shuffle, central finite differences of the loss).                         */
/* ======================================================================== */
void orc_conv3x3(const double *in, int cin, int n, const double *W, const double *b, int cout,
                 int relu, double *out) {
    size_t pl = (size_t)n * n;
    for (int o = 0; o < cout; ++o)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                double acc = b[o];
                for (int i = 0; i < cin; ++i)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int yy = (y + dy + n) % n, xx = (x + dx + n) % n;
                            acc += W[(((size_t)o * cin + i) * 3 + dy + 1) * 3 + dx + 1] *
                                   in[i * pl + (size_t)yy * n + xx];
                        }
                if (relu && acc < 0.0) acc = 0.0;
                out[o * pl + (size_t)y * n + x] = acc;
            }
}

void orc_conv3x3_bwd(const double *in, int cin, int n, const double *W, int cout,
                     const double *dout, double *din, double *dW, double *db) {
    size_t pl = (size_t)n * n;
    for (int o = 0; o < cout; ++o) {
        double s = 0.0;
        for (size_t k = 0; k < pl; ++k) s += dout[o * pl + k];
        db[o] += s;
        for (int i = 0; i < cin; ++i)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    double g = 0.0;
                    for (int y = 0; y < n; ++y)
                        for (int x = 0; x < n; ++x) {
                            int yy = (y + dy + n) % n, xx = (x + dx + n) % n;
                            g += dout[o * pl + (size_t)y * n + x] * in[i * pl + (size_t)yy * n + xx];
                        }
                    dW[(((size_t)o * cin + i) * 3 + dy + 1) * 3 + dx + 1] += g;
                }
    }
    if (!din) return;
    for (int i = 0; i < cin; ++i)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                double acc = 0.0;
                for (int o = 0; o < cout; ++o)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            /* in[i][y][x] feeds out[o][y - dy][x - dx] through tap (dy, dx) */
                            int yy = (y - dy + n) % n, xx = (x - dx + n) % n;
                            acc += W[(((size_t)o * cin + i) * 3 + dy + 1) * 3 + dx + 1] *
                                   dout[o * pl + (size_t)yy * n + xx];
                        }
                din[i * pl + (size_t)y * n + x] = acc;
            }
}

void orc_pixel_shuffle4(const double *in, int C, int n, double *out) {
    int nf = 4 * n;
    for (int c = 0; c < C; ++c)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x)
                for (int sy = 0; sy < 4; ++sy)
                    for (int sx = 0; sx < 4; ++sx)
                        out[((size_t)c * nf + 4 * y + sy) * nf + 4 * x + sx] =
                            in[((size_t)(16 * c + 4 * sy + sx) * n + y) * n + x];
}

void orc_pixel_unshuffle4(const double *in, int C, int n, double *out) {
    int nf = 4 * n;
    for (int c = 0; c < C; ++c)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x)
                for (int sy = 0; sy < 4; ++sy)
                    for (int sx = 0; sx < 4; ++sx)
                        out[((size_t)(16 * c + 4 * sy + sx) * n + y) * n + x] =
                            in[((size_t)c * nf + 4 * y + sy) * nf + 4 * x + sx];
}

/* Relative RMSE, Eq. L2norm_u: sqrt(sum (x - x_true)^2 / sum x_true^2) per variable. */
/* ---- final fine-grid iteration and conservativity indicator (see oracle.h) ---- */
void orc_burgers_gamma(const double *x, const double *xprev, int n, double dx, double nu, double dt,
                       int flux_kind, double c, double *gamma) {
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    orc_burgers_rhs(x, n, dx, nu, flux_kind, c, L);
    for (int i = 0; i < n; ++i) gamma[i] = (x[i] - xprev[i]) / dt - L[i];
    free(L);
}

void orc_burgers_sweep(const double *x, const double *xprev, int n, double dx, double nu, double dt,
                       double alpha, int flux_kind, double c, double *out) {
    double *g = (double *)malloc(sizeof(double) * (size_t)n);
    orc_burgers_gamma(x, xprev, n, dx, nu, dt, flux_kind, c, g);
    const double D = 1.0 + 2.0 * nu * dt / (dx * dx);
    /* x_prev + dt L(x) - x = -dt Gamma */
    for (int i = 0; i < n; ++i) out[i] = x[i] + alpha * (-dt * g[i]) / D;
    free(g);
}

void orc_ns2d_gamma(const double *q, const double *qprev, int n, double h, double gamma, double mu,
                    double prandtl, double dt, double *g) {
    const size_t np = (size_t)4 * n * n;
    double *L = (double *)malloc(sizeof(double) * np);
    orc_ns2d_rhs(q, n, h, gamma, mu, prandtl, L);
    for (size_t i = 0; i < np; ++i) g[i] = (q[i] - qprev[i]) / dt - L[i];
    free(L);
}

void orc_ns2d_sweep(const double *q, const double *qprev, int n, double h, double gamma, double mu,
                    double prandtl, double dt, double alpha, double *out) {
    const size_t plane = (size_t)n * n;
    double *g = (double *)malloc(sizeof(double) * 4 * plane);
    orc_ns2d_gamma(q, qprev, n, h, gamma, mu, prandtl, dt, g);
    const double kappa = mu * gamma / ((gamma - 1.0) * prandtl);
    for (size_t p = 0; p < plane; ++p) {
        const double rho = q[p];
        const double D[4] = {1.0, 1.0 + dt * (14.0 / 3.0) * mu / (rho * h * h),
                             1.0 + dt * (14.0 / 3.0) * mu / (rho * h * h),
                             1.0 + dt * 4.0 * kappa * (gamma - 1.0) / (rho * h * h)};
        for (int v = 0; v < 4; ++v) out[v * plane + p] = q[v * plane + p] + alpha * (-dt * g[v * plane + p]) / D[v];
    }
    free(g);
}

void orc_recentre(double *members, int ne, int64_t nx, const double *xstar) {
    for (int64_t p = 0; p < nx; ++p) {
        double m = 0.0;
        for (int i = 0; i < ne; ++i) m += members[(size_t)i * nx + p];
        m /= ne;
        const double shift = xstar[p] - m;
        for (int i = 0; i < ne; ++i) members[(size_t)i * nx + p] += shift;
    }
}

void orc_rmse(const double *x, const double *truth, int V, int64_t npts, double *out) {
    for (int v = 0; v < V; ++v) {
        double num = 0.0, den = 0.0;
        for (int64_t k = 0; k < npts; ++k) {
            double d = x[v * npts + k] - truth[v * npts + k];
            num += d * d;
            den += truth[v * npts + k] * truth[v * npts + k];
        }
        out[v] = sqrt(num / den);
    }
}
