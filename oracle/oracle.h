/*
 * oracle.h -- plain FP64 CPU oracle of the MGEnKF analysis cycle.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The GPU library never
 * includes this header and shares no code, table or helper with it.
 *
 * Every routine follows the paper's statement of the method in FP64, without
 * blocking, fusion or reordering beyond what the definition states:
 *   - EnKF definitions (ensemble matrix, mean, normalised anomalies,
 *     perturbed observations, gain): Sec. 2.1.2, Eqs. Ensemble_Matrix ..
 *     ensemble_update, and Algorithm 1 (stochastic EnKF with anomalies);
 *   - coarse-mesh filter (state part): Algorithm 3, steps 2, 3, 7, 8;
 *   - multigrid correction: Algorithm 4, steps 2, 4, 5; Sec. 3 step 5;
 *   - projectors: 4th-order Lagrange interpolators (end of Sec. 2.2);
 *   - relative RMSE: Eq. L2norm_u (Sec. 4);
 *   - models: viscous Burgers (Eq. burgers), compressible NS (Eqs. Mass,
 *     Momentum, Energy) with the periodic discretisations stated in each
 *     routine's comment.
 * Parity status of each routine is stated beside it.
 */
#ifndef MGENKF_ORACLE_H
#define MGENKF_ORACLE_H
#include <stdint.h>

/* OpenMP threads of the parallel loops (over independent problems/members:
 * results do not depend on it); used to time the oracle on one core. */
void orc_set_threads(int n);

/* ---- counter-based RNG: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----
 * Pinned: against numpy.random.Philox (library) and published known answers. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Standard normals z[n], n = 0..count-1, drawn by Box-Muller from Philox
 * blocks ctr = (ctr0, n/4, 0, 0), key = (seed, tag); lanes (0,1) and (2,3)
 * of a block give one Box-Muller pair each.  u = ((x >> 11) + 1) * 2^-53. */
void orc_normals(uint64_t seed, uint64_t tag, uint64_t ctr0, int64_t count, double *z);
/* Parity: pinned (moments, kurtosis, Kolmogorov-Smirnov, lag correlations). */

/* ---- 1-D viscous Burgers (Eq. burgers), periodic, flux form ----
 * L(u)_j = -(F_{j+1} - F_{j-1}) / (2 dx) + nu (u_{j+1} - 2 u_j + u_{j-1}) / dx^2
 * with F = u^2/2 (flux_kind 0) or F = c u (flux_kind 1, linear advection,
 * used only to pin the scheme against its Fourier amplification factor).
 * Time: SSP-RK3 in Shu-Osher form.  nprob independent grids of n points,
 * stored one after the other. */
void orc_burgers_rhs(const double *u, int n, double dx, double nu, int flux_kind, double c,
                     double *L);
void orc_burgers_rk3(double *u, int nprob, int n, double dx, double nu, double dt, int nsteps,
                     int flux_kind, double c);
/* Parity: pinned (Fourier amplification factor of the linear-flux scheme,
 * second-order convergence to the Cole-Hopf solution, mass conservation, a
 * hand-computed right-hand side). */

/* ---- 2-D compressible Navier-Stokes (Eqs. Mass, Momentum, Energy) ----
 * Periodic square, q = (rho, rho u, rho v, E) as 4 planes of n x n (x fastest).
 * Non-dimensional: p = (gamma-1)(E - rho |u|^2 / 2), T = p / rho, constant
 * mu, kappa = mu gamma / ((gamma-1) Pr).  Inviscid fluxes: central
 * differences of nodal fluxes.  Viscous and heat fluxes: evaluated at cell
 * faces (compact normal derivative, averaged central tangential derivative)
 * and differenced across the cell, so every flux telescopes.  SSP-RK3. */
void orc_ns2d_rhs(const double *q, int n, double h, double gamma, double mu, double prandtl,
                  double *L);
/* Burgers with a time-varying inlet (Sec. 4, Eqs. burgers and
 * inlet-1D-Burgers): node 0 = u0 (1 + theta1 sin(omega t + theta2)), outlet
 * extrapolated linearly, flux-form central interior, SSP-RK3 with the inlet at
 * each stage time; theta is nprob x 2.  Parity: pinned (a uniform state with
 * theta1 = 0 stays exact; the small-amplitude inlet signal converges at second
 * order to the closed-form time-harmonic solution of the linearised equation). */
void orc_burgers_inlet_rk3(double *u, int nprob, int n, double dx, double nu, double dt, int nsteps,
                           double t0, const double *theta, double u0, double omega);

/* Centred sixth-order filter of the NS model (Secs. 5, 6; Bogey and Bailly):
 * reading: the 7-point stencil with transfer function 1 - sigma sin^6(k h/2),
 * along x then y on the 4 conserved planes of nprob periodic n x n grids.
 * Parity: pinned (Fourier-mode damping in closed form, conservation of the
 * totals, constants kept, grid-scale mode removed at sigma = 1). */
void orc_ns2d_filter6(double *q, int nprob, int n, double sigma);
void orc_ns2d_rk3(double *q, int nprob, int n, double h, double gamma, double mu,
                  double prandtl, double dt, int nsteps);
/* Parity: pinned (conservation of the four totals, steady uniform state,
 * x-y transpose symmetry, acoustic dispersion, viscous decay of a shear mode;
 * the 4 x 4 discrete symbol of the right-hand side linearised about rest,
 * which fixes the 4/3 and -2/3 stress factors, the cross terms and kappa;
 * exact states for the heat flux kappa lap T (density wave at constant p)
 * and for the viscous work tau . u (transverse shear, longitudinal stretch)). */

/* ---- projectors Pi_C, Pi_F (end of Sec. 2.2) ----
 * Vertex-centred nested periodic grids, coarse node J at fine node r J.
 * Pi_F: 4-point Lagrange interpolation over coarse nodes J-1..J+2 (tensor
 * product in 2-D).  Pi_C: the same interpolant at coincident nodes
 * (injection).  dim = 1 or 2, V variables, nc coarse points per side. */
void orc_lagrange_weights(int npts, const double *nodes, double s, double *w);
void orc_restrict(const double *fine, int dim, int V, int nc, int r, double *coarse);
void orc_prolong_add(const double *dc, int dim, int V, int nc, int r, double *fine);
/* H^C: Pi_F row at each observed fine node; obs_idx = flat fine index
 * (y*nf + x in 2-D), obs_var = variable.  y[j] = (Pi_F xc)[obs_var[j]][obs_idx[j]] */
void orc_obs_coarse(const double *xc, int dim, int V, int nc, int r, int ny,
                    const int32_t *obs_idx, const int32_t *obs_var, double *y);
/* Parity: pinned (Pi_C Pi_F = I, exactness on cubics, fourth-order error on
 * Fourier modes, H^C equal to the Pi_F row). */

/* ---- Cholesky (textbook), returns 0 or the failing pivot index + 1 ----
 * Parity: pinned (L L^T = A by brute force, the library factor, the index of a
 * failing pivot); the solve through the EnKF analysis's dense brute force. */
int orc_cholesky(double *A, int n);
void orc_chol_solve(const double *Lf, int n, double *b, int nrhs);

/* ---- EnKF analysis on the coarse mesh + multigrid correction ----
 * Algorithm 3 (state part, steps 2-3 and 7-8) then Algorithm 4 step 5 first
 * line.  members: ne x nx (member-major), updated in place to the analysis.
 * xstar: Pi_C of the fine forecast.  yo: ny observations.  eps: ne x ny
 * observation perturbations (already scaled by sigma).  gain_form:
 *   0 = literal gain K = X Y^T (Y Y^T + R)^-1 with exact R = sigma^2 I
 *   1 = ensemble-space form T = (I + Y^T R^-1 Y)^-1 Y^T R^-1 [D | d*]
 *   2 = literal gain with the sample R^e = E E^T of the centred E (Sec. 2.1.2)
 * dC (out): x^C' - x^C* = K (yo - H^C x*).  Returns 0, or 1 if the innovation
 * matrix is not SPD (members and dC untouched). */
int orc_enkf_analyse(int dim, int V, int nc, int r, int ne, int ny, const int32_t *obs_idx,
                     const int32_t *obs_var, const double *yo, const double *eps, double sigma,
                     int gain_form, double *members, const double *xstar, double *dC);
/* Parity: pinned (dense brute force for the three gain forms at small sizes,
 * the sigma limits, convergence to the Kalman filter as Ne grows). */

/* Dense Kalman gain K (nx x ny) of the literal form, for brute-force pins. */
int orc_enkf_gain(int nx, int ne, int ny, const double *X, const double *Y, const double *Rm,
                  double *K);

/* ---- learned correction (residual over Pi_F; no counterpart in the paper,
 * whose conclusion names better projection operators as future work) ----
 * 3x3 cross-correlation with periodic padding, one sample:
 *   out[o][y][x] = b[o] + sum_{i, dy, dx} W[o][i][dy+1][dx+1] in[i][(y+dy) mod n][(x+dx) mod n]
 * optionally followed by ReLU.  Backward: accumulates dW, db and (if din is
 * not NULL) writes din = W^T * dout (the adjoint correlation). */
void orc_conv3x3(const double *in, int cin, int n, const double *W, const double *b, int cout,
                 int relu, double *out);
void orc_conv3x3_bwd(const double *in, int cin, int n, const double *W, int cout,
                     const double *dout, double *din, double *dW, double *db);
/* pixel shuffle by 4: in = 16 C channels of n x n, out = C channels of 4n x 4n,
 * out[c][4y + sy][4x + sx] = in[16 c + 4 sy + sx][y][x]; unshuffle is its adjoint. */
void orc_pixel_shuffle4(const double *in, int C, int n, double *out);
void orc_pixel_unshuffle4(const double *in, int C, int n, double *out);
/* Parity: pinned (a library convolution, automatic differentiation of the
 * backward pass, a library pixel shuffle, central differences of the loss
 * gradient). */

/* ---- final fine-grid iteration (Algorithm 4 step 6) and the conservativity
 * indicator (Eq. Conservativity_rhov) ----
 * Reading: the last model step of the observation interval in implicit-Euler
 * form, Psi(x) = x - dt L(x) = c with c = x_prev (the fine state one step
 * before the analysis time), and one relaxed Jacobi (matrix-splitting) sweep
 * from the analysis state x (Sec. 3 tailoring: one iteration, alpha = 0.5):
 *   out = x + alpha D^-1 (x_prev + dt L(x) - x),
 * D the diagonal of dPsi/dx at x.  Burgers (central fluxes have no diagonal
 * term): D = 1 + 2 nu dt / dx^2.  NS-2D, per point: D = 1 for rho, 1 + dt
 * (14/3) mu / (rho h^2) for rho u and rho v (compact face derivatives: 8/3 from
 * tau_xx or tau_yy, 2 from tau_xy), 1 + dt 4 kappa (gamma - 1) / (rho h^2) for
 * E (heat fluxes through T = (gamma - 1)(E - rho |u|^2 / 2) / rho).
 * Gamma = (x - x_prev) / dt - L(x): the residual of that implicit step, the
 * paper's conservativity indicator (there for rho v).  Parity: pinned
 * (identity at alpha = 0, implicit solution is a fixed point, closed-form
 * damping of Fourier modes, D against a finite-difference Jacobian). */
void orc_burgers_sweep(const double *x, const double *xprev, int n, double dx, double nu, double dt,
                       double alpha, int flux_kind, double c, double *out);
void orc_burgers_gamma(const double *x, const double *xprev, int n, double dx, double nu, double dt,
                       int flux_kind, double c, double *gamma);
void orc_ns2d_sweep(const double *q, const double *qprev, int n, double h, double gamma, double mu,
                    double prandtl, double dt, double alpha, double *out);
void orc_ns2d_gamma(const double *q, const double *qprev, int n, double h, double gamma, double mu,
                    double prandtl, double dt, double *g);

/* ---- fine-to-coarse feedback (the paper's conclusion: project the fine
 * run's information onto the members) ----
 * Reading: before each analysis, re-centre the forecast ensemble on the
 * restricted fine forecast x^C*: x^(i) <- x^(i) - mean_i x^(i) + x^C*.  The
 * anomalies are unchanged.  members: ne x nx, member-major.  Parity: pinned
 * (mean equals x^C*, anomalies unchanged, analysis mean = x^C' + K mean(eps)). */
void orc_recentre(double *members, int ne, int64_t nx, const double *xstar);

/* ---- relative RMSE, Eq. L2norm_u, one value per variable ----
 * Parity: pinned (closed forms: uniform relative error per plane, an offset
 * on a sine, the truth as the denominator). */
void orc_rmse(const double *x, const double *truth, int V, int64_t npts, double *out);

#endif
