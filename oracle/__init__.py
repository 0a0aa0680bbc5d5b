"""Plain FP64 CPU oracle of the MGEnKF analysis cycle (ctypes wrapper).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library (``paper_2012_10091_gb300``) never imports it and
shares no code with it: the two meet only through the seeded input generators
in ``paper_2012_10091_gb300.workloads``, which hold none of the method's
arithmetic.

The arithmetic lives in ``oracle.c`` (FP64, literal, each routine citing the
paper).  This module only marshals numpy arrays and sequences the cycle of
Algorithm 4 (fine forecast, coarse member forecast, restriction, coarse EnKF
analysis, prolonged correction, RMSE).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

# tag of the observation-perturbation stream in the Philox key (ASCII "EPS\0")
EPS_TAG = 0x45505300
# tag of the parameter random walk of the Dual EnKF (ASCII "THTA")
THETA_TAG = 0x54485441


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, i64, u64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            L.orc_philox4x64_10.argtypes = [P, P, P]
            L.orc_normals.argtypes = [u64, u64, u64, i64, P]
            L.orc_burgers_rhs.argtypes = [P, i32, f64, f64, i32, f64, P]
            L.orc_burgers_rk3.argtypes = [P, i32, i32, f64, f64, f64, i32, i32, f64]
            L.orc_ns2d_rhs.argtypes = [P, i32, f64, f64, f64, f64, P]
            L.orc_burgers_sweep.argtypes = [P, P, i32, f64, f64, f64, f64, i32, f64, P]
            L.orc_recentre.argtypes = [P, i32, i64, P]
            L.orc_burgers_gamma.argtypes = [P, P, i32, f64, f64, f64, i32, f64, P]
            L.orc_ns2d_sweep.argtypes = [P, P, i32, f64, f64, f64, f64, f64, f64, P]
            L.orc_ns2d_gamma.argtypes = [P, P, i32, f64, f64, f64, f64, f64, P]
            L.orc_ns2d_rk3.argtypes = [P, i32, i32, f64, f64, f64, f64, f64, i32]
            L.orc_lagrange_weights.argtypes = [i32, P, f64, P]
            L.orc_restrict.argtypes = [P, i32, i32, i32, i32, P]
            L.orc_prolong_add.argtypes = [P, i32, i32, i32, i32, P]
            L.orc_obs_coarse.argtypes = [P, i32, i32, i32, i32, i32, P, P, P]
            L.orc_cholesky.argtypes = [P, i32]
            L.orc_cholesky.restype = i32
            L.orc_chol_solve.argtypes = [P, i32, P, i32]
            L.orc_enkf_analyse.argtypes = [i32, i32, i32, i32, i32, i32, P, P, P, P, f64, i32, P, P, P]
            L.orc_enkf_analyse.restype = i32
            L.orc_enkf_gain.argtypes = [i32, i32, i32, P, P, P, P]
            L.orc_enkf_gain.restype = i32
            L.orc_rmse.argtypes = [P, P, i32, i64, P]
            L.orc_set_threads.argtypes = [i32]
            L.orc_ns2d_filter6.argtypes = [P, i32, i32, f64]
            L.orc_burgers_inlet_rk3.argtypes = [P, i32, i32, f64, f64, f64, i32, f64, P, f64, f64]
            _LIB = L
    return _LIB


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's parallel loops (timing only: every
    parallel loop runs over independent problems or members)."""
    lib().orc_set_threads(int(n))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


# --------------------------------------------------------------------------
# primitives
# --------------------------------------------------------------------------
def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def normals(seed: int, tag: int, ctr0: int, count: int) -> np.ndarray:
    z = np.zeros(max(count, 1), dtype=np.float64)
    lib().orc_normals(seed, tag, ctr0, count, _p(z))
    return z[:count]


def obs_perturbations(seed: int, cycle: int, ne: int, ny: int, sigma: float) -> np.ndarray:
    """eps^(i) ~ N(0, sigma^2 I) for one analysis (Eq. perturbed_y), ne x ny."""
    return sigma * normals(seed, EPS_TAG, cycle, ne * ny).reshape(ne, ny)


def burgers_rhs(u, dx, nu, flux_kind=0, c=0.0) -> np.ndarray:
    u = _f64(u)
    L = np.zeros_like(u)
    lib().orc_burgers_rhs(_p(u), u.size, dx, nu, flux_kind, c, _p(L))
    return L


def burgers_rk3(u, dx, nu, dt, nsteps, flux_kind=0, c=0.0) -> np.ndarray:
    """Advance every row of ``u`` (nprob x n, or n) by nsteps SSP-RK3 steps."""
    x = _f64(u).copy()
    shape = x.shape
    x2 = x.reshape(-1, shape[-1])
    lib().orc_burgers_rk3(_p(x2), x2.shape[0], x2.shape[1], dx, nu, dt, nsteps, flux_kind, c)
    return x2.reshape(shape)


def burgers_inlet_rk3(u, dx, nu, dt, nsteps, t0, theta, u0=1.0, omega=2 * np.pi) -> np.ndarray:
    """Advance every row of u (nprob x n, or n) with its inlet parameters
    theta (nprob x 2: amplitude, phase) from time t0 (see oracle.h)."""
    x = _f64(u).copy()
    shape = x.shape
    x2 = x.reshape(-1, shape[-1])
    th = _f64(theta).reshape(x2.shape[0], 2)
    lib().orc_burgers_inlet_rk3(_p(x2), x2.shape[0], x2.shape[1], dx, nu, dt, nsteps, t0, _p(th), u0, omega)
    return x2.reshape(shape)


def _ns_side(q) -> int:
    """Points per side of a 4 x n x n state given flat or shaped."""
    n = q.shape[-1] if q.ndim > 1 else int(round((q.size // 4) ** 0.5))
    if q.size % (4 * n * n):
        raise ValueError("NS-2D state must hold 4 x n x n values per grid")
    return n


def ns2d_rhs(q, h, gamma, mu, prandtl) -> np.ndarray:
    q = _f64(q)
    L = np.zeros_like(q)
    if q.size != 4 * _ns_side(q) ** 2:
        raise ValueError("ns2d_rhs takes one grid")
    lib().orc_ns2d_rhs(_p(q), _ns_side(q), h, gamma, mu, prandtl, _p(L))
    return L


def recentre(members, xstar) -> np.ndarray:
    """Members re-centred on x^C* (fine-to-coarse feedback; see oracle.h)."""
    m = _f64(members).copy()
    xs = _f64(xstar)
    ne = m.shape[0]
    lib().orc_recentre(_p(m), ne, m.size // ne, _p(xs))
    return m


def burgers_sweep(x, xprev, dx, nu, dt, alpha, flux_kind=0, c=0.0) -> np.ndarray:
    """One relaxed Jacobi sweep of the implicit last step (Algorithm 4 step 6; see oracle.h)."""
    x, xp = _f64(x), _f64(xprev)
    out = np.empty_like(x)
    lib().orc_burgers_sweep(_p(x), _p(xp), x.size, dx, nu, dt, alpha, flux_kind, c, _p(out))
    return out


def burgers_gamma(x, xprev, dx, nu, dt, flux_kind=0, c=0.0) -> np.ndarray:
    """Conservativity residual (x - x_prev)/dt - L(x) (Eq. Conservativity_rhov)."""
    x, xp = _f64(x), _f64(xprev)
    out = np.empty_like(x)
    lib().orc_burgers_gamma(_p(x), _p(xp), x.size, dx, nu, dt, flux_kind, c, _p(out))
    return out


def ns2d_sweep(q, qprev, h, gamma, mu, prandtl, dt, alpha) -> np.ndarray:
    q, qp = _f64(q), _f64(qprev)
    n = _ns_side(q)
    if q.size != 4 * n * n or qp.size != q.size:
        raise ValueError("ns2d_sweep takes one grid and its previous state")
    out = np.empty_like(q)
    lib().orc_ns2d_sweep(_p(q), _p(qp), n, h, gamma, mu, prandtl, dt, alpha, _p(out))
    return out


def ns2d_gamma(q, qprev, h, gamma, mu, prandtl, dt) -> np.ndarray:
    q, qp = _f64(q), _f64(qprev)
    n = _ns_side(q)
    if q.size != 4 * n * n or qp.size != q.size:
        raise ValueError("ns2d_gamma takes one grid and its previous state")
    out = np.empty_like(q)
    lib().orc_ns2d_gamma(_p(q), _p(qp), n, h, gamma, mu, prandtl, dt, _p(out))
    return out


def gamma_normalised(gamma, x, xprev, dt, V) -> np.ndarray:
    """Gamma* = Gamma / C per variable with C = max over the grid of
    |(x - x_prev)/dt| (Sec. 6, the normalisation of the conservativity maps;
    reading: the maximum is over the grid points at the analysis time)."""
    g = _f64(gamma).reshape(V, -1)
    rate = (_f64(x) - _f64(xprev)).reshape(V, -1) / dt
    c = np.abs(rate).max(axis=1, keepdims=True)
    return (g / np.where(c > 0, c, 1.0)).reshape(-1)


def ns2d_rk3(q, h, gamma, mu, prandtl, dt, nsteps) -> np.ndarray:
    """Advance (nprob x) 4 x n x n conserved states by nsteps SSP-RK3 steps."""
    x = _f64(q).copy()
    shape = x.shape
    n = _ns_side(x)
    x2 = x.reshape(-1, 4, n, n)
    lib().orc_ns2d_rk3(_p(x2), x2.shape[0], n, h, gamma, mu, prandtl, dt, nsteps)
    return x2.reshape(shape)


def ns2d_filter6(q, sigma) -> np.ndarray:
    """Centred sixth-order filter (Secs. 5, 6) of (nprob x) 4 x n x n conserved states."""
    x = _f64(q).copy()
    shape = x.shape
    n = _ns_side(x)
    x2 = x.reshape(-1, 4, n, n)
    lib().orc_ns2d_filter6(_p(x2), x2.shape[0], n, float(sigma))
    return x2.reshape(shape)


def lagrange_weights(nodes, s) -> np.ndarray:
    nd = _f64(nodes)
    w = np.zeros_like(nd)
    lib().orc_lagrange_weights(nd.size, _p(nd), s, _p(w))
    return w


def restrict(fine, dim, V, nc, r) -> np.ndarray:
    f = _f64(fine)
    out = np.zeros(V * nc**dim, dtype=np.float64)
    lib().orc_restrict(_p(f), dim, V, nc, r, _p(out))
    return out


def prolong_add(dc, fine, dim, V, nc, r) -> np.ndarray:
    d = _f64(dc)
    f = _f64(fine).copy()
    lib().orc_prolong_add(_p(d), dim, V, nc, r, _p(f))
    return f


def obs_coarse(xc, dim, V, nc, r, obs_idx, obs_var) -> np.ndarray:
    x = _f64(xc)
    oi, ov = _i32(obs_idx), _i32(obs_var)
    y = np.zeros(oi.size, dtype=np.float64)
    lib().orc_obs_coarse(_p(x), dim, V, nc, r, oi.size, _p(oi), _p(ov), _p(y))
    return y


def cholesky(A):
    a = _f64(A).copy()
    st = lib().orc_cholesky(_p(a), a.shape[0])
    return st, a


def enkf_gain(X, Y, R):
    X, Y, R = _f64(X), _f64(Y), _f64(R)
    nx, ne = X.shape
    ny = Y.shape[0]
    K = np.zeros((nx, ny))
    st = lib().orc_enkf_gain(nx, ne, ny, _p(X), _p(Y), _p(R), _p(K))
    return st, K


def enkf_analyse(members, xstar, yo, eps, sigma, obs_idx, obs_var, dim, V, nc, r, gain_form=1):
    """Returns (status, members_analysed, dC).  See orc_enkf_analyse."""
    m = _f64(members).copy()
    ne = m.shape[0]
    xs, y, e = _f64(xstar), _f64(yo), _f64(eps)
    oi, ov = _i32(obs_idx), _i32(obs_var)
    dC = np.zeros(m.shape[1], dtype=np.float64)
    st = lib().orc_enkf_analyse(dim, V, nc, r, ne, oi.size, _p(oi), _p(ov), _p(y), _p(e), sigma,
                                gain_form, _p(m), _p(xs), _p(dC))
    return st, m, dC


def rmse(x, truth, V) -> np.ndarray:
    x, t = _f64(x), _f64(truth)
    out = np.zeros(V)
    lib().orc_rmse(_p(x), _p(t), V, x.size // V, _p(out))
    return out


# --------------------------------------------------------------------------
# the cycle of Algorithm 4 (state part of Algorithm 3 on the coarse mesh)
# --------------------------------------------------------------------------
class MGEnKF:
    """FP64 oracle of one MGEnKF run.  All inputs come from the caller.

    model: "burgers1d" or "ns2d"; fine (V*nf^dim), members (ne x V*nc^dim).
    """

    def __init__(self, model, nf, ratio, length, dt, fine, members, obs_idx, obs_var, sigma,
                 seed, nu=0.0, gamma=1.4, prandtl=0.72, gain_form=1, alpha=0.0, recentre=False,
                 filter_sigma=0.0):
        self.model = model
        self.dim = 1 if model == "burgers1d" else 2
        self.V = 1 if model == "burgers1d" else 4
        self.nf, self.r = nf, ratio
        self.nc = nf // ratio
        self.length, self.dt, self.nu = length, dt, nu
        self.gamma, self.prandtl = gamma, prandtl
        self.fine = _f64(fine).copy()
        self.members = _f64(members).copy()
        self.obs_idx, self.obs_var = _i32(obs_idx), _i32(obs_var)
        self.sigma, self.seed, self.gain_form = sigma, seed, gain_form
        self.cycle = 0
        self.xstar = None
        self.dC = None
        self.alpha = alpha          # final fine iteration (Algorithm 4 step 6); 0 = none
        self.recentre = recentre    # re-centre the forecast ensemble on x^C* before each analysis
        self.fine_prev = None       # fine state one model step before the analysis time
        self.filter_sigma = filter_sigma  # NS: sixth-order filter after every model step (0 = off)

    def _advance(self, x, n, nsteps):
        h = self.length / n
        if self.model == "burgers1d":
            return burgers_rk3(x, h, self.nu, self.dt, nsteps)
        q = x.reshape(-1, 4, n, n)
        if self.filter_sigma > 0:
            for _ in range(nsteps):   # the model step is the RK3 step followed by the filter
                q = ns2d_filter6(ns2d_rk3(q, h, self.gamma, self.nu, self.prandtl, self.dt, 1),
                                 self.filter_sigma)
            return q.reshape(x.shape)
        return ns2d_rk3(q, h, self.gamma, self.nu, self.prandtl, self.dt, nsteps).reshape(x.shape)

    def forecast(self, nsteps):
        """Algorithm 4 step 2 (fine) and Algorithm 3 step 2 (members)."""
        if nsteps > 0:
            self.fine_prev = self._advance(self.fine, self.nf, nsteps - 1)
            self.fine = self._advance(self.fine_prev, self.nf, 1)
        self.members = self._advance(self.members, self.nc, nsteps)

    def analyse(self, yo, eps=None):
        """Algorithm 4 step 4 then Algorithm 3 steps 2-8 and Algorithm 4 step 5."""
        ne, ny = self.members.shape[0], self.obs_idx.size
        if eps is None:
            eps = obs_perturbations(self.seed, self.cycle, ne, ny, self.sigma)
        self.xstar = restrict(self.fine, self.dim, self.V, self.nc, self.r)
        if self.recentre:
            self.members = recentre(self.members, self.xstar)
        st, m, dC = enkf_analyse(self.members, self.xstar, yo, eps, self.sigma, self.obs_idx,
                                 self.obs_var, self.dim, self.V, self.nc, self.r, self.gain_form)
        if st == 0:
            self.members, self.dC = m, dC
        self.cycle += 1
        return st

    def prolong_correct(self):
        """x^F,a = x^F,f + Pi_F(x^C' - x^C*), then (alpha > 0) the final fine
        iteration of Algorithm 4 step 6."""
        self.fine = prolong_add(self.dC, self.fine, self.dim, self.V, self.nc, self.r)
        if self.alpha > 0.0 and self.fine_prev is not None:
            self.fine = self.sweep(self.alpha)

    def sweep(self, alpha):
        h = self.length / self.nf
        if self.model == "burgers1d":
            return burgers_sweep(self.fine, self.fine_prev, h, self.nu, self.dt, alpha)
        return ns2d_sweep(self.fine, self.fine_prev, h, self.gamma, self.nu, self.prandtl, self.dt, alpha)

    def gamma_residual(self):
        """Conservativity residual of the fine state (Eq. Conservativity_rhov)."""
        h = self.length / self.nf
        if self.model == "burgers1d":
            return burgers_gamma(self.fine, self.fine_prev, h, self.nu, self.dt)
        return ns2d_gamma(self.fine, self.fine_prev, h, self.gamma, self.nu, self.prandtl, self.dt)

    def rmse(self, truth):
        return rmse(self.fine, truth, self.V)


# --------------------------------------------------------------------------
# learned correction: residual CNN over Pi_F (8 -> 32 -> 32 -> 64 channels,
# periodic 3x3 convolutions, ReLU, pixel shuffle by 4)
# --------------------------------------------------------------------------
CNN_SHAPES = [("W1", (32, 8, 3, 3)), ("b1", (32,)), ("W2", (32, 32, 3, 3)), ("b2", (32,)),
              ("W3", (64, 32, 3, 3)), ("b3", (64,))]


def _cnn_sigs():
    L = lib()
    if getattr(L, "_cnn_ready", False):
        return L
    P, i32 = ctypes.c_void_p, ctypes.c_int
    L.orc_conv3x3.argtypes = [P, i32, i32, P, P, i32, i32, P]
    L.orc_conv3x3_bwd.argtypes = [P, i32, i32, P, i32, P, P, P, P]
    L.orc_pixel_shuffle4.argtypes = [P, i32, i32, P]
    L.orc_pixel_unshuffle4.argtypes = [P, i32, i32, P]
    L._cnn_ready = True
    return L


def conv3x3(x, W, b, relu=False):
    L = _cnn_sigs()
    x, W, b = _f64(x), _f64(W), _f64(b)
    cout, cin = W.shape[0], W.shape[1]
    n = x.shape[-1]
    out = np.zeros((cout, n, n))
    L.orc_conv3x3(_p(x), cin, n, _p(W), _p(b), cout, int(relu), _p(out))
    return out


def conv3x3_bwd(x, W, dout, want_din=True):
    L = _cnn_sigs()
    x, W, dout = _f64(x), _f64(W), _f64(dout)
    cout, cin = W.shape[0], W.shape[1]
    n = x.shape[-1]
    dW = np.zeros_like(W)
    db = np.zeros(cout)
    din = np.zeros((cin, n, n)) if want_din else None
    L.orc_conv3x3_bwd(_p(x), cin, n, _p(W), cout, _p(dout), _p(din) if want_din else None, _p(dW), _p(db))
    return din, dW, db


def pixel_shuffle4(x):
    L = _cnn_sigs()
    x = _f64(x)
    C, n = x.shape[0] // 16, x.shape[-1]
    out = np.zeros((C, 4 * n, 4 * n))
    L.orc_pixel_shuffle4(_p(x), C, n, _p(out))
    return out


def pixel_unshuffle4(x):
    L = _cnn_sigs()
    x = _f64(x)
    C, n = x.shape[0], x.shape[-1] // 4
    out = np.zeros((16 * C, n, n))
    L.orc_pixel_unshuffle4(_p(x), C, n, _p(out))
    return out


def cnn_forward(params, dC, xstar, stats):
    """Fine correction of one sample: Pi_F(dC) + s_out * shuffle(CNN(normalised [dC, x*])).
    dC, xstar: 4 x nc x nc.  stats: dict(mu_in (8), s_in (8), s_out (4)).
    Returns (prediction 4 x 4nc x 4nc, cache for the backward pass)."""
    nc = dC.shape[-1]
    a0 = (np.concatenate([dC, xstar]) - stats["mu_in"][:, None, None]) / stats["s_in"][:, None, None]
    z1 = conv3x3(a0, params["W1"], params["b1"])
    a1 = np.maximum(z1, 0.0)
    z2 = conv3x3(a1, params["W2"], params["b2"])
    a2 = np.maximum(z2, 0.0)
    z3 = conv3x3(a2, params["W3"], params["b3"])
    res = pixel_shuffle4(z3) * stats["s_out"][:, None, None]
    base = prolong_add(dC.reshape(-1), np.zeros(4 * (4 * nc) ** 2), 2, 4, nc, 4).reshape(4, 4 * nc, 4 * nc)
    return base + res, dict(a0=a0, z1=z1, a1=a1, z2=z2, a2=a2)


def cnn_loss_grad(params, dC, xstar, target, stats):
    """Loss = mean over fine points and channels of ((pred - target) / s_out)^2,
    and its gradient with respect to every parameter."""
    pred, c = cnn_forward(params, dC, xstar, stats)
    s_out = stats["s_out"][:, None, None]
    r = (pred - target) / s_out
    N = r.size
    loss = float(np.sum(r * r) / N)
    dpred = 2.0 * r / s_out / N
    dz3 = pixel_unshuffle4(dpred * s_out)
    da2, dW3, db3 = conv3x3_bwd(c["a2"], params["W3"], dz3)
    dz2 = da2 * (c["z2"] > 0)
    da1, dW2, db2 = conv3x3_bwd(c["a1"], params["W2"], dz2)
    dz1 = da1 * (c["z1"] > 0)
    _, dW1, db1 = conv3x3_bwd(c["a0"], params["W1"], dz1, want_din=False)
    return loss, dict(W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3)


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) with bias correction; state holds m, v, t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = b1 * m + (1 - b1) * grads[k]
        v[...] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1**t)
        vh = v / (1 - b2**t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


# --------------------------------------------------------------------------
# Dual EnKF parameter estimation (Algorithm 3 with its parameter rows, inside
# Algorithm 4) on the Burgers inlet model of Sec. 4
# --------------------------------------------------------------------------
def open_prolong_rows(nc: int, r: int):
    """Pi_F on an open 1-D grid (coarse node J at fine node r J, no wrap): for
    every fine node k the first of its 4 coarse nodes j0 = clamp(k // r - 1,
    0, nc - 4) and the cubic Lagrange weights through j0 .. j0 + 3 at k / r
    (one-sided near the ends; beyond the last coarse node it extrapolates)."""
    j0 = np.empty(nc * r, dtype=np.int64)
    w = np.empty((nc * r, 4))
    for k in range(nc * r):
        j0[k] = min(max(k // r - 1, 0), nc - 4)
        w[k] = lagrange_weights(np.arange(j0[k], j0[k] + 4, dtype=np.float64), k / r)
    return j0, w


def open_prolong(dC, nc: int, r: int) -> np.ndarray:
    j0, w = open_prolong_rows(nc, r)
    idx = j0[:, None] + np.arange(4)[None, :]
    return (w * _f64(dC)[idx]).sum(axis=1)


def open_obs_rows(obs_idx, nc: int, r: int):
    """H^C rows of fine-node observations: the open Pi_F row at each node."""
    j0, w = open_prolong_rows(nc, r)
    k = np.asarray(obs_idx, dtype=np.int64)
    return j0[k], w[k]


def _anomalies(A) -> np.ndarray:
    """Normalised anomalies (Eq. Ensemble_Anomaly) of the ensemble rows of A (ne x p), p x ne."""
    A = _f64(A)
    return (A - A.mean(axis=0)).T / np.sqrt(A.shape[0] - 1)


class DualMGEnKF:
    """FP64 oracle of the multigrid Dual EnKF on the Burgers inlet model.

    One cycle follows Algorithm 4 with Algorithm 3 on the coarse grid:
      step 2 (Alg. 4): fine forecast with the analysed parameter mean;
      step 2 (Alg. 3): parameter forecast theta^f = theta^a + tau (random walk,
        tau ~ N(0, q I)) and member forecast with theta^f;
      steps 3-5: observation ensemble y^o + eps^(i), parameter gain
        K^theta = Theta Y^T (Y Y^T + R)^-1, theta^a = theta^f + K^theta (y^o,(i) - y^f,(i));
      steps 6-8: member forecast again from the previous analysis with theta^a,
        state gain K^x = X Y^T (Y Y^T + R)^-1 from it, member update;
      steps 4-5 (Alg. 4): x^C' - x^C* = K^x (y^o - H^C x^C*), fine correction Pi_F.
    R is the exact sigma^2 I (the reading of the build); projections are the
    open-grid 4-point Lagrange interpolants (one-sided at the ends)."""

    def __init__(self, nf, ratio, length, dt, nu, fine, members, theta, theta_fine, obs_idx, sigma,
                 seed, theta_q, u0=1.0, omega=2 * np.pi, t0=0.0):
        self.nf, self.r = nf, ratio
        self.nc = nf // ratio
        self.length, self.dt, self.nu = length, dt, nu
        self.u0, self.omega = u0, omega
        self.fine = _f64(fine).copy()
        self.members = _f64(members).copy()
        self.theta = _f64(theta).reshape(-1, 2).copy()
        self.theta_fine = _f64(theta_fine).reshape(2).copy()
        self.obs_idx = np.asarray(obs_idx, dtype=np.int64)
        self.sigma, self.seed, self.theta_q = sigma, seed, theta_q
        self.t = t0
        self.cycle = 0
        self.hj0, self.hw = open_obs_rows(self.obs_idx, self.nc, self.r)

    def observe(self, xc) -> np.ndarray:
        """H^C of coarse states (rows of xc), ne x ny (or ny)."""
        xc = _f64(xc)
        idx = self.hj0[:, None] + np.arange(4)[None, :]
        return (self.hw * xc[..., idx]).sum(axis=-1)

    def _gain(self, A, Yf) -> np.ndarray:
        Y = _anomalies(Yf)                       # ny x ne
        C = Y @ Y.T + self.sigma ** 2 * np.eye(Y.shape[0])
        return np.linalg.solve(C, (A @ Y.T).T).T  # A Y^T C^-1

    def free_run(self, nsteps):
        """Forecast without analysis (spin-up): fine with its parameters, members with theirs."""
        dxf, dxc = self.length / self.nf, self.length / self.nc
        self.fine = burgers_inlet_rk3(self.fine, dxf, self.nu, self.dt, nsteps, self.t, self.theta_fine,
                                      self.u0, self.omega)
        self.members = burgers_inlet_rk3(self.members, dxc, self.nu, self.dt, nsteps, self.t, self.theta,
                                         self.u0, self.omega)
        self.t += nsteps * self.dt

    def cycle_step(self, nsteps, yo, eps=None, tau=None):
        ne = self.members.shape[0]
        ny = self.obs_idx.size
        dxf, dxc = self.length / self.nf, self.length / self.nc
        yo = _f64(yo)
        fine_f = burgers_inlet_rk3(self.fine, dxf, self.nu, self.dt, nsteps, self.t, self.theta_fine,
                                   self.u0, self.omega)
        if tau is None:
            tau = np.sqrt(self.theta_q) * normals(self.seed, THETA_TAG, self.cycle, 2 * ne).reshape(ne, 2)
        theta_f = self.theta + tau
        xf = burgers_inlet_rk3(self.members, dxc, self.nu, self.dt, nsteps, self.t, theta_f,
                               self.u0, self.omega)
        if eps is None:
            eps = obs_perturbations(self.seed, self.cycle, ne, ny, self.sigma)
        Yf = self.observe(xf)
        Kt = self._gain(_anomalies(theta_f), Yf)               # 2 x ny
        theta_a = theta_f + (yo[None, :] + eps - Yf) @ Kt.T
        xf2 = burgers_inlet_rk3(self.members, dxc, self.nu, self.dt, nsteps, self.t, theta_a,
                                self.u0, self.omega)
        Yf2 = self.observe(xf2)
        Kx = self._gain(_anomalies(xf2), Yf2)                  # nc x ny
        self.members = xf2 + (yo[None, :] + eps - Yf2) @ Kx.T
        xs = fine_f[::self.r][:self.nc]
        dC = Kx @ (yo - self.observe(xs))
        self.fine = fine_f + open_prolong(dC, self.nc, self.r)
        self.theta = theta_a
        self.theta_fine = theta_a.mean(axis=0)
        self.t += nsteps * self.dt
        self.cycle += 1
        self.xstar, self.dC = xs, dC
        return theta_a
