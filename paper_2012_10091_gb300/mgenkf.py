"""Python binding of the MGEnKF C ABI (``include/mgenkf.h``, ``include/mgenkf_ops.h``).

Argument marshalling only: every function forwards to the entry point of the
same name in ``libmgenkf.so``.  Arrays may be numpy arrays (host memory) or
objects with ``data_ptr()`` (torch tensors, host or device); the library tells
host from device pointers itself.  There is no fallback: if the compiled
library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgenkf.so")

MGENKF_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_SPD", 5: "NONFINITE",
                6: "UNSUPPORTED", 7: "TIMEOUT"}
MGENKF_BURGERS1D, MGENKF_NS2D = 1, 2
MGENKF_FP64, MGENKF_MIXED = 0, 1
MGENKF_GAIN_ENSEMBLE, MGENKF_GAIN_DIRECT = 0, 1
MGENKF_PROLONG_LAGRANGE4 = 0
MGENKF_FIELD_XSTAR, MGENKF_FIELD_YF, MGENKF_FIELD_T, MGENKF_FIELD_DC, MGENKF_FIELD_EPS = 0, 1, 2, 3, 4
MGENKF_FIELD_GAMMA = 5
MGENKF_FIELD_RATE = 6
MGENKF_FIELD_GAMMA_NORM = 7
EPS_TAG = 0x45505300


class MGEnKFError(RuntimeError):
    def __init__(self, status: int, where: str, text: str):
        self.status = status
        super().__init__(f"{where}: MGENKF_ERR_{STATUS_NAMES.get(status, status)}: {text}")


class mgenkf_config(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("n_fine", ctypes.c_int32), ("ratio", ctypes.c_int32),
                ("n_members", ctypes.c_int32), ("n_obs", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("gain_form", ctypes.c_int32),
                ("prolong", ctypes.c_int32), ("length", ctypes.c_double), ("dt", ctypes.c_double),
                ("nu", ctypes.c_double), ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double),
                ("obs_sigma", ctypes.c_double), ("seed", ctypes.c_uint64)]


class mgenkf_dual_config(ctypes.Structure):
    _fields_ = [("n_fine", ctypes.c_int32), ("ratio", ctypes.c_int32), ("n_members", ctypes.c_int32),
                ("n_obs", ctypes.c_int32), ("length", ctypes.c_double), ("dt", ctypes.c_double),
                ("nu", ctypes.c_double), ("u0", ctypes.c_double), ("omega", ctypes.c_double),
                ("obs_sigma", ctypes.c_double), ("theta_q", ctypes.c_double), ("seed", ctypes.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2012_10091_gb300.build` (there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                 ctypes.c_double, ctypes.c_size_t)
    sigs = {
        "mgenkf_create": [ctypes.POINTER(mgenkf_config), P, P, P, ctypes.POINTER(P)],
        "mgenkf_set_state": [P, P, P],
        "mgenkf_forecast": [P, i32],
        "mgenkf_forecast_autotune": [P, i32],
        "mgenkf_get_forecast_choice": [P, P, P],
        "mgenkf_set_forecast_choice": [P, i32, i32],
        "mgenkf_analyse": [P, P, P],
        "mgenkf_prolong_correct": [P],
        "mgenkf_cycle": [P, i32, P, P, P],
        "mgenkf_get_state": [P, P, P],
        "mgenkf_rmse": [P, P, P],
        "mgenkf_get_field": [P, i32, P, sz],
        "mgenkf_sync": [P],
        "mgenkf_save": [P, ctypes.c_char_p],
        "mgenkf_load": [P, ctypes.c_char_p],
        "mgenkf_destroy": [P],
        "mgk_forecast": [i32, i32, P, i32, i32, f64, f64, f64, f64, f64, i32, P],
        "mgk_normals": [u64, u64, u64, i64, P, P],
        "mgk_gain_ensemble_noalloc": [P, P, i32, i32, f64, P, P, P],
        "mgk_fma_probe": [i32, i32, P, ctypes.POINTER(f64), P],
        "mgk_cnn_create": [i32, i32, ctypes.POINTER(P)],
        "mgk_cnn_destroy": [P],
        "mgk_cnn_set_params": [P, P, P],
        "mgk_cnn_get_params": [P, P, P],
        "mgk_cnn_forward": [P, P, P, i32, P, i32, P],
        "mgk_cnn_loss_grad": [P, P, P, P, i32, P, P],
        "mgk_cnn_adam_step": [P, ctypes.c_float, P],
        "mgk_cnn_coarse_size": [P],
        "mgenkf_set_prolong_cnn": [P, P],
        "mgenkf_set_regularisation": [P, f64],
        "mgenkf_set_recentre": [P, i32],
        "mgenkf_set_wait_limit": [P, ctypes.c_int64],
        "mgenkf_set_filter": [P, f64],
        "mgenkf_batch_create": [P, i32, P, ctypes.POINTER(P)],
        "mgenkf_batch_cycle": [P, i32, P, P],
        "mgenkf_batch_forecast": [P, i32],
        "mgenkf_batch_sync": [P],
        "mgenkf_batch_autotune": [P, i32],
        "mgenkf_batch_tiles": [P, P, P, i32, P],
        "mgenkf_batch_set_tiles": [P, P, P, i32],
        "mgenkf_batch_destroy": [P],
        "mgenkf_dual_create": [ctypes.POINTER(mgenkf_dual_config), P, P, ctypes.POINTER(P)],
        "mgenkf_dual_set_state": [P, P, P, P, P, f64],
        "mgenkf_dual_free_run": [P, i32],
        "mgenkf_dual_cycle": [P, i32, P],
        "mgenkf_dual_get_state": [P, P, P, P, P],
        "mgenkf_dual_destroy": [P],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.mgenkf_last_error.argtypes = [P]
    L.mgenkf_last_error.restype = ctypes.c_char_p
    L.mgenkf_dual_last_error.argtypes = [P]
    L.mgenkf_dual_last_error.restype = ctypes.c_char_p
    L.mgenkf_batch_last_error.argtypes = [P]
    L.mgenkf_batch_last_error.restype = ctypes.c_char_p
    L.mgk_kernel_launches.argtypes = []
    L.mgk_kernel_launches.restype = ctypes.c_uint64
    L.mgk_last_error.argtypes = []
    L.mgk_last_error.restype = ctypes.c_char_p
    L.mgk_fma_probe_threads.argtypes = []
    L.mgk_fma_probe_threads.restype = ctypes.c_int32
    return L


lib = _load()


def _ptr(x):
    """Raw address of a numpy array, a tensor-like object, an int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _as_f64(x):
    if x is None or hasattr(x, "data_ptr"):
        return x
    return np.ascontiguousarray(x, dtype=np.float64)


def _check(st, where, h=None):
    if st != MGENKF_OK:
        text = (lib.mgenkf_last_error(h) if h else lib.mgk_last_error()) or b""
        raise MGEnKFError(st, where, text.decode())


# ---------------------------------------------------------------------------
# entry points, same names as the C ABI
# ---------------------------------------------------------------------------
def mgenkf_create(cfg: mgenkf_config, obs_index, obs_var, stream=None):
    oi = np.ascontiguousarray(obs_index, dtype=np.int32)
    ov = np.ascontiguousarray(obs_var, dtype=np.int32)
    h = ctypes.c_void_p()
    st = lib.mgenkf_create(ctypes.byref(cfg), oi.ctypes.data, ov.ctypes.data, stream, ctypes.byref(h))
    _check(st, "mgenkf_create")
    return h.value


def mgenkf_set_state(h, fine, members):
    fine, members = _as_f64(fine), _as_f64(members)
    _check(lib.mgenkf_set_state(h, _ptr(fine), _ptr(members)), "mgenkf_set_state", h)


def mgenkf_forecast(h, nsteps: int):
    _check(lib.mgenkf_forecast(h, nsteps), "mgenkf_forecast", h)


def mgenkf_analyse(h, y_obs, eps=None):
    y_obs, eps = _as_f64(y_obs), _as_f64(eps)
    _check(lib.mgenkf_analyse(h, _ptr(y_obs), _ptr(eps)), "mgenkf_analyse", h)


def mgenkf_prolong_correct(h):
    _check(lib.mgenkf_prolong_correct(h), "mgenkf_prolong_correct", h)


def mgenkf_cycle(h, nsteps, y_obs, truth_fine=None, rmse_out=None):
    y_obs, truth_fine = _as_f64(y_obs), _as_f64(truth_fine)
    _check(lib.mgenkf_cycle(h, nsteps, _ptr(y_obs), _ptr(truth_fine), _ptr(rmse_out)),
           "mgenkf_cycle", h)


def mgenkf_get_state(h, fine_out=None, members_out=None):
    _check(lib.mgenkf_get_state(h, _ptr(fine_out), _ptr(members_out)), "mgenkf_get_state", h)


def mgenkf_rmse(h, truth_fine, out):
    truth_fine = _as_f64(truth_fine)
    _check(lib.mgenkf_rmse(h, _ptr(truth_fine), _ptr(out)), "mgenkf_rmse", h)


def mgenkf_get_field(h, field: int, out, count: int):
    _check(lib.mgenkf_get_field(h, field, _ptr(out), count), "mgenkf_get_field", h)


def mgenkf_sync(h) -> int:
    """Returns the device-side status (0 = OK); does not raise for NOT_SPD/NONFINITE."""
    return lib.mgenkf_sync(h)


def mgenkf_save(h, path: str):
    _check(lib.mgenkf_save(h, path.encode()), "mgenkf_save", h)


def mgenkf_load(h, path: str):
    _check(lib.mgenkf_load(h, path.encode()), "mgenkf_load", h)


def mgenkf_last_error(h) -> str:
    return (lib.mgenkf_last_error(h) or b"").decode()


def mgenkf_destroy(h):
    _check(lib.mgenkf_destroy(h), "mgenkf_destroy")


def mgk_forecast(model, precision, state, nprob, n, length, dt, nu, gamma=1.4, prandtl=0.72,
                 nsteps=1, stream=None):
    _check(lib.mgk_forecast(model, precision, _ptr(state), nprob, n, length, dt, nu, gamma, prandtl,
                            nsteps, stream), "mgk_forecast")


def mgk_normals(seed, tag, ctr0, count, out, stream=None):
    _check(lib.mgk_normals(seed, tag, ctr0, count, _ptr(out), stream), "mgk_normals")


def mgk_fma_probe(fp64, iters, sink, stream=None) -> float:
    """Launch the FMA throughput probe; returns the launch's flop count."""
    fl = ctypes.c_double()
    _check(lib.mgk_fma_probe(int(bool(fp64)), iters, _ptr(sink), ctypes.byref(fl), stream), "mgk_fma_probe")
    return fl.value


def mgk_fma_probe_threads() -> int:
    return int(lib.mgk_fma_probe_threads())


def mgk_gain_ensemble_noalloc(Y, Z, n_members, n_obs, obs_sigma, T, info=None, stream=None):
    """Y, Z, T: contiguous float64 CUDA tensors of at least n_members*n_obs,
    (n_members+1)*n_obs and (n_members+1)*n_members elements; info: optional
    int32 CUDA tensor.  The library reads and writes exactly those counts."""
    import torch
    need = {"Y": (Y, torch.float64, n_members * n_obs), "Z": (Z, torch.float64, (n_members + 1) * n_obs),
            "T": (T, torch.float64, (n_members + 1) * n_members)}
    if info is not None:
        need["info"] = (info, torch.int32, 1)
    for name, (t, dt, count) in need.items():
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise MGEnKFError(1, "mgk_gain_ensemble_noalloc", f"{name} must be a contiguous {dt} CUDA tensor")
        if t.numel() < max(count, 0):
            raise MGEnKFError(1, "mgk_gain_ensemble_noalloc", f"{name} holds {t.numel()} elements, needs {count}")
    _check(lib.mgk_gain_ensemble_noalloc(_ptr(Y), _ptr(Z), n_members, n_obs, obs_sigma, _ptr(T),
                                         _ptr(info), stream), "mgk_gain_ensemble_noalloc")


CNN_NPARAMS = 30080
CNN_SHAPES = [("W1", (32, 8, 3, 3)), ("b1", (32,)), ("W2", (32, 32, 3, 3)), ("b2", (32,)),
              ("W3", (64, 32, 3, 3)), ("b3", (64,))]


class CNN:
    """Learned correction of the prolongation (see include/mgenkf_ops.h)."""

    def __init__(self, n_coarse, batch_max=1):
        h = ctypes.c_void_p()
        _check(lib.mgk_cnn_create(n_coarse, batch_max, ctypes.byref(h)), "mgk_cnn_create")
        self.h, self.nc, self.bmax = h.value, n_coarse, batch_max

    def close(self):
        if self.h:
            lib.mgk_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params=None, stats=None):
        """params: dict of CNN_SHAPES arrays or a flat float32 vector; stats:
        (mu_in[8], s_in[8], s_out[4]) concatenated, or a dict with those keys."""
        pv = None
        if params is not None:
            if isinstance(params, dict):
                params = np.concatenate([np.asarray(params[k], np.float32).reshape(-1) for k, _ in CNN_SHAPES])
            pv = np.ascontiguousarray(params, dtype=np.float32)
            assert pv.size == CNN_NPARAMS
        sv = None
        if stats is not None:
            if isinstance(stats, dict):
                stats = np.concatenate([stats["mu_in"], stats["s_in"], stats["s_out"]])
            sv = np.ascontiguousarray(stats, dtype=np.float32)
            assert sv.size == 20
        _check(lib.mgk_cnn_set_params(self.h, _ptr(pv), _ptr(sv)), "mgk_cnn_set_params")

    def get_params(self):
        p = np.empty(CNN_NPARAMS, np.float32)
        g = np.empty(CNN_NPARAMS, np.float32)
        _check(lib.mgk_cnn_get_params(self.h, _ptr(p), _ptr(g)), "mgk_cnn_get_params")
        return p, g

    def forward(self, dC, xstar, batch, residual, accumulate=False, stream=None):
        _check(lib.mgk_cnn_forward(self.h, _ptr(dC), _ptr(xstar), batch, _ptr(residual), int(accumulate),
                                   stream), "mgk_cnn_forward")

    def loss_grad(self, dC, xstar, target, batch, loss_out=None, stream=None):
        _check(lib.mgk_cnn_loss_grad(self.h, _ptr(dC), _ptr(xstar), _ptr(target), batch, _ptr(loss_out),
                                     stream), "mgk_cnn_loss_grad")

    def adam_step(self, lr, stream=None):
        _check(lib.mgk_cnn_adam_step(self.h, lr, stream), "mgk_cnn_adam_step")


def unflatten_cnn(flat):
    out, o = {}, 0
    for k, shp in CNN_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def mgk_kernel_launches() -> int:
    return int(lib.mgk_kernel_launches())


# ---------------------------------------------------------------------------
# object wrapper over one handle
# ---------------------------------------------------------------------------
class MGEnKF:
    """One MGEnKF run on the GPU (handle owner).  See include/mgenkf.h."""

    def __init__(self, *, model, n_fine, ratio, n_members, obs_index, obs_var, length, dt, nu,
                 obs_sigma, seed=0, precision=MGENKF_FP64, gain_form=MGENKF_GAIN_ENSEMBLE,
                 gamma=1.4, prandtl=0.72, stream=None):
        self.cfg = mgenkf_config(model=model, n_fine=n_fine, ratio=ratio, n_members=n_members,
                                 n_obs=len(obs_index), precision=precision, gain_form=gain_form,
                                 prolong=MGENKF_PROLONG_LAGRANGE4, length=length, dt=dt, nu=nu,
                                 gamma=gamma, prandtl=prandtl, obs_sigma=obs_sigma, seed=seed)
        self.h = mgenkf_create(self.cfg, obs_index, obs_var, stream)
        self.dim = 1 if model == MGENKF_BURGERS1D else 2
        self.V = 1 if model == MGENKF_BURGERS1D else 4
        self.nc = n_fine // ratio
        self.nx = self.V * self.nc**self.dim
        self.nxf = self.V * n_fine**self.dim
        self.ne, self.ny = n_members, len(obs_index)

    @classmethod
    def from_workload(cls, w, gain_form=MGENKF_GAIN_ENSEMBLE, precision=None, stream=None):
        from . import workloads as W
        idx, var = W.observation_layout(w)
        prec = {"fp64": MGENKF_FP64, "mixed": MGENKF_MIXED}[precision or w.precision]
        return cls(model=MGENKF_BURGERS1D if w.model == W.BURGERS1D else MGENKF_NS2D,
                   n_fine=w.nf, ratio=w.ratio, n_members=w.ne, obs_index=idx, obs_var=var,
                   length=w.length, dt=w.dt, nu=w.nu, obs_sigma=w.sigma, seed=w.seed,
                   precision=prec, gain_form=gain_form, gamma=w.gamma, prandtl=w.prandtl,
                   stream=stream)

    def close(self):
        if self.h:
            mgenkf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, fine, members):
        mgenkf_set_state(self.h, fine, members)

    def forecast(self, nsteps):
        mgenkf_forecast(self.h, nsteps)

    def forecast_choice(self) -> tuple:
        """(members, fine run) layout of the FP32 NS-2D forecast: column-march
        choices (SEGMENT_ROWS and NARROW_BANDS decode them), or (-1, -1) for
        the 2-D tile kernel."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.mgenkf_get_forecast_choice(self.h, ctypes.byref(a), ctypes.byref(b)),
               "mgenkf_get_forecast_choice", self.h)
        return a.value, b.value

    def set_forecast_choice(self, members: int, fine: int):
        _check(lib.mgenkf_set_forecast_choice(self.h, members, fine), "mgenkf_set_forecast_choice", self.h)

    def forecast_autotune(self, reps=3) -> tuple:
        _check(lib.mgenkf_forecast_autotune(self.h, reps), "mgenkf_forecast_autotune", self.h)
        return self.forecast_choice()

    def analyse(self, y_obs, eps=None):
        mgenkf_analyse(self.h, y_obs, eps)

    def prolong_correct(self):
        mgenkf_prolong_correct(self.h)

    def cycle(self, nsteps, y_obs, truth=None, rmse_out=None):
        mgenkf_cycle(self.h, nsteps, y_obs, truth, rmse_out)

    def sync(self) -> int:
        return mgenkf_sync(self.h)

    def get_state(self):
        fine = np.empty(self.nxf)
        mem = np.empty((self.ne, self.nx))
        mgenkf_get_state(self.h, fine, mem)
        return fine, mem

    def field(self, which):
        n = {MGENKF_FIELD_XSTAR: self.nx, MGENKF_FIELD_DC: self.nx,
             MGENKF_FIELD_YF: (self.ne + 1) * self.ny, MGENKF_FIELD_T: (self.ne + 1) * self.ne,
             MGENKF_FIELD_EPS: self.ne * self.ny}[which]
        out = np.empty(n)
        mgenkf_get_field(self.h, which, out, n)
        return out

    def set_regularisation(self, alpha):
        """Final fine iteration (Algorithm 4 step 6) with relaxation alpha; alpha < 0 turns
        the recording of the previous fine state off.  See include/mgenkf.h."""
        _check(lib.mgenkf_set_regularisation(self.h, float(alpha)), "mgenkf_set_regularisation", self.h)

    def set_filter(self, sigma):
        """Centred sixth-order filter of the NS model after every model step (sigma in
        [0, 1]; 0 = off).  See include/mgenkf.h."""
        _check(lib.mgenkf_set_filter(self.h, float(sigma)), "mgenkf_set_filter", self.h)

    def set_recentre(self, on=True):
        """Re-centre the forecast ensemble on x^C* before each analysis (fine-to-coarse feedback)."""
        _check(lib.mgenkf_set_recentre(self.h, 1 if on else 0), "mgenkf_set_recentre", self.h)

    def set_wait_limit(self, cycles):
        """Bound (SM clock cycles) of the tensor-core member update's operand wait."""
        _check(lib.mgenkf_set_wait_limit(self.h, int(cycles)), "mgenkf_set_wait_limit", self.h)

    def gamma_residual(self):
        """Conservativity residual of the fine run (Eq. Conservativity_rhov), FP64."""
        out = np.empty(self.nxf)
        mgenkf_get_field(self.h, MGENKF_FIELD_GAMMA, out, self.nxf)
        return out

    def state_rate(self):
        """(x - x_prev)/dt of the fine run, FP64 (the time-derivative term of Gamma)."""
        out = np.empty(self.nxf)
        mgenkf_get_field(self.h, MGENKF_FIELD_RATE, out, self.nxf)
        return out

    def gamma_normalised(self):
        """Gamma* = Gamma / C per variable, C = max over the grid of |(x - x_prev)/dt|
        (the normalisation of the paper's conservativity maps), FP64, formed by the library."""
        out = np.empty(self.nxf)
        mgenkf_get_field(self.h, MGENKF_FIELD_GAMMA_NORM, out, self.nxf)
        return out

    def set_prolong_cnn(self, cnn):
        """Attach a CNN (or None) whose residual prolong_correct adds to Pi_F(dC)."""
        _check(lib.mgenkf_set_prolong_cnn(self.h, cnn.h if cnn is not None else None),
               "mgenkf_set_prolong_cnn", self.h)
        self._cnn = cnn

    def save(self, path):
        mgenkf_save(self.h, path)

    def load(self, path):
        mgenkf_load(self.h, path)

    def rmse(self, truth):
        out = np.empty(self.V)
        mgenkf_rmse(self.h, truth, out)
        return out


# ---------------------------------------------------------------------------
# batches of independent NS-2D problems (mgenkf_batch_* in include/mgenkf.h)
# ---------------------------------------------------------------------------
# choices of the batched forecast: rows per segment of the column march and
# whether its bands are narrow (at most 122 columns)
SEGMENT_ROWS = {c: (32, 16, 64, 128, 256, 24, 48, 20)[c % 8] for c in range(16)}
NARROW_BANDS = {c: c // 8 == 1 for c in range(16)}


def _bcheck(st, where, b):
    if st != MGENKF_OK:
        text = lib.mgenkf_batch_last_error(b) or b""
        raise MGEnKFError(st, where, text.decode())


class Batch:
    """Independent NS-2D mixed-precision MGEnKF problems cycled together: one
    CUDA graph launch per cycle.  `runs` are MGEnKF objects, which the batch
    keeps alive and which must not be used on their own while it exists."""

    def __init__(self, runs, stream=None):
        self.runs = list(runs)
        self.ny = [r.ny for r in self.runs]
        arr = (ctypes.c_void_p * len(self.runs))(*[r.h for r in self.runs])
        out = ctypes.c_void_p()
        _check(lib.mgenkf_batch_create(arr, len(self.runs), _ptr(stream), ctypes.byref(out)),
               "mgenkf_batch_create")
        self.b = out.value

    def close(self):
        if self.b:
            lib.mgenkf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cycle(self, nsteps, y_obs, innov_out=None):
        """y_obs: all problems' observations concatenated in run order (host or
        device FP64).  innov_out: optional buffer of one FP64 per problem that
        receives the RMS of the cycle's innovations y^o - H^C x^C*."""
        _bcheck(lib.mgenkf_batch_cycle(self.b, nsteps, _ptr(_as_f64(y_obs)), _ptr(innov_out)),
                "mgenkf_batch_cycle", self.b)

    def forecast(self, nsteps):
        _bcheck(lib.mgenkf_batch_forecast(self.b, nsteps), "mgenkf_batch_forecast", self.b)

    def sync(self) -> int:
        return int(lib.mgenkf_batch_sync(self.b))

    def autotune(self, reps=3):
        _bcheck(lib.mgenkf_batch_autotune(self.b, reps), "mgenkf_batch_autotune", self.b)
        return self.tiles()

    def tiles(self) -> dict:
        """{grid size: forecast choice} (SEGMENT_ROWS and NARROW_BANDS decode it)."""
        cnt = ctypes.c_int32()
        _bcheck(lib.mgenkf_batch_tiles(self.b, None, None, 0, ctypes.byref(cnt)), "mgenkf_batch_tiles", self.b)
        n = cnt.value
        sizes, shapes = (ctypes.c_int32 * n)(), (ctypes.c_int32 * n)()
        _bcheck(lib.mgenkf_batch_tiles(self.b, sizes, shapes, n, ctypes.byref(cnt)), "mgenkf_batch_tiles", self.b)
        return {int(sizes[i]): int(shapes[i]) for i in range(n)}

    def set_tiles(self, table: dict):
        n = len(table)
        sizes = (ctypes.c_int32 * n)(*[int(k) for k in table])
        shapes = (ctypes.c_int32 * n)(*[int(v) for v in table.values()])
        _bcheck(lib.mgenkf_batch_set_tiles(self.b, sizes, shapes, n), "mgenkf_batch_set_tiles", self.b)

    def save_tiles(self, path):
        """Persist the tuned table (JSON, grid size -> forecast choice) for later runs."""
        import json
        with open(path, "w") as f:
            json.dump({"tiles": {str(k): v for k, v in self.tiles().items()},
                       "segment_rows": {str(k): v for k, v in SEGMENT_ROWS.items()},
                       "narrow_bands": {str(k): v for k, v in NARROW_BANDS.items()}}, f, indent=1)

    def load_tiles(self, path):
        import json
        with open(path) as f:
            self.set_tiles({int(k): int(v) for k, v in json.load(f)["tiles"].items()})


class DualMGEnKF:
    """Dual EnKF parameter estimation on the Burgers inlet model (the
    mgenkf_dual_* entry points; see include/mgenkf.h).  FP64."""

    def __init__(self, n_fine, ratio, n_members, obs_index, length, dt, nu, obs_sigma, theta_q, seed,
                 u0=1.0, omega=2 * np.pi, stream=None):
        oi = np.ascontiguousarray(obs_index, dtype=np.int32)
        cfg = mgenkf_dual_config(n_fine, ratio, n_members, oi.size, length, dt, nu, u0, omega, obs_sigma,
                                 theta_q, seed)
        h = ctypes.c_void_p()
        st = lib.mgenkf_dual_create(ctypes.byref(cfg), oi.ctypes.data, stream, ctypes.byref(h))
        _check(st, "mgenkf_dual_create")
        self.h = h.value
        self.nf, self.nc, self.ne = n_fine, n_fine // ratio, n_members

    def _chk(self, st, where):
        if st != MGENKF_OK:
            raise MGEnKFError(st, where, (lib.mgenkf_dual_last_error(self.h) or b"").decode())

    def set_state(self, fine, members, theta, theta_fine, t0):
        f, m, th, tf = (_as_f64(a) for a in (fine, members, theta, theta_fine))
        self._chk(lib.mgenkf_dual_set_state(self.h, _ptr(f), _ptr(m), _ptr(th), _ptr(tf), float(t0)),
                  "mgenkf_dual_set_state")

    def free_run(self, nsteps):
        self._chk(lib.mgenkf_dual_free_run(self.h, int(nsteps)), "mgenkf_dual_free_run")

    def cycle(self, nsteps, y_obs):
        y = _as_f64(y_obs)
        self._chk(lib.mgenkf_dual_cycle(self.h, int(nsteps), _ptr(y)), "mgenkf_dual_cycle")

    def get_state(self):
        fine = np.empty(self.nf)
        mem = np.empty((self.ne, self.nc))
        th = np.empty((self.ne, 2))
        tf = np.empty(2)
        self._chk(lib.mgenkf_dual_get_state(self.h, _ptr(fine), _ptr(mem), _ptr(th), _ptr(tf)),
                  "mgenkf_dual_get_state")
        return fine, mem, th, tf

    def close(self):
        if self.h:
            lib.mgenkf_dual_destroy(self.h)
            self.h = None
