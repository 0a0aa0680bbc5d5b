"""Seeded synthetic workloads of the MGEnKF analysis cycle.

This module holds the input recipes only: grid sizes, time steps, initial
conditions, observation positions and observation noise, all drawn from
numpy generators seeded per stream.  It contains none of the method's
arithmetic (no model step, projector, observation operator or filter), so
both the GPU path and the CPU oracle may take their inputs from it.

The paper's experiments use self-generated truth simulations (Sec. 4, Sec. 6);
the workloads below keep that structure: a truth run, a fine model run started
from a perturbed initial state, Ne coarse members with their own perturbations,
and point observations of the truth with Gaussian noise (Eq. z_mdl).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

BURGERS1D = "burgers1d"
NS2D = "ns2d"

# stream identifiers of the seeded generators
_S_TRUTH, _S_MODEL, _S_MEMBERS, _S_OBSPOS, _S_OBSNOISE, _S_PHASE, _S_BATCH = 1, 2, 3, 4, 5, 6, 7


def _rng(seed: int, stream: int, *extra: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([seed, stream, *extra]))


@dataclass
class Workload:
    name: str
    model: str
    nf: int                 # fine points per side
    ratio: int              # coarsening ratio r_C
    ne: int                 # ensemble members
    n_probes: int           # observed fine nodes
    sigma: float            # observation noise std (R = sigma^2 I)
    steps_per_cycle: int    # model steps between analyses
    cycles: int
    dt: float
    length: float
    nu: float               # Burgers viscosity, or mu = 1/Re for NS
    precision: str          # "fp64" or "mixed"
    seed: int = 0
    gamma: float = 1.4
    prandtl: float = 0.72
    mach: float = 0.3
    truth_kind: str = "sin"
    obs_kind: str = "equispaced"
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return 1 if self.model == BURGERS1D else 2

    @property
    def V(self) -> int:
        return 1 if self.model == BURGERS1D else 4

    @property
    def nc(self) -> int:
        return self.nf // self.ratio

    @property
    def nx(self) -> int:
        return self.V * self.nc**self.dim

    @property
    def nxf(self) -> int:
        return self.V * self.nf**self.dim

    @property
    def ny(self) -> int:
        return self.n_probes * (1 if self.model == BURGERS1D else 2)

    def member_steps_per_cycle(self) -> int:
        return self.ne * self.steps_per_cycle


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def burgers_small(seed: int = 0) -> Workload:
    """1-D viscous Burgers, periodic [0, 2 pi], fine 256 / coarse 64, FP64,
    dt = 1e-3, Ne = 32, 16 equispaced observations every 20 steps, sigma 0.05,
    50 cycles; truth u0 = sin x, model u0 = A sin x + 0.05 N(0,1), A ~ N(0.8, 0.1^2)."""
    return Workload("burgers_256_64_ne32_fp64", BURGERS1D, nf=256, ratio=4, ne=32, n_probes=16,
                    sigma=0.05, steps_per_cycle=20, cycles=50, dt=1e-3, length=2 * math.pi,
                    nu=0.01, precision="fp64", seed=seed, truth_kind="sin", obs_kind="equispaced")


def burgers_large(seed: int = 0, precision: str = "mixed") -> Workload:
    """1-D viscous Burgers, fine 16384 / coarse 4096, Ne = 128, 512 random
    observation points, sigma 0.02, 200 cycles; truth = sum_k k^-1 sin(kx + phi_k).
    One dt for both grids, set by fine-grid RK3 diffusion stability at half
    the limit, over an observation interval of 0.02."""
    nf, nu, t_obs = 16384, 0.01, 0.02
    dx = 2 * math.pi / nf
    dt_lim = 0.5 * 0.628 * dx * dx / nu
    steps = math.ceil(t_obs / dt_lim)
    return Workload("burgers_16384_4096_ne128_" + precision, BURGERS1D, nf=nf, ratio=4, ne=128,
                    n_probes=512, sigma=0.02, steps_per_cycle=steps, cycles=200, dt=t_obs / steps,
                    length=2 * math.pi, nu=nu, precision=precision, seed=seed,
                    truth_kind="multisine", obs_kind="random")


def burgers_custom(nf, ratio, ne, n_probes, steps_per_cycle=20, cycles=5, dt=1e-3, sigma=0.05,
                   precision="fp64", seed=0, obs_kind="random", truth_kind="sin") -> Workload:
    """Burgers workload of arbitrary size (parity cases: ragged sizes, r = 1)."""
    return Workload(f"burgers_{nf}_{nf // ratio}_ne{ne}_{precision}", BURGERS1D, nf=nf,
                    ratio=ratio, ne=ne, n_probes=n_probes, sigma=sigma,
                    steps_per_cycle=steps_per_cycle, cycles=cycles, dt=dt, length=2 * math.pi,
                    nu=0.01, precision=precision, seed=seed, truth_kind=truth_kind,
                    obs_kind=obs_kind)


def ns2d_shear(nf: int = 512, ratio: int = 4, ne: int = 64, n_probes: int = 1024,
               cycles: int = 100, precision: str = "mixed", seed: int = 0,
               delta: float = 0.02) -> Workload:
    """2-D compressible NS, periodic [0,1]^2, Re = 1000, Mach 0.3 double shear
    layer (thickness delta, 0.02 by default) + 1e-3 N(0,1) velocity
    perturbation, probes of (rho u, rho v) every 10 steps with sigma 0.01.
    dt: the acoustic CFL step 0.5 sqrt(3) h / (|u| + c), capped at 0.8 of the
    RK3 limit of heat conduction, 2.51 h^2 / (8 mu gamma / Pr) (the cap binds
    from about 1024 points per side)."""
    mach = 0.3
    h = 1.0 / nf
    mu, gamma, pr = 1e-3, 1.4, 0.72
    dt = min(0.5 * math.sqrt(3.0) * h / (1.0 + 1.0 / mach), 0.8 * 2.51 * h * h / (8.0 * mu * gamma / pr))
    return Workload(f"ns2d_{nf}_{nf // ratio}_ne{ne}_{precision}", NS2D, nf=nf, ratio=ratio, ne=ne,
                    n_probes=n_probes, sigma=0.01, steps_per_cycle=10, cycles=cycles, dt=dt,
                    length=1.0, nu=1e-3, precision=precision, seed=seed, mach=mach,
                    truth_kind="shear", obs_kind="random", extra={"delta": delta})


def ns2d_batch(nprob: int = 96, seed: int = 0, coarse=(64, 96, 128, 192), members=(16, 32, 64, 128),
               n_obs=(256, 2048), ratio: int = 4, cycles: int = 100) -> list:
    """Independent 2-D NS problems of uneven sizes: per problem a coarse side
    drawn uniformly from `coarse` (fine = ratio x per side), Ne from `members`,
    an even observation count drawn uniformly from [n_obs[0], n_obs[1]]
    (n_obs / 2 velocity probes), its own seed, 10 steps per cycle.  The shear
    layer is 0.02 thick from 128 coarse points per side up and 0.02 * 128 / nc
    below, so that it spans the same number of coarse cells."""
    g = _rng(seed, _S_BATCH)
    out = []
    for i in range(nprob):
        nc = int(g.choice(coarse))
        ne = int(g.choice(members))
        ny = 2 * int(g.integers(n_obs[0] // 2, n_obs[1] // 2 + 1))
        delta = 0.02 * max(1.0, 128.0 / nc)
        w = ns2d_shear(nf=ratio * nc, ratio=ratio, ne=ne, n_probes=ny // 2, cycles=cycles,
                       precision="mixed", seed=seed * 100003 + i + 1, delta=delta)
        out.append(dataclasses.replace(w, name=f"batch{i}_{w.name}"))
    return out


# --------------------------------------------------------------------------
# initial states, observation positions and noise
# --------------------------------------------------------------------------
def _burgers_profile(w: Workload, x: np.ndarray) -> np.ndarray:
    if w.truth_kind == "sin":
        return np.sin(x)
    phases = _rng(w.seed, _S_PHASE).uniform(0.0, 2 * math.pi, size=8)
    return sum(np.sin(k * x + phases[k - 1]) / k for k in range(1, 9))


def _shear_u(y: np.ndarray, delta: float = 0.02) -> np.ndarray:
    return np.tanh((y - 0.5) / delta) - np.tanh(y / delta) - np.tanh((y - 1.0) / delta)


def _ns_state(w: Workload, n: int, up: np.ndarray, vp: np.ndarray) -> np.ndarray:
    y = np.arange(n) * (w.length / n)
    u = np.broadcast_to(_shear_u(y, w.extra.get("delta", 0.02))[:, None], (n, n)) + up
    v = vp
    rho = np.ones((n, n))
    p0 = 1.0 / (w.gamma * w.mach**2)
    E = p0 / (w.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E]).reshape(-1)


def initial_truth(w: Workload) -> np.ndarray:
    """Fine-grid truth at t = 0 (FP64, V * nf^dim)."""
    if w.model == BURGERS1D:
        x = np.arange(w.nf) * (w.length / w.nf)
        return _burgers_profile(w, x).astype(np.float64)
    g = _rng(w.seed, _S_TRUTH)
    up = 1e-3 * g.standard_normal((w.nf, w.nf))
    vp = 1e-3 * g.standard_normal((w.nf, w.nf))
    return _ns_state(w, w.nf, up, vp)


def initial_fine_model(w: Workload) -> np.ndarray:
    """Fine model run at t = 0: perturbed truth recipe (FP64)."""
    g = _rng(w.seed, _S_MODEL)
    if w.model == BURGERS1D:
        x = np.arange(w.nf) * (w.length / w.nf)
        A = g.normal(0.8, 0.1)
        return A * _burgers_profile(w, x) + 0.05 * g.standard_normal(w.nf)
    up = 1e-3 * g.standard_normal((w.nf, w.nf))
    vp = 1e-3 * g.standard_normal((w.nf, w.nf))
    return _ns_state(w, w.nf, up, vp)


def initial_members(w: Workload) -> np.ndarray:
    """Ne coarse members at t = 0 (ne x V * nc^dim), each with its own draws."""
    g = _rng(w.seed, _S_MEMBERS)
    out = np.empty((w.ne, w.nx), dtype=np.float64)
    if w.model == BURGERS1D:
        xc = np.arange(w.nc) * (w.length / w.nc)
        prof = _burgers_profile(w, xc)
        for i in range(w.ne):
            A = g.normal(0.8, 0.1)
            out[i] = A * prof + 0.05 * g.standard_normal(w.nc)
        return out
    for i in range(w.ne):
        up = 1e-3 * g.standard_normal((w.nc, w.nc))
        vp = 1e-3 * g.standard_normal((w.nc, w.nc))
        out[i] = _ns_state(w, w.nc, up, vp)
    return out


def observation_layout(w: Workload):
    """(obs_idx, obs_var): flat fine-grid node and observed variable per scalar
    observation.  Burgers observes u; NS observes rho u and rho v per probe."""
    nfp = w.nf**w.dim
    if w.obs_kind == "equispaced":
        nodes = (np.arange(w.n_probes) * (nfp // w.n_probes)).astype(np.int64)
    else:
        g = _rng(w.seed, _S_OBSPOS)
        nodes = np.sort(g.choice(nfp, size=w.n_probes, replace=False))
    if w.model == BURGERS1D:
        return nodes.astype(np.int32), np.zeros(w.n_probes, dtype=np.int32)
    idx = np.repeat(nodes, 2).astype(np.int32)
    var = np.tile(np.array([1, 2], dtype=np.int32), w.n_probes)
    return idx, var


def observation_noise(w: Workload, cycle: int) -> np.ndarray:
    """N(0, sigma^2) noise added to the truth samples of one analysis."""
    return w.sigma * _rng(w.seed, _S_OBSNOISE, cycle).standard_normal(w.ny)


def sample_truth(w: Workload, truth_state: np.ndarray, obs_idx, obs_var) -> np.ndarray:
    """Pick the observed entries of a fine truth state (H^F is injection)."""
    nfp = w.nf**w.dim
    return np.asarray(truth_state, dtype=np.float64)[np.asarray(obs_var) * nfp + np.asarray(obs_idx)]


def make_inputs(w: Workload) -> dict:
    obs_idx, obs_var = observation_layout(w)
    return dict(truth0=initial_truth(w), fine0=initial_fine_model(w), members0=initial_members(w),
                obs_idx=obs_idx, obs_var=obs_var)
