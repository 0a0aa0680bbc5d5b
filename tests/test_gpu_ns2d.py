"""GPU parity of the 2-D compressible Navier-Stokes forecast (Eqs. Mass,
Momentum, Energy; SSP-RK3) against the CPU oracle, and of a short MGEnKF run
on the shear-layer workload through the C ABI."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import gpu_run, oracle_run, rel_err
from paper_2012_10091_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GAMMA, PR = 1.4, 0.72


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import mgenkf
    return mgenkf


def _smooth_states(nprob, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    x = np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    for _ in range(nprob):
        rho = 1.0 + 0.1 * np.sin(2 * np.pi * X + rng.uniform(0, 6)) * np.cos(2 * np.pi * Y)
        u = 0.3 * np.sin(2 * np.pi * Y + rng.uniform(0, 6)) + 0.01 * rng.standard_normal((n, n))
        v = 0.2 * np.cos(2 * np.pi * X) + 0.01 * rng.standard_normal((n, n))
        p = 8.0 + 0.2 * np.cos(2 * np.pi * (X + Y))
        E = p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)
        out.append(np.stack([rho, rho * u, rho * v, E]))
    return np.stack(out)


@pytest.mark.parametrize("n,nprob", [(8, 3), (16, 2), (40, 2), (64, 1), (136, 1)])
def test_ns2d_fp64_matches_oracle(M, n, nprob):
    import torch
    q0 = _smooth_states(nprob, n, n)
    # dt within the acoustic (CFL 0.2) and heat-conduction (kappa dt / h^2 <= 0.1) limits
    h, mu, steps = 1.0 / n, 1e-2, 12
    dt = min(0.2 * h, 0.1 * h * h * (GAMMA - 1) * PR / (mu * GAMMA) * 2)
    ref = O.ns2d_rk3(q0, h, GAMMA, mu, PR, dt, steps)
    d = torch.tensor(q0, dtype=torch.float64, device="cuda")
    M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_FP64, d, nprob, n, 1.0, dt, mu, GAMMA, PR, nsteps=steps)
    torch.cuda.synchronize()
    got = d.cpu().numpy()
    for k in range(4):
        assert np.max(np.abs(got[:, k] - ref[:, k])) <= 1e-12 * np.max(np.abs(ref[:, k])), k
    # conservation of the four totals on the GPU path as well
    for k in range(4):
        assert abs(got[:, k].sum() - q0[:, k].sum()) <= 1e-12 * np.abs(q0[:, k]).sum()


def test_ns2d_fp32_matches_oracle(M):
    import torch
    n, nprob = 64, 2
    q0 = _smooth_states(nprob, n, 5)
    h, mu, dt, steps = 1.0 / n, 1e-3, 0.2 / n, 40
    ref = O.ns2d_rk3(q0, h, GAMMA, mu, PR, dt, steps)
    d = torch.tensor(q0, dtype=torch.float32, device="cuda")
    M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_MIXED, d, nprob, n, 1.0, dt, mu, GAMMA, PR, nsteps=steps)
    torch.cuda.synchronize()
    got = d.cpu().double().numpy()
    # FP32 rounding (2^-24) of O(10) energies over 40 steps of 3 stages
    for k in range(4):
        assert np.max(np.abs(got[:, k] - ref[:, k])) <= 2e-5 * np.max(np.abs(ref[:, k])), k


@pytest.mark.parametrize("n,nprob", [(264, 16), (1064, 1)])
def test_ns2d_fp32_multi_tile_matches_oracle(M, n, nprob):
    # The stateless forecast runs the column march.  16 x 264^2: one band of
    # 132 threads per grid, 9 row segments of 32 rows (the last one 8 rows),
    # 144 CTAs.  1064^2: 3 bands of 356, 356 and 352 columns with 3-column
    # halos (the last band ragged), 67 segments of 16 rows (the last 8).
    import torch
    q0 = _smooth_states(nprob, n, 11)
    h, mu, steps = 1.0 / n, 1e-3, 10
    dt = min(0.2 * h, 0.1 * h * h * (GAMMA - 1) * PR / (mu * GAMMA) * 2)
    ref = O.ns2d_rk3(q0, h, GAMMA, mu, PR, dt, steps)
    d = torch.tensor(q0, dtype=torch.float32, device="cuda")
    M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_MIXED, d, nprob, n, 1.0, dt, mu, GAMMA, PR, nsteps=steps)
    torch.cuda.synchronize()
    got = d.cpu().double().numpy()
    # element-wise, each plane against its own maximum: FP32 rounding of O(10)
    # energies over 10 steps of 3 stages
    for k in range(4):
        assert np.max(np.abs(got[:, k] - ref[:, k])) <= 2e-5 * np.max(np.abs(ref[:, k])), k
    # an odd step count ends in the state buffer as well
    d = torch.tensor(q0, dtype=torch.float32, device="cuda")
    M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_MIXED, d, nprob, n, 1.0, dt, mu, GAMMA, PR, nsteps=3)
    torch.cuda.synchronize()
    ref3 = O.ns2d_rk3(q0, h, GAMMA, mu, PR, dt, 3)
    got3 = d.cpu().double().numpy()
    for k in range(4):
        assert np.max(np.abs(got3[:, k] - ref3[:, k])) <= 1e-5 * np.max(np.abs(ref3[:, k])), k


@pytest.mark.parametrize("steps,kernel", [(10, "march"), (3, "march"), (10, "tile"), (3, "tile")])
def test_ns2d_handle_forecast_at_full_size_matches_oracle(M, steps, kernel):
    # A handle of the 512^2 / 128^2, 64-member workload advances its members
    # and fine run with the column march (its default choice: the members and
    # the fine run on two streams; an odd step count ends with a copy back) or
    # with the tile kernel: 64 x 16 + 256 = 1280 tiles of 32 x 32 points over
    # 2 x 152 resident CTAs (4.2 tiles per CTA).
    w = W.ns2d_shear(nf=512, ratio=4, ne=64, n_probes=1024, cycles=1, precision="mixed")
    inp = W.make_inputs(w)
    g = M.MGEnKF.from_workload(w, precision="mixed")
    if kernel == "tile":
        g.set_forecast_choice(-1, -1)
    else:
        assert min(g.forecast_choice()) >= 0
    g.set_state(inp["fine0"], inp["members0"])
    g.forecast(steps)
    assert g.sync() == 0
    fine, mem = g.get_state()
    g.close()
    h_f, h_c = w.length / w.nf, w.length / w.nc
    ref_f = O.ns2d_rk3(inp["fine0"].reshape(4, w.nf, w.nf), h_f, w.gamma, w.nu, w.prandtl, w.dt, steps)
    ref_m = O.ns2d_rk3(inp["members0"].reshape(w.ne, 4, w.nc, w.nc), h_c, w.gamma, w.nu, w.prandtl, w.dt, steps)
    got_f = fine.reshape(4, w.nf, w.nf)
    got_m = mem.reshape(w.ne, 4, w.nc, w.nc)
    # Element-wise.  The FP32 rounding of a momentum plane is set by its fluxes
    # (rho u u + p, rho u v), not by the plane itself: in the shear layer
    # |rho v| <= 1e-3 while |rho u| ~ 1, so both momentum planes are measured
    # against the larger momentum; rho and E against themselves.
    for got, ref in ((got_f, ref_f), (got_m, ref_m)):
        mom = max(np.max(np.abs(ref[..., 1, :, :])), np.max(np.abs(ref[..., 2, :, :])))
        for k in range(4):
            scale = mom if k in (1, 2) else np.max(np.abs(ref[..., k, :, :]))
            assert np.max(np.abs(got[..., k, :, :] - ref[..., k, :, :])) <= 2e-5 * scale, k


def _choice_handle(M):
    # fine 544^2 (two whole-width bands, five narrow ones), coarse 136^2 (one
    # whole-width band, two narrow ones): ragged bands and segments everywhere
    w = W.ns2d_shear(nf=544, ratio=4, ne=6, n_probes=64, cycles=1, precision="mixed")
    inp = W.make_inputs(w)
    return w, inp, M.MGEnKF.from_workload(w, precision="mixed")


def _advance(g, inp, steps):
    g.set_state(inp["fine0"], inp["members0"])
    g.forecast(steps)
    assert g.sync() == 0
    return g.get_state()


@pytest.mark.parametrize("steps", [2, 3])
def test_ns2d_handle_forecast_choices_are_bit_exact(M, steps):
    """Every layout of a handle's FP32 forecast (the tile kernel, each column
    march choice per grid) runs the same per-point arithmetic: bit-equal
    states after an even and an odd number of steps."""
    w, inp, g = _choice_handle(M)
    default = g.forecast_choice()
    assert all(c in M.SEGMENT_ROWS for c in default)
    ref_f, ref_m = _advance(g, inp, steps)
    g.set_forecast_choice(-1, -1)
    assert g.forecast_choice() == (-1, -1)
    tf, tm = _advance(g, inp, steps)
    np.testing.assert_array_equal(tf, ref_f)
    np.testing.assert_array_equal(tm, ref_m)
    n = len(M.SEGMENT_ROWS)
    for c in range(n):
        g.set_forecast_choice(c, (c + 3) % n)
        f, m = _advance(g, inp, steps)
        np.testing.assert_array_equal(f, ref_f)
        np.testing.assert_array_equal(m, ref_m)
    g.close()


def test_ns2d_forecast_autotune_and_choice_checks(M):
    w, inp, g = _choice_handle(M)
    ref_f, ref_m = _advance(g, inp, 3)
    got = g.forecast_autotune(reps=1)
    assert all(c in M.SEGMENT_ROWS for c in got) and g.forecast_choice() == got
    f, m = _advance(g, inp, 3)
    np.testing.assert_array_equal(f, ref_f)
    np.testing.assert_array_equal(m, ref_m)
    for bad in ((-1, 0), (0, -1), (len(M.SEGMENT_ROWS), 0), (0, -2)):
        with pytest.raises(M.MGEnKFError):
            g.set_forecast_choice(*bad)
    assert g.forecast_choice() == got
    g.close()
    # FP64 handles have one forecast kernel: nothing to choose
    w64 = W.ns2d_shear(nf=64, ratio=4, ne=4, n_probes=8, cycles=1, precision="fp64")
    g64 = M.MGEnKF.from_workload(w64)
    assert g64.forecast_autotune(reps=1) == (-1, -1)
    with pytest.raises(M.MGEnKFError):
        g64.set_forecast_choice(0, 0)
    g64.close()


def test_ns2d_rejects_bad_sizes(M):
    import torch
    d = torch.zeros(4 * 12 * 12, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MGEnKFError):
        M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_FP64, d, 1, 12, 1.0, 1e-3, 1e-3, GAMMA, PR, nsteps=1)


@pytest.mark.parametrize("gain_form", [0, 1])
def test_ns2d_mgenkf_cycles_match_oracle(M, gain_form):
    w = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=3, precision="fp64", delta=0.08)
    mg, rm_o, _ = oracle_run(w, w.cycles)
    g, rm_g, _ = gpu_run(w, w.cycles, gain_form=gain_form)
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-10
    assert rel_err(mem, mg.members) < 1e-10
    np.testing.assert_allclose(rm_g, rm_o, rtol=1e-8)
    g.close()


def test_ns2d_mixed_cycles_close_to_oracle(M):
    w = W.ns2d_shear(nf=64, ratio=4, ne=12, n_probes=20, cycles=3, precision="mixed", delta=0.08)
    mg, rm_o, _ = oracle_run(w, w.cycles)
    g, rm_g, _ = gpu_run(w, w.cycles)
    fine, mem = g.get_state()
    assert rel_err(fine, mg.fine) < 1e-3
    assert rel_err(mem, mg.members) < 1e-3
    g.close()
