"""GPU parity of the batched model forecast (Burgers SSP-RK3) and of the
Philox normals against the CPU oracle."""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import mgenkf
    return mgenkf


def _init(nprob, n, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(n) * 2 * math.pi / n
    return np.stack([0.8 * np.sin(x + rng.uniform(0, 6)) + 0.05 * rng.standard_normal(n)
                     for _ in range(nprob)])


# whole-CTA grids (<= 4096) incl. ragged thread tails, and cluster-split grids
@pytest.mark.parametrize("n,nprob", [(4, 3), (64, 32), (100, 5), (256, 2), (1000, 3), (4095, 2),
                                     (4096, 4), (5000, 2), (16384, 1), (32768, 1)])
def test_burgers_fp64_matches_oracle(M, n, nprob):
    import torch
    u0 = _init(nprob, n, n)
    dx, nu = 2 * math.pi / n, 0.01
    dt = min(1e-3, 0.3 * dx * dx / nu, 0.5 * dx)
    steps = 37
    ref = O.burgers_rk3(u0, dx, nu, dt, steps)
    d = torch.tensor(u0, dtype=torch.float64, device="cuda")
    M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_FP64, d, nprob, n, 2 * math.pi, dt, nu, nsteps=steps)
    torch.cuda.synchronize()
    got = d.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,nprob", [(64, 32), (4096, 8), (16384, 1)])
def test_burgers_fp32_matches_oracle(M, n, nprob):
    import torch
    u0 = _init(nprob, n, n + 1)
    dx, nu = 2 * math.pi / n, 0.01
    dt = min(1e-3, 0.3 * dx * dx / nu)
    steps = 200
    ref = O.burgers_rk3(u0, dx, nu, dt, steps)
    d = torch.tensor(u0, dtype=torch.float32, device="cuda")
    M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_MIXED, d, nprob, n, 2 * math.pi, dt, nu, nsteps=steps)
    torch.cuda.synchronize()
    # FP32 rounding of ~1e-7 per step, accumulated over 200 steps
    assert np.max(np.abs(d.cpu().double().numpy() - ref)) <= 2e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("amp,dt", [(50.0, 2e-5), (1e-3, 1e-4), (1.0, 0.0), (1.0, 1e-16)])
def test_burgers_fp32_scaled_state_edge_cases(M, amp, dt):
    # The folded FP32 kernel carries v = a u with a = dt / (4 dx): large and
    # small states and a step so small that a falls below 2^-40 (the generic
    # kernel takes over) match the oracle; dt = 0 is refused before any launch.
    import torch
    n, nprob = 4096, 3
    u0 = amp * _init(nprob, n, 11)
    dx, nu = 2 * math.pi / n, 0.01
    steps = 50
    d = torch.tensor(u0, dtype=torch.float32, device="cuda")
    if dt == 0.0:
        with pytest.raises(M.MGEnKFError) as e:
            M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_MIXED, d, nprob, n, 2 * math.pi, dt, nu, nsteps=steps)
        assert e.value.status == 1
        torch.cuda.synchronize()
        np.testing.assert_array_equal(d.cpu().double().numpy(), u0.astype(np.float32).astype(np.float64))
        return
    ref = O.burgers_rk3(u0, dx, nu, dt, steps)
    M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_MIXED, d, nprob, n, 2 * math.pi, dt, nu, nsteps=steps)
    torch.cuda.synchronize()
    got = d.cpu().double().numpy()
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_burgers_zero_steps_and_empty_batch(M):
    import torch
    u0 = _init(2, 128, 3)
    d = torch.tensor(u0, dtype=torch.float64, device="cuda")
    M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_FP64, d, 2, 128, 2 * math.pi, 1e-3, 0.01, nsteps=0)
    M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_FP64, d, 0, 128, 2 * math.pi, 1e-3, 0.01, nsteps=5)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy(), u0)


def test_burgers_rejects_oversize_grid(M):
    import torch
    d = torch.zeros(65536, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MGEnKFError) as e:
        M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_FP64, d, 1, 65536, 1.0, 1e-3, 0.01, nsteps=1)
    assert e.value.status == 1


@pytest.mark.parametrize("count,ctr0", [(1, 0), (4, 7), (1023, 3), (100_000, 11)])
def test_philox_normals_match_oracle(M, count, ctr0):
    import torch
    out = torch.empty(count, dtype=torch.float64, device="cuda")
    M.mgk_normals(5, M.EPS_TAG, ctr0, count, out)
    torch.cuda.synchronize()
    ref = O.normals(5, M.EPS_TAG, ctr0, count)
    # same Philox words bit for bit; log/cos/sin may differ by a few ulp between libms
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-14, atol=1e-14)


def test_fp32_forecast_has_no_drift_over_long_horizon(M):
    # fine grid of the large Burgers workload over two observation intervals
    # (8662 steps, dt L ~ one FP32 ulp of u per step): the compensated FP32
    # state stays within the random-walk rounding bound of the FP64 oracle,
    # sqrt(3 * nsteps) * 2^-24 ~ 1e-5 relative; a biased update would drift far
    # beyond it.
    import torch
    from paper_2012_10091_gb300 import workloads as W
    w = W.burgers_large()
    u0 = W.initial_truth(w)
    steps = 2 * w.steps_per_cycle
    ref = O.burgers_rk3(u0, w.length / w.nf, w.nu, w.dt, steps)
    d = torch.tensor(u0, dtype=torch.float32, device="cuda")
    M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_MIXED, d, 1, w.nf, w.length, w.dt, w.nu, nsteps=steps)
    torch.cuda.synchronize()
    err = np.max(np.abs(d.cpu().double().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 1e-5, err


@pytest.mark.parametrize("nf", [8192, 16384, 32768])
def test_split_grid_halo_exchange_paths_agree(M, nf):
    # A handle's mixed forecast advances its split fine grid (a cluster of
    # CTAs exchanging halos over distributed shared memory) in one launch with
    # the members; the stateless forecast advances it alone.  Same arithmetic
    # on every segment: the same bits.
    import torch
    from paper_2012_10091_gb300 import workloads as W
    w = W.burgers_custom(nf, 8 if nf > 16384 else 4, 8, 16, precision="mixed",
                         dt=0.3 * (2 * math.pi / nf) ** 2 / 0.01)
    inp = W.make_inputs(w)
    g = M.MGEnKF.from_workload(w, precision="mixed")
    g.set_state(inp["fine0"], inp["members0"])
    g.forecast(300)
    assert g.sync() == 0
    fine, _ = g.get_state()
    d = torch.tensor(inp["fine0"], dtype=torch.float32, device="cuda")
    M.mgk_forecast(M.MGENKF_BURGERS1D, M.MGENKF_MIXED, d, 1, nf, w.length, w.dt, w.nu, nsteps=300)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fine.astype(np.float32), d.cpu().numpy())
    g.close()
