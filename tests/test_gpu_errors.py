"""Failure detection of the C ABI, injected on the host (bad arguments,
non-finite observations, a singular innovation matrix from R = 0): every
failure is reported as a status and leaves the run's state unchanged.
No GPU fault, trap or hang is involved."""
import numpy as np
import pytest

from paper_2012_10091_gb300 import workloads as W

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


def _handle(M, w, **kw):
    g = M.MGEnKF.from_workload(w, **kw)
    inp = W.make_inputs(w)
    g.set_state(inp["fine0"], inp["members0"])
    return g, inp


def test_invalid_configs_are_rejected(M):
    w = W.burgers_custom(256, 4, 8, 5)
    idx, var = W.observation_layout(w)
    base = dict(model=M.MGENKF_BURGERS1D, n_fine=256, ratio=4, n_members=8, obs_index=idx,
                obs_var=var, length=6.28, dt=1e-3, nu=0.01, obs_sigma=0.1)
    for bad in [dict(ratio=3), dict(n_members=1), dict(ratio=0), dict(n_fine=2 ** 17, ratio=4),
                dict(obs_sigma=0.0), dict(dt=0.0), dict(model=7)]:
        kw = {**base, **bad}
        with pytest.raises(M.MGEnKFError) as e:
            M.MGEnKF(**kw)
        assert e.value.status == 1, bad
    with pytest.raises(M.MGEnKFError):
        M.MGEnKF(**{**base, "obs_index": np.array([0, 1, 2, 3, 99999])})


def test_nonfinite_host_observation(M):
    w = W.burgers_custom(256, 4, 8, 5)
    g, inp = _handle(M, w)
    yo = np.zeros(w.ny)
    yo[2] = np.nan
    with pytest.raises(M.MGEnKFError) as e:
        g.analyse(yo)
    assert e.value.status == 5
    fine, mem = g.get_state()
    np.testing.assert_array_equal(mem, inp["members0"])


def test_nonfinite_device_observation_leaves_state_unchanged(M):
    import torch
    w = W.burgers_custom(256, 4, 8, 5)
    g, inp = _handle(M, w)
    yo = torch.zeros(w.ny, dtype=torch.float64, device="cuda")
    yo[1] = float("inf")
    g.analyse(yo)
    g.prolong_correct()
    assert g.sync() == 5
    fine, mem = g.get_state()
    np.testing.assert_array_equal(mem, inp["members0"])
    np.testing.assert_array_equal(fine, inp["fine0"])
    # the handle stays usable
    g.analyse(np.zeros(w.ny))
    assert g.sync() == 0


@pytest.mark.parametrize("nf,n_obs", [(256, 12), (256, 64), (512, 300)])
def test_singular_innovation_matrix_reported(M, nf, n_obs):
    # direct form with R = 0 and n_obs > Ne - 1: Y Y^T is singular.  The three
    # sizes take the three Cholesky paths: one CTA with the matrix in shared
    # memory, the 8-CTA cluster (32 <= n <= 256), one CTA on global memory.
    w = W.burgers_custom(nf, 1, 4, n_obs, sigma=0.0)
    g, inp = _handle(M, w, gain_form=M.MGENKF_GAIN_DIRECT)
    g.analyse(np.ones(w.ny), np.zeros((w.ne, w.ny)))
    g.prolong_correct()
    assert g.sync() == 4
    fine, mem = g.get_state()
    np.testing.assert_array_equal(mem, inp["members0"])
    np.testing.assert_array_equal(fine, inp["fine0"])


def test_misaligned_fp32_ns_state_is_rejected(M):
    """The FP32 NS-2D forecast copies its halo in 16-byte chunks: a state that
    does not start on a 16-byte boundary is refused on the host, before any
    launch, and an aligned one advances."""
    import torch
    n = 16
    buf = torch.ones(4 * n * n + 4, dtype=torch.float32, device="cuda")
    buf[3 * n * n + 1:] = 10.0
    with pytest.raises(M.MGEnKFError) as e:
        M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_MIXED, buf.data_ptr() + 4, 1, n, 1.0, 1e-4, 1e-3, 1.4, 0.72,
                       nsteps=1)
    assert "16-byte" in str(e.value)
    x = buf[:4 * n * n].clone()
    x[3 * n * n:] = 10.0
    M.mgk_forecast(M.MGENKF_NS2D, M.MGENKF_MIXED, x, 1, n, 1.0, 1e-4, 1e-3, 1.4, 0.72, nsteps=1)
    torch.cuda.synchronize()
    assert torch.allclose(x[3 * n * n:], torch.full_like(x[3 * n * n:], 10.0))


def test_tensor_core_wait_that_runs_out_is_reported(M):
    """The member update's operand wait is bounded.  With its bound set to 0
    cycles the wait runs out at the first poll (the copy it waits for was just
    issued): the kernel records MGENKF_ERR_TIMEOUT, issues no tensor-core work,
    lets its own copies land, frees its tensor memory and returns; the members
    and the fine run are unchanged and the next analysis with the default
    bound succeeds.  No GPU fault or hang is involved."""
    w = W.burgers_custom(1024, 4, 32, 64, obs_kind="random", precision="mixed")
    g, inp = _handle(M, w, precision="mixed")
    f0, m0 = g.get_state()
    rng = np.random.default_rng(5)
    yo = rng.standard_normal(w.ny) * 0.3
    g.set_wait_limit(0)
    g.analyse(yo)
    g.prolong_correct()
    assert g.sync() == 7  # MGENKF_ERR_TIMEOUT
    f1, m1 = g.get_state()
    np.testing.assert_array_equal(f1, f0)
    np.testing.assert_array_equal(m1, m0)
    g.set_wait_limit(2_000_000_000)
    g.analyse(yo)
    g.prolong_correct()
    assert g.sync() == 0
    f2, m2 = g.get_state()
    assert np.max(np.abs(m2 - m0)) > 0 and np.max(np.abs(f2 - f0)) > 0
    with pytest.raises(M.MGEnKFError):
        g.set_wait_limit(-1)
    g.close()
