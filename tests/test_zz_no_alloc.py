"""The allocation-free gain solve (mgk_gain_ensemble_noalloc) gives the same
gain coefficients T as the handle's analysis.

Some callers of this library cannot call cudaMalloc (their own pool owns all
device memory, or they run under a fixed memory budget); this entry point
serves them with a fixed scratch array inside the library.  The test feeds it
the observation anomalies Y and innovations Z of one analysis of the existing
entry point (mgenkf_analyse, ensemble-space form, FP64) and compares the two T
on two calls in a row, so that a stale status word or leftover scratch from
the first call would show up in the second.  The member counts cover the
smallest ensemble, the one-CTA Cholesky and the largest size the scratch holds
(the clustered Cholesky and the largest shared-memory solve).  This file sorts
last so that a run stopping at its first failure has already run every other
test."""
import ctypes
import math

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


@pytest.mark.parametrize("ne", [2, 16, 96, 128])
def test_noalloc_gain_matches_handle_analysis_twice(M, ne):
    import torch
    w = W.burgers_custom(512, 4, ne, 70, obs_kind="random", sigma=0.07)
    inp = W.make_inputs(w)
    g = M.MGEnKF.from_workload(w, gain_form=M.MGENKF_GAIN_ENSEMBLE, precision="fp64")
    g.set_state(inp["fine0"], inp["members0"])
    rng = np.random.default_rng(3 + ne)
    yo = rng.standard_normal(w.ny) * 0.3
    eps = w.sigma * rng.standard_normal((w.ne, w.ny))
    g.analyse(yo, eps)
    assert g.sync() == 0
    yf = g.field(M.MGENKF_FIELD_YF).reshape(w.ne + 1, w.ny)
    T_ref = g.field(M.MGENKF_FIELD_T).reshape(w.ne + 1, w.ne)
    g.close()
    # observation anomalies and innovations of that analysis (Algorithm 3 step 7)
    Y = (yf[:w.ne] - yf[:w.ne].mean(0)) / math.sqrt(w.ne - 1)
    Z = np.vstack([yo + eps - yf[:w.ne], yo - yf[w.ne]])
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    Zd = torch.tensor(Z, dtype=torch.float64, device="cuda")
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        T = torch.full((w.ne + 1, w.ne), float("nan"), dtype=torch.float64, device="cuda")
        M.mgk_gain_ensemble_noalloc(Yd, Zd, w.ne, w.ny, w.sigma, T, info)
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        got = T.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - T_ref)) <= 1e-10 * np.max(np.abs(T_ref))


def test_noalloc_gain_rejects_sizes_beyond_its_scratch(M):
    import torch
    Y = torch.zeros((129, 4), dtype=torch.float64, device="cuda")
    Z = torch.zeros((130, 4), dtype=torch.float64, device="cuda")
    T = torch.zeros((130, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(M.MGEnKFError) as e:
        M.mgk_gain_ensemble_noalloc(Y, Z, 129, 4, 0.1, T)
    assert e.value.status == 1 and "128" in str(e.value)


def test_noalloc_gain_rejects_host_and_short_buffers(M):
    import torch
    ne, ny = 8, 5
    Y = torch.zeros((ne, ny), dtype=torch.float64, device="cuda")
    Z = torch.zeros((ne + 1, ny), dtype=torch.float64, device="cuda")
    T = torch.zeros((ne + 1, ne), dtype=torch.float64, device="cuda")
    # the binding refuses wrong dtypes, host tensors and short buffers
    for bad in (Y.float(), Y.cpu(), Y[:, :2].contiguous()):
        with pytest.raises(M.MGEnKFError) as e:
            M.mgk_gain_ensemble_noalloc(bad, Z, ne, ny, 0.1, T)
        assert e.value.status == 1
    # the C entry point itself refuses host memory before launching anything
    host = np.zeros((ne + 1) * ny)
    st = M.lib.mgk_gain_ensemble_noalloc(ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(Z.data_ptr()),
                                         ne, ny, 0.1, ctypes.c_void_p(T.data_ptr()), None, None)
    assert st == 1 and b"device memory" in M.lib.mgk_last_error()
    # and still works afterwards
    M.mgk_gain_ensemble_noalloc(Y, Z, ne, ny, 0.1, T)
    torch.cuda.synchronize()
