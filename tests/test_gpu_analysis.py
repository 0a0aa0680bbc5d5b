"""GPU parity of the coarse-mesh EnKF analysis and the multigrid correction
(Algorithm 3 state part, Algorithm 4 steps 4-5) against the CPU oracle, step
by step, for both gain forms, FP64 and mixed precision, on ragged sizes."""
import numpy as np
import pytest

import oracle as O
from helpers import rel_err
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


CASES = [  # nf, ratio, ne, n_probes: several tiles and ragged tails
    (256, 4, 32, 16), (240, 3, 7, 11), (4096, 4, 37, 130), (1000, 8, 130, 257), (64, 1, 5, 3)]


def _one_analysis(M, w, gain_form, precision, explicit_eps):
    inp = W.make_inputs(w)
    g = M.MGEnKF.from_workload(w, gain_form=gain_form, precision=precision)
    g.set_state(inp["fine0"], inp["members0"])
    rng = np.random.default_rng(w.nf + w.ne)
    yo = rng.standard_normal(w.ny) * 0.5
    eps = w.sigma * rng.standard_normal((w.ne, w.ny)) if explicit_eps else None
    g.analyse(yo, eps)
    g.prolong_correct()
    assert g.sync() == 0
    fine, mem = g.get_state()
    fields = {k: g.field(k) for k in (M.MGENKF_FIELD_XSTAR, M.MGENKF_FIELD_YF, M.MGENKF_FIELD_T,
                                      M.MGENKF_FIELD_DC, M.MGENKF_FIELD_EPS)}
    g.close()
    # oracle on the same inputs (rounded to FP32 first in mixed precision)
    f0, m0 = inp["fine0"], inp["members0"]
    if precision == "mixed":
        f0, m0 = f0.astype(np.float32).astype(np.float64), m0.astype(np.float32).astype(np.float64)
    e = eps if explicit_eps else O.obs_perturbations(w.seed, 0, w.ne, w.ny, w.sigma)
    xstar = O.restrict(f0, 1, 1, w.nc, w.ratio)
    st, m_ref, dC_ref = O.enkf_analyse(m0, xstar, yo, e, w.sigma, inp["obs_idx"], inp["obs_var"],
                                       1, 1, w.nc, w.ratio, gain_form=0 if gain_form else 1)
    assert st == 0
    fine_ref = O.prolong_add(dC_ref, f0, 1, 1, w.nc, w.ratio)
    return dict(fine=fine, mem=mem, fields=fields, xstar=xstar, e=e, m_ref=m_ref, dC_ref=dC_ref,
                fine_ref=fine_ref, m0=m0, f0=f0, yo=yo)


@pytest.mark.parametrize("gain_form", [0, 1])
@pytest.mark.parametrize("nf,ratio,ne,npr", CASES)
def test_fp64_analysis_matches_oracle(M, nf, ratio, ne, npr, gain_form):
    if gain_form == 1 and npr > 512:
        pytest.skip("direct form checked on moderate n_obs")
    w = W.burgers_custom(nf, ratio, ne, npr, obs_kind="random", sigma=0.3)
    r = _one_analysis(M, w, gain_form, "fp64", explicit_eps=False)
    np.testing.assert_allclose(r["fields"][M.MGENKF_FIELD_EPS].reshape(w.ne, w.ny), r["e"],
                               rtol=1e-14, atol=1e-15)
    np.testing.assert_array_equal(r["fields"][M.MGENKF_FIELD_XSTAR], r["xstar"])
    yf_ref = np.stack([O.obs_coarse(x, 1, 1, w.nc, w.ratio, *W.observation_layout(w))
                       for x in list(r["m0"]) + [r["xstar"]]])
    assert rel_err(r["fields"][M.MGENKF_FIELD_YF].reshape(w.ne + 1, w.ny), yf_ref) < 1e-13
    assert rel_err(r["fields"][M.MGENKF_FIELD_DC], r["dC_ref"]) < 1e-10
    assert rel_err(r["mem"] - r["m0"], r["m_ref"] - r["m0"]) < 1e-10
    assert rel_err(r["fine"], r["fine_ref"]) < 1e-12


@pytest.mark.parametrize("nf,ratio,ne,npr", [(256, 4, 32, 16), (4096, 4, 37, 130), (16384, 4, 128, 512)])
def test_mixed_analysis_matches_oracle(M, nf, ratio, ne, npr):
    w = W.burgers_custom(nf, ratio, ne, npr, obs_kind="random", sigma=0.05, precision="mixed")
    r = _one_analysis(M, w, 0, "mixed", explicit_eps=True)
    # BF16 anomalies X and gain coefficients T (8-bit significands, rounding
    # 2^-9 each) with FP32 accumulation: the increment X T carries a relative
    # error of a few 2^-8; tolerance 5 * 2^-8 = 2e-2 of the largest increment.
    # The states themselves are FP32 (2^-24), so their error is that increment
    # error plus FP32 rounding of the state.
    tol = 2e-2
    inc, inc_ref = r["mem"] - r["m0"], r["m_ref"] - r["m0"]
    assert rel_err(inc, inc_ref) < tol
    assert rel_err(r["fields"][M.MGENKF_FIELD_DC], r["dC_ref"]) < tol
    bound = tol * np.max(np.abs(inc_ref)) + 1e-6 * np.max(np.abs(r["m_ref"]))
    assert np.max(np.abs(r["mem"] - r["m_ref"])) < bound
    dfine = r["fine_ref"] - r["f0"]
    bound_f = tol * np.max(np.abs(dfine)) + 1e-6 * np.max(np.abs(r["fine_ref"]))
    assert np.max(np.abs(r["fine"] - r["fine_ref"])) < bound_f


@pytest.mark.parametrize("nf,ratio,ne,npr", [(256, 4, 32, 16), (4096, 4, 37, 130), (16384, 4, 128, 512)])
def test_mixed_gain_coefficients_match_oracle(M, nf, ratio, ne, npr):
    """The mixed path forms S = I + Y^T R^-1 Y and Y^T R^-1 [D | d*] in
    double-FP32 arithmetic (each FP64 operand split into two FP32 values): its
    gain coefficients T agree with the oracle's gain K = Y^T (Y Y^T + R)^-1
    (Algorithm 3 step 8, X = I) applied to [D | d*] to 1e-9 of the largest
    coefficient, where FP32 products would be off by about 1e-6."""
    w = W.burgers_custom(nf, ratio, ne, npr, obs_kind="random", sigma=0.05, precision="mixed")
    r = _one_analysis(M, w, 0, "mixed", explicit_eps=True)
    idx, var = W.observation_layout(w)
    yf = np.stack([O.obs_coarse(x, 1, 1, w.nc, w.ratio, idx, var) for x in list(r["m0"]) + [r["xstar"]]])
    Y = (yf[:ne] - yf[:ne].mean(axis=0)) / np.sqrt(ne - 1)          # ne x ny
    D = r["yo"][None, :] + r["e"] - yf[:ne]                          # ne x ny
    dstar = r["yo"] - yf[ne]
    st, K = O.enkf_gain(np.eye(ne), Y.T, w.sigma ** 2 * np.eye(w.ny))
    assert st == 0
    T_ref = np.vstack([D @ K.T, (K @ dstar)[None, :]])               # (ne + 1) x ne, row c = column c of T
    T = r["fields"][M.MGENKF_FIELD_T].reshape(ne + 1, ne)
    assert np.max(np.abs(T - T_ref)) <= 1e-9 * np.max(np.abs(T_ref))


def test_mixed_perturbations_follow_the_oracle_stream(M):
    # The mixed path draws the same Philox words and evaluates Box-Muller in
    # FP32 (each uniform rounded to FP32): the perturbations stay within FP32
    # rounding of the oracle's FP64 normals, element by element, over two
    # analyses (the device counter advances the stream).
    w = W.burgers_custom(1024, 4, 37, 130, obs_kind="random", sigma=0.3, precision="mixed")
    inp = W.make_inputs(w)
    g = M.MGEnKF.from_workload(w, precision="mixed")
    g.set_state(inp["fine0"], inp["members0"])
    for k in range(2):
        g.analyse(np.zeros(w.ny))
        assert g.sync() == 0
        got = g.field(M.MGENKF_FIELD_EPS).reshape(w.ne, w.ny)
        ref = O.obs_perturbations(w.seed, k, w.ne, w.ny, w.sigma)
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5 * w.sigma)
        assert np.max(np.abs(got - ref)) > 0.0  # FP32 arithmetic, not the FP64 values
    g.close()


def test_explicit_perturbations_are_used(M):
    w = W.burgers_custom(256, 4, 9, 7, obs_kind="random", sigma=0.2)
    r = _one_analysis(M, w, 0, "fp64", explicit_eps=True)
    np.testing.assert_array_equal(r["fields"][M.MGENKF_FIELD_EPS].reshape(w.ne, w.ny), r["e"])
    assert rel_err(r["mem"] - r["m0"], r["m_ref"] - r["m0"]) < 1e-10


@pytest.mark.parametrize("nf,ratio,ne,npr", [(4096, 4, 37, 130), (16384, 4, 128, 512), (1000, 4, 255, 60)])
def test_tensor_core_update_matches_cuda_core_update(M, nf, ratio, ne, npr, monkeypatch):
    # same BF16 operands, FP32 accumulation in different orders: the two member
    # updates agree to FP32 rounding of the sums (well inside 1e-5 of the increment)
    w = W.burgers_custom(nf, ratio, ne, npr, obs_kind="random", sigma=0.05, precision="mixed")
    inp = W.make_inputs(w)
    rng = np.random.default_rng(11)
    yo = rng.standard_normal(w.ny) * 0.2
    eps = w.sigma * rng.standard_normal((w.ne, w.ny))
    out = {}
    for mode in ("tc", "simt"):
        if mode == "simt":
            monkeypatch.setenv("MGENKF_UPDATE", "simt")
        g = M.MGEnKF.from_workload(w, precision="mixed")
        g.set_state(inp["fine0"], inp["members0"])
        g.analyse(yo, eps)
        assert g.sync() == 0
        _, mem = g.get_state()
        out[mode] = (mem, g.field(M.MGENKF_FIELD_DC))
        g.close()
    inc = out["simt"][0] - inp["members0"].astype(np.float32)
    scale = max(np.max(np.abs(inc)), 1e-30)
    assert np.max(np.abs(out["tc"][0] - out["simt"][0])) <= 1e-5 * scale + 2e-7
    dscale = max(np.max(np.abs(out["simt"][1])), 1e-30)
    assert np.max(np.abs(out["tc"][1] - out["simt"][1])) <= 1e-5 * dscale
