"""Batches of independent NS-2D MGEnKF problems (uneven grid sizes, ensemble
sizes and observation counts) cycled by one CUDA graph launch per cycle: the
batch must give exactly what each problem's own handle gives (forecast of
Eqs. Mass, Momentum, Energy; Algorithm 4 analysis and correction, with the
observation-perturbation counter advancing per analysis), for every tile
shape and after the autotuner, and must agree with the CPU oracle."""
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


def _problems():
    # coarse sides 8..40 (fine 32..160; ragged against every tile shape),
    # Ne 5..16, 16..64 observations
    return W.ns2d_batch(nprob=6, seed=3, coarse=(8, 16, 24, 40), members=(5, 8, 12, 16), n_obs=(16, 64))


def _inputs(ws, cycles):
    inps = [W.make_inputs(w) for w in ws]
    yos = [[W.sample_truth(w, inp["truth0"], inp["obs_idx"], inp["obs_var"]) + W.observation_noise(w, k)
            for k in range(cycles)] for w, inp in zip(ws, inps)]
    return inps, yos


def _runs(M, ws, inps, gain_forms=None):
    runs = []
    for j, (w, inp) in enumerate(zip(ws, inps)):
        gf = gain_forms[j] if gain_forms else M.MGENKF_GAIN_ENSEMBLE
        g = M.MGEnKF.from_workload(w, precision="mixed", gain_form=gf)
        g.set_state(inp["fine0"], inp["members0"])
        runs.append(g)
    return runs


def _per_handle(M, ws, inps, yos, nsteps, gain_forms=None):
    out = []
    for j, g in enumerate(_runs(M, ws, inps, gain_forms)):
        # the handles step with the 2-D tile kernel, the batch with the column
        # march: two kernels that must agree bit for bit
        g.set_forecast_choice(-1, -1)
        for k, n in enumerate(nsteps):
            g.cycle(n, yos[j][k])
        assert g.sync() == 0
        out.append(g.get_state())
        g.close()
    return out


def _batched(M, b, ws, yos, nsteps, innov=None):
    for k, n in enumerate(nsteps):
        out = np.empty(len(ws)) if innov is not None else None
        b.cycle(n, np.concatenate([yos[j][k] for j in range(len(ws))]), out)
        if innov is not None:
            innov.append(out)
    assert b.sync() == 0
    return [g.get_state() for g in b.runs]


@pytest.mark.parametrize("grouped,parts,split", [("1", "1", "ne"), ("1", "2", "ne"), ("1", "4", "ne"),
                                                  ("1", "2", "work"), ("0", "1", "ne")])
def test_batch_equals_per_problem_handles(M, monkeypatch, grouped, parts, split):
    """Grouped analysis (one launch per analysis step over the problems of a
    part; with several parts, part p's analysis runs beside part p + 1's
    forecast; parts ordered by Ne or balanced by work alone) and the
    per-problem chains on the graph's branches (MGENKF_BATCH_GROUPED=0) all
    give each problem's own handle results, bit for bit."""
    monkeypatch.setenv("MGENKF_BATCH_GROUPED", grouped)
    monkeypatch.setenv("MGENKF_BATCH_PARTS", parts)
    monkeypatch.setenv("MGENKF_BATCH_SPLIT", split)
    ws = _problems()
    assert len({w.nc for w in ws}) > 1 and len({w.ne for w in ws}) > 1
    nsteps = [10, 10, 7, 10]        # a changed step count recaptures the graph
    inps, yos = _inputs(ws, len(nsteps))
    ref = _per_handle(M, ws, inps, yos, nsteps)
    b = M.Batch(_runs(M, ws, inps))
    b.set_tiles({w.nc: 0 for w in ws} | {w.nf: 0 for w in ws})
    got = _batched(M, b, ws, yos, nsteps)
    for (f0, m0), (f1, m1) in zip(ref, got):
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(m1, m0)
    b.close()


@pytest.mark.parametrize("shape", list(range(16)))
def test_every_tile_shape_matches(M, shape):
    ws = _problems()
    nsteps = [10, 10]
    inps, yos = _inputs(ws, len(nsteps))
    ref = _per_handle(M, ws, inps, yos, nsteps)
    b = M.Batch(_runs(M, ws, inps))
    b.set_tiles({w.nc: shape for w in ws} | {w.nf: shape for w in ws})
    assert set(b.tiles().values()) == {shape}
    got = _batched(M, b, ws, yos, nsteps)
    for (f0, m0), (f1, m1) in zip(ref, got):
        # the per-point arithmetic does not depend on the segment length or
        # on the band width
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(m1, m0)
    b.close()


def test_autotune_and_persisted_tiles(M, tmp_path):
    ws = _problems()
    inps, yos = _inputs(ws, 2)
    b = M.Batch(_runs(M, ws, inps))
    tiles = b.autotune(reps=2)
    assert set(tiles) == {w.nc for w in ws} | {w.nf for w in ws}
    assert set(tiles.values()) <= set(M.SEGMENT_ROWS)
    path = tmp_path / "tiles.json"
    b.save_tiles(path)
    b.set_tiles({k: (v + 1) % len(M.SEGMENT_ROWS) for k, v in tiles.items()})
    b.load_tiles(path)
    assert b.tiles() == tiles
    # autotuning ran stages on scratch only: the states are still the initial ones
    for g, inp in zip(b.runs, inps):
        f, m = g.get_state()
        np.testing.assert_allclose(f, inp["fine0"], rtol=1e-6, atol=1e-6)
    got = _batched(M, b, ws, yos, [10, 10])
    ref = _per_handle(M, ws, inps, yos, [10, 10])
    for (f0, m0), (f1, m1) in zip(ref, got):
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(m1, m0)
    b.close()


def test_batch_matches_oracle(M):
    ws = _problems()
    cycles = 2
    inps, yos = _inputs(ws, cycles)
    b = M.Batch(_runs(M, ws, inps))
    innov = []
    got = _batched(M, b, ws, yos, [10] * cycles, innov)
    for j, (w, inp) in enumerate(zip(ws, inps)):
        mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"], inp["obs_idx"],
                      inp["obs_var"], w.sigma, w.seed, nu=w.nu, gamma=w.gamma, prandtl=w.prandtl, gain_form=1)
        for k in range(cycles):
            mg.forecast(10)
            assert mg.analyse(yos[j][k]) == 0
            # innovation y^o - H^C x^C* of the fine forecast (Algorithm 4)
            hs = O.obs_coarse(mg.xstar, 2, 4, w.nc, w.ratio, inp["obs_idx"], inp["obs_var"])
            d_rms = np.sqrt(np.mean((yos[j][k] - hs) ** 2))
            np.testing.assert_allclose(innov[k][j], d_rms, rtol=1e-3)
            mg.prolong_correct()
        assert rel_err(got[j][0], mg.fine) < 1e-3
        assert rel_err(got[j][1], mg.members) < 1e-3
    b.close()


def test_batch_rejects_bad_handles(M):
    ws = _problems()[:2]
    inps, _ = _inputs(ws, 1)
    runs = _runs(M, ws, inps)
    with pytest.raises(M.MGEnKFError):
        M.Batch([runs[0], runs[0]])
    g64 = M.MGEnKF.from_workload(ws[0], precision="fp64")
    with pytest.raises(M.MGEnKFError):
        M.Batch([runs[0], g64])
    wb = W.ns2d_shear(nf=64, ratio=4, ne=4, n_probes=8, precision="mixed")
    gb = M.MGEnKF(model=M.MGENKF_NS2D, n_fine=64, ratio=4, n_members=4, obs_index=[0, 0], obs_var=[1, 2],
                  length=1.0, dt=wb.dt, nu=wb.nu, obs_sigma=0.01, precision=M.MGENKF_MIXED, gamma=1.3)
    with pytest.raises(M.MGEnKFError):
        M.Batch([runs[0], gb])
    with pytest.raises(M.MGEnKFError):
        M.Batch([])
    for g in runs + [g64, gb]:
        g.close()


def test_batch_on_a_nonblocking_stream(M):
    """Handles and batch on a non-blocking stream with device observations and
    device innovation output (the benchmark's configuration)."""
    import torch
    ws = _problems()
    nsteps = [10, 10, 10]
    inps, yos = _inputs(ws, len(nsteps))
    ref = _per_handle(M, ws, inps, yos, nsteps)
    st = torch.cuda.Stream()
    runs = []
    for w, inp in zip(ws, inps):
        g = M.MGEnKF.from_workload(w, precision="mixed", stream=st.cuda_stream)
        g.set_state(inp["fine0"], inp["members0"])
        runs.append(g)
    b = M.Batch(runs, stream=st.cuda_stream)
    b.autotune(reps=1)
    y = torch.tensor(np.stack([np.concatenate([yos[j][k] for j in range(len(ws))]) for k in range(len(nsteps))]),
                     device="cuda")
    innov = torch.zeros((len(nsteps), len(ws)), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for k, n in enumerate(nsteps):
        b.cycle(n, y[k], innov[k])
    assert b.sync() == 0
    assert torch.isfinite(innov).all() and (innov > 0).all()
    for g, (f0, m0) in zip(b.runs, ref):
        f1, m1 = g.get_state()
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(m1, m0)
    b.close()


def test_batch_at_multi_tile_sizes_matches_oracle(M):
    """Problems of the batched workload's own sizes (coarse 64^2-128^2, fine 4x
    per side, 16-32 members): the column march of every grid size runs many
    more CTAs than are resident (each member grid 2-4 row segments, each fine
    grid 8-16), against the CPU oracle over two cycles."""
    ws = W.ns2d_batch(nprob=8, seed=5, coarse=(64, 96, 128), members=(16, 32), n_obs=(256, 512))
    cycles = 2
    inps, yos = _inputs(ws, cycles)
    b = M.Batch(_runs(M, ws, inps))
    got = _batched(M, b, ws, yos, [10] * cycles)
    for j, (w, inp) in enumerate(zip(ws, inps)):
        mg = O.MGEnKF(w.model, w.nf, w.ratio, w.length, w.dt, inp["fine0"], inp["members0"], inp["obs_idx"],
                      inp["obs_var"], w.sigma, w.seed, nu=w.nu, gamma=w.gamma, prandtl=w.prandtl, gain_form=1)
        for k in range(cycles):
            mg.forecast(10)
            assert mg.analyse(yos[j][k]) == 0
            mg.prolong_correct()
        assert rel_err(got[j][0], mg.fine) < 1e-3
        assert rel_err(got[j][1], mg.members) < 1e-3
    b.close()


def test_grouped_cycle_launches(M, monkeypatch):
    """A grouped batch cycle (one part) launches the forecast steps of each
    grid size and a fixed number of analysis launches, whatever the problem
    count; the per-problem chains launch about 13 kernels per problem."""
    monkeypatch.setenv("MGENKF_BATCH_PARTS", "1")
    ws = _problems()
    inps, yos = _inputs(ws, 1)
    counts = {}
    for grouped in ("1", "0"):
        monkeypatch.setenv("MGENKF_BATCH_GROUPED", grouped)
        b = M.Batch(_runs(M, ws, inps))
        n0 = M.mgk_kernel_launches()
        b.cycle(4, np.concatenate([yos[j][0] for j in range(len(ws))]))
        assert b.sync() == 0
        counts[grouped] = M.mgk_kernel_launches() - n0
        b.close()
    nsizes = len({w.nc for w in ws} | {w.nf for w in ws})
    # forecast: 4 step launches per grid size (plus a copy-back per size at most)
    assert counts["1"] <= 5 * nsizes + 14
    assert counts["0"] >= counts["1"] + 10 * (len(ws) - 1)


def test_batch_with_a_direct_form_problem(M):
    """A problem the grouped kernels do not take (direct gain form) sends the
    batch to the per-problem chains; the results are still each handle's own."""
    ws = _problems()
    forms = [M.MGENKF_GAIN_ENSEMBLE] * len(ws)
    forms[1] = M.MGENKF_GAIN_DIRECT
    nsteps = [10, 10]
    inps, yos = _inputs(ws, len(nsteps))
    ref = _per_handle(M, ws, inps, yos, nsteps, forms)
    b = M.Batch(_runs(M, ws, inps, forms))
    got = _batched(M, b, ws, yos, nsteps)
    for (f0, m0), (f1, m1) in zip(ref, got):
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(m1, m0)
    b.close()


def test_grouped_analysis_at_every_member_count_equals_handles(M):
    """Member counts 16..128 in one batch: one-CTA and clustered Cholesky,
    split and unsplit gain products, 1..17 solve CTAs per problem, 32..256
    TMEM columns in one grouped update; bit for bit each handle's results."""
    ws = W.ns2d_batch(nprob=6, seed=4, coarse=(16, 24), members=(16, 32, 64, 128), n_obs=(64, 512))
    assert {w.ne for w in ws} >= {16, 128}
    nsteps = [6, 6]
    inps, yos = _inputs(ws, len(nsteps))
    ref = _per_handle(M, ws, inps, yos, nsteps)
    b = M.Batch(_runs(M, ws, inps))
    got = _batched(M, b, ws, yos, nsteps)
    for (f0, m0), (f1, m1) in zip(ref, got):
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(m1, m0)
    b.close()


def _shear(nf, ne, n_probes, seed):
    import dataclasses
    w = W.ns2d_shear(nf=nf, ratio=4, ne=ne, n_probes=n_probes, cycles=4, precision="mixed", seed=seed)
    return dataclasses.replace(w, name=f"edge_{nf}_{ne}_{seed}")


@pytest.mark.parametrize("case", ["one problem", "extremes", "fallback"])
def test_batch_edge_cases_equal_handles(M, case):
    """A batch of one problem; Ne = 2 and Ne = 160, the largest the grouped
    kernels take (its tensor-core update has room for one member buffer only,
    so each tile's load waits for the previous tile's epilogue), beside a
    ragged Ne = 17; and a batch with Ne = 161, which runs one chain per
    problem: each problem's results are its own handle's, bit for bit."""
    if case == "one problem":
        ws = [_shear(64, 8, 32, 1)]
    elif case == "extremes":
        ws = [_shear(64, 2, 24, 2), _shear(64, 160, 200, 3), _shear(96, 17, 40, 4)]
    else:
        ws = [_shear(64, 161, 60, 5), _shear(64, 16, 30, 6)]
    nsteps = [5, 5]
    inps, yos = _inputs(ws, len(nsteps))
    ref = _per_handle(M, ws, inps, yos, nsteps)
    b = M.Batch(_runs(M, ws, inps))
    got = _batched(M, b, ws, yos, nsteps)
    for (f0, m0), (f1, m1) in zip(ref, got):
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(m1, m0)
    b.close()
