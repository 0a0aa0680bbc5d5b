"""Training of the learned prolongation correction on the GPU and what it
gains: trained on pairs from four seeded runs, evaluated on a fifth seed, the
network's fine correction is much closer to the correction of a
full-resolution EnKF than plain prolongation is; attached to a handle it runs
inside the cycle."""
import numpy as np
import pytest

from paper_2012_10091_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import surrogate
    return surrogate


def _w(seed):
    return W.ns2d_shear(nf=64, ratio=4, ne=16, n_probes=64, cycles=100, precision="mixed", delta=0.08, seed=seed)


def test_trained_network_beats_plain_prolongation_on_unseen_run(S):
    sets = [S.generate_pairs(_w(seed), 100) for seed in range(5)]
    train, val = S.concat_pairs(*sets[:4]), sets[4]
    cnn, stats, hist = S.fit(train, epochs=20, batch=8, lr=3e-4, val_pairs=val)
    # untrained network = plain prolongation; the trained one halves the error at least
    assert min(hist["val"]) < 0.5 * hist["val_plain"], hist
    assert hist["train"][-1] < hist["train"][0]
    # the trained network runs inside the cycle and keeps the run finite
    rm = S.run_cycles(_w(7), 10, cnn)
    assert np.all(np.isfinite(rm))
    cnn.close()


def test_untrained_network_in_cycle_equals_plain_prolongation(S):
    from paper_2012_10091_gb300 import mgenkf as M
    cnn = M.CNN(16, 1)
    cnn.set_params(S.init_params(0), dict(mu_in=np.zeros(8), s_in=np.ones(8), s_out=np.ones(4)))
    rp = S.run_cycles(_w(3), 5)
    rc = S.run_cycles(_w(3), 5, cnn)
    np.testing.assert_allclose(rc, rp, rtol=1e-6)
    cnn.close()
