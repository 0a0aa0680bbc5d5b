"""Pins of the oracle's counter-based generator (Philox4x64-10) and of its
Box-Muller normals, against the published known answers, numpy's independent
Philox implementation, and the N(0,1) distribution."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert [int(x) for x in O.philox4x64_10(ctr, key)] == expect


@pytest.mark.parametrize("key,counter", [((0, 0), (0, 0, 0, 0)), ((123, 456), (7, 8, 9, 10)),
                                         ((2**64 - 1, 5), (2**64 - 1, 3, 0, 0)),
                                         ((0xDEADBEEF, 0), (41, 0, 2**63, 1))])
def test_philox_matches_numpy(key, counter):
    # numpy's Philox advances the 256-bit counter (with carry) before each block
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(counter, dtype=np.uint64))
    c = list(counter)
    for _ in range(3):
        c[0] = (c[0] + 1) % 2**64
        k = 1
        while c[k - 1] == 0 and k < 4:
            c[k] = (c[k] + 1) % 2**64
            if c[k] != 0:
                break
            k += 1
        got = [int(x) for x in O.philox4x64_10(c, key)]
        assert got == [int(x) for x in g.random_raw(4)]


def test_normals_distribution():
    from scipy import stats
    z = O.normals(seed=0, tag=O.EPS_TAG, ctr0=3, count=400_000)
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5 * np.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # the two members of a Box-Muller pair and neighbouring blocks are uncorrelated
    for lag in (1, 2, 4):
        assert abs(np.corrcoef(z[:-lag], z[lag:])[0, 1]) < 5 / np.sqrt(n)


def test_normals_streams_independent_and_prefix_stable():
    a = O.normals(0, O.EPS_TAG, 0, 1000)
    b = O.normals(0, O.EPS_TAG, 1, 1000)
    c = O.normals(1, O.EPS_TAG, 0, 1000)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.15 and abs(np.corrcoef(a, c)[0, 1]) < 0.15
    # count does not change the values already drawn (ragged tails)
    np.testing.assert_array_equal(O.normals(0, O.EPS_TAG, 0, 997), a[:997])
