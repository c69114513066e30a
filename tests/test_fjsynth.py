"""The seeded input generators: determinism and the distributions they claim."""
import numpy as np

import fjsynth
from fjsynth import workloads as W


def test_rmat_independent_of_thread_count():
    a = fjsynth.rmat(12, 8, seed=3, weighted=True, nthreads=1)
    b = fjsynth.rmat(12, 8, seed=3, weighted=True, nthreads=7)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_rmat_quadrant_frequencies():
    src, dst, w = fjsynth.rmat(10, 64, seed=11, weighted=True)
    top_src = src >> 9
    top_dst = dst >> 9
    n = src.shape[0]
    freq = [np.mean((top_src == i) & (top_dst == j)) for i, j in ((0, 0), (0, 1), (1, 0), (1, 1))]
    np.testing.assert_allclose(freq, [0.57, 0.19, 0.19, 0.05], atol=4 / np.sqrt(n))
    assert w.min() >= 0.5 and w.max() <= 1.5
    assert src.max() < 1024 and dst.max() < 1024


def test_ba_structure():
    src, dst = fjsynth.ba(5000, 5, seed=2)
    assert src.shape[0] == 15 + (5000 - 6) * 5
    deg = np.bincount(np.concatenate([src, dst]), minlength=5000)
    assert deg.min() >= 5
    # every new node links to 5 distinct earlier nodes
    new = src >= 6
    assert np.all(dst[new] < src[new])
    pairs = set(zip(src.tolist(), dst.tolist()))
    assert len(pairs) == src.shape[0]


def test_opinion_distributions():
    n = 200000
    u = fjsynth.opinions(n, fjsynth.OP_UNIFORM, seed=1)
    assert 0 <= u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.005
    b = fjsynth.opinions(n, fjsynth.OP_BETA_MIX, seed=1)
    assert abs(b[0::2].mean() - 2 / 7) < 0.005 and abs(b[1::2].mean() - 5 / 7) < 0.005
    # Beta(2,5) variance = 2*5 / (7^2 * 8)
    assert abs(b[0::2].var() - 10 / 392) < 0.002
    a = fjsynth.opinions(n, fjsynth.OP_ARCSINE, seed=1)
    assert abs(a.mean() - 0.5) < 0.005 and abs(a.var() - 0.125) < 0.003
    sgn = fjsynth.opinions(n, fjsynth.OP_SIGN, seed=1)
    assert set(np.unique(sgn)) == {-1.0, 1.0} and abs(sgn.mean()) < 0.01
    for kind in (fjsynth.OP_EXP, fjsynth.OP_PARETO):
        x = fjsynth.opinions(n, kind, seed=1)
        assert x.min() > 0 and x.max() == 1.0
    assert not np.array_equal(fjsynth.opinions(100, 0, 1, vec=0), fjsynth.opinions(100, 0, 1, vec=1))


def test_workload_shapes():
    g = W.rmat_directed(10)
    assert g["n"] == 1024 and g["src"].shape[0] == 16 * 1024 and g["w"] is not None
    assert np.array_equal(g["S"][0], g["S"][0].astype(np.float32).astype(np.float64))
    r = W.ragged_ba(count=8, lo=100, hi=2000)
    assert len(r["graphs"]) == 8 and all(100 <= x["n"] <= 2000 for x in r["graphs"])
    a, b, c = W.symmetrize_arcs(np.array([1, 2], np.int32), np.array([3, 4], np.int32))
    assert a.tolist() == [1, 3, 2, 4] and b.tolist() == [3, 1, 4, 2]
