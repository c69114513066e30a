"""Small exact fixtures (tests/golden/fj_small.json, written by
tests/golden/make_golden.py from the definitions in rational arithmetic):
the oracle must reproduce them to FP64 rounding, the CUDA path to its
certified tolerance."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fj_small.json")


def fixtures():
    with open(GOLDEN) as f:
        return json.load(f)["graphs"]


def csr(g):
    a = np.array(g["arcs"], np.float64).reshape(-1, 3)
    src, dst = a[:, 0].astype(np.int32), a[:, 1].astype(np.int32)
    return oracle.csr_from_arcs(g["n"], src, dst, a[:, 2].astype(np.float32))


@pytest.mark.parametrize("g", fixtures(), ids=lambda g: g["name"])
def test_oracle_matches_exact_fixture(g):
    rp, col, w = csr(g)
    s = np.array(g["s"])
    z = oracle.lu_solve(g["n"], rp, col, w, s)
    np.testing.assert_allclose(z, g["z"], rtol=1e-14, atol=1e-15)
    m = oracle.metrics(g["n"], rp, col, w, s, np.array(g["z"]), directed=g["directed"])
    for k, v in g["metrics"].items():
        assert abs(m[k] - v) <= 1e-14 * max(1.0, abs(v)), (k, m[k], v)


@pytest.mark.gpu
@pytest.mark.parametrize("g", fixtures(), ids=lambda g: g["name"])
def test_cuda_path_matches_exact_fixture(g):
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi
    from gpu_common import to_dev

    rp, col, w = csr(g)
    n = g["n"]
    s = np.array(g["s"])
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=g["directed"])
    (s_d,) = to_dev(s)
    z_d, info, st = G.solve(s_d, eps=1e-9, omega=1.0, precision=capi.FJ_PREC_FP64)
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    z = z_d.cpu().numpy()
    np.testing.assert_allclose(z, g["z"], rtol=1e-8, atol=1e-12)
    m = G.metrics(s_d, z_d)
    for k, v in g["metrics"].items():
        assert abs(m[k] - v) <= 1e-7 * max(1.0, abs(v)), (k, m[k], v)
