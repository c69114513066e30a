"""Parity at the full benchmark sizes, in the launch configuration bench.py times.

At these sizes the oracle cannot solve the systems in seconds, so the checks
are properties that hold at any size, computed by the oracle on the CPU from
its own CSR (built from the same generator output, never from the GPU):
  - ingest: the GPU CSR (offsets, columns, weights, FP64 degrees) equals the
    oracle's bit for bit;
  - certificate: the residual of the returned z, evaluated exactly by the
    oracle (compensated sums), meets the solver's test at every node, which
    bounds max_v |z_v - z*_v| by max_v |r_v| (Lemma 5, (I + L)^{-1} is
    row-stochastic and nonnegative); that bound, relative to max |z|, must be
    within the FP32 tolerance 1e-5;
  - metrics: fj_metrics on the returned z equals the oracle's Table 1 sums on
    the same z within the bound on two summation orders of the same m terms,
    2 m 2^-53 relative (m = n for C, P, I; m = nnz for D).
"""
import numpy as np
import pytest

import oracle
from fjsynth import workloads as W
from gpu_common import FP32_TOL, certificate_holds, csr_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi as c
    return c


def _dev(*arrays):
    import torch
    return [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _ingest(capi, g):
    if g["directed"]:
        src, dst, w = g["src"], g["dst"], g["w"]
    else:
        src, dst, w = W.symmetrize_arcs(g["src"], g["dst"], g["w"])
    G = capi.Graph.from_arcs(g["n"], *_dev(src, dst, w), directed=g["directed"])
    rp, col, wc = csr_of(g)
    grp, gcol, gw, gdeg = G.export(weights=wc is not None)
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    if wc is not None:
        assert np.array_equal(gw, wc)
    assert np.array_equal(gdeg, oracle.out_degree(g["n"], rp, wc))
    del grp, gcol, gw, gdeg
    return G, rp, col, wc


def _check_solution(n, rp, col, w, s, z, info, directed, G):
    ok, r = certificate_holds(n, rp, col, w, s, z, info["c_eff"], info["eps_prime"])
    assert ok, float(np.max(np.abs(r) / (s + info["c_eff"])))
    assert np.max(np.abs(r)) / np.max(np.abs(z)) <= FP32_TOL
    m = G.metrics(s, z)
    mo = oracle.metrics(n, rp, col, w, s, z, directed=directed)
    _metrics_agree(m, mo, n, int(rp[-1]))


def _metrics_agree(m, mo, n, nnz):
    for k in ("P", "D", "I", "C", "mean_z"):
        terms = nnz if k == "D" else n
        assert abs(m[k] - mo[k]) <= 2.0 * terms * 2.0 ** -53 * abs(mo[k]) + 1e-300, k


def test_rmat22_directed_full_size(capi):
    """Directed R-MAT scale 22 (65,243,118 arcs after dedup), FP32, omega 1.6, 8 colours."""
    g = W.rmat_directed(22)
    G, rp, col, w = _ingest(capi, g)
    n, s = g["n"], g["S"][0]
    (s_d,) = _dev(s)
    z_d, info, st = G.solve(s_d, eps=1e-6, omega=1.6, palette=8, precision=capi.FJ_PREC_FP32)
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    _check_solution(n, rp, col, w, s, z_d.cpu().numpy(), info[0], True, G)


def test_rmat22_undirected_64_vectors_full_size(capi):
    """Undirected R-MAT scale 22, 64 vectors (U / Beta(1/2,1/2) / +-1), one batch;
    every vector certificate-checked."""
    g = W.rmat_multirhs(22, 64)
    G, rp, col, w = _ingest(capi, g)
    n = g["n"]
    S = np.ascontiguousarray(np.stack(g["S"], axis=1))
    (S_d,) = _dev(S)
    Z_d, infos, st = G.solve_batch(S_d, eps=1e-6, omega=1.7, precision=capi.FJ_PREC_FP32)
    assert st == capi.FJ_OK
    Z = Z_d.cpu().numpy()
    mets = G.metrics_batch(S_d, Z_d)
    for j in range(64):
        s, z = np.ascontiguousarray(S[:, j]), np.ascontiguousarray(Z[:, j])
        assert infos[j]["converged"] == 1
        ok, r = certificate_holds(n, rp, col, w, s, z, infos[j]["c_eff"], infos[j]["eps_prime"])
        assert ok, j
        assert np.max(np.abs(r)) / np.max(np.abs(z)) <= FP32_TOL
        if j % 16 == 0:
            mo = oracle.metrics(n, rp, col, w, s, z, directed=False)
            _metrics_agree(mets[j], mo, n, int(rp[-1]))


def test_rmat24_undirected_full_size(capi):
    """Undirected R-MAT scale 24 (268,435,456 generated edges), Beta(2,5)/Beta(5,2)
    opinions, FP32, omega 1.8."""
    g = W.rmat_undirected(24)
    G, rp, col, w = _ingest(capi, g)
    n, s = g["n"], g["S"][0]
    (s_d,) = _dev(s)
    z_d, info, st = G.solve(s_d, eps=1e-6, omega=1.8, precision=capi.FJ_PREC_FP32)
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    z = z_d.cpu().numpy()
    _check_solution(n, rp, col, w, s, z, info[0], False, G)
    # undirected: 1^T z = 1^T s
    assert abs(z.sum() - s.sum()) <= 1e-6 * np.abs(s).sum()
