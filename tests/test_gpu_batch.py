"""Multi-right-hand-side push (fj_solve_batch) against the FP64 oracle.

Every vector of a batch is compared with the oracle's certified truth for that
vector alone (relative max-norm error 1e-6 on the FP64 path, 1e-5 on the FP32
path), and its FP64 residual is recomputed on the CPU to check the certificate
|r_v| <= eps' s'_v of Lemma 5 column by column.  Sizes span many warp tiles,
long-row chunks (hub rows of R-MAT) and a ragged lane split (k = 33).
"""
import numpy as np
import pytest

import oracle
from fjsynth import OP_ARCSINE, OP_SIGN, OP_UNIFORM
from fjsynth import workloads as W
from gpu_common import FP32_TOL, FP64_TOL, METRIC_TOL, certificate_holds, csr_of, rel_inf, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi as c
    return c


def _check_columns(n, rp, col, w, S, Z, infos, tol, truth_cols, omega_truth=1.5):
    k = S.shape[1]
    for j in range(k):
        inf = infos[j]
        assert inf["converged"] == 1, (j, inf)
        ok, r = certificate_holds(n, rp, col, w, S[:, j], Z[:, j], inf["c_eff"], inf["eps_prime"])
        assert ok, (j, float(np.max(np.abs(r) / (S[:, j] + inf["c_eff"]))))
        # the shift of Alg. 2 per vector: c_eff = c + max(0, -min s)
        assert inf["c_eff"] == pytest.approx(1e-5 + max(0.0, -float(S[:, j].min())), rel=0, abs=1e-15)
    for j in truth_cols:
        z_star, _ = oracle.truth(n, rp, col, w, S[:, j], omega=omega_truth)
        assert rel_inf(Z[:, j], z_star) <= tol, j


@pytest.mark.parametrize("k,omega,schedule", [(8, 1.5, 2), (8, 1.0, 1), (33, 1.2, 2)])
def test_batch_fp64_ba20k(capi, k, omega, schedule):
    g = W.ba_graph(20000, 5, nvec=k)
    rp, col, w = csr_of(g)
    n = g["n"]
    S = np.ascontiguousarray(np.stack(g["S"], axis=1))
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    (S_d,) = to_dev(S)
    Z_d, infos, st = G.solve_batch(S_d, eps=1e-6, omega=omega, precision=capi.FJ_PREC_FP64, schedule=schedule)
    assert st == capi.FJ_OK
    Z = Z_d.cpu().numpy()
    _check_columns(n, rp, col, w, S, Z, infos, FP64_TOL, truth_cols=[0, k // 2, k - 1])


def test_batch_fp32_rmat_undirected_64_mixed_kinds(capi):
    """64 vectors cycling U[0,1], Beta(1/2,1/2) and +-1 labels (signed: shifted per vector)."""
    g = W.rmat_undirected(14, 16, 4, kinds=(OP_UNIFORM, OP_ARCSINE, OP_SIGN), nvec=64)
    rp, col, w = csr_of(g)
    n = g["n"]
    S = np.ascontiguousarray(np.stack(g["S"], axis=1))
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    (S_d,) = to_dev(S)
    Z_d, infos, st = G.solve_batch(S_d, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    assert st == capi.FJ_OK
    Z = Z_d.cpu().numpy()
    _check_columns(n, rp, col, w, S, Z, infos, FP32_TOL, truth_cols=[0, 1, 2, 63])
    # undirected: 1^T z = 1^T s for every vector
    np.testing.assert_allclose(Z.sum(axis=0), S.sum(axis=0), rtol=0, atol=1e-6 * np.abs(S).sum(axis=0).max())
    # batched Table 1 measures: against the oracle's sums on the same z, and on the truth
    mets = G.metrics_batch(S_d, Z_d)
    for j in (0, 1, 2, 33, 63):
        mo = oracle.metrics(n, rp, col, w, S[:, j], Z[:, j], directed=False)
        for key in ("P", "D", "I", "C", "mean_z"):
            assert abs(mets[j][key] - mo[key]) <= 1e-12 * abs(mo[key]) + 1e-15, (j, key)
    for j in (0, 2):
        z_star, _ = oracle.truth(n, rp, col, w, S[:, j], omega=1.5)
        mt = oracle.metrics(n, rp, col, w, S[:, j], z_star, directed=False)
        for key in ("P", "D", "I", "C"):
            assert abs(mets[j][key] - mt[key]) <= METRIC_TOL * abs(mt[key]), (j, key)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_directed_weighted_matches_single(capi, precision):
    g = W.rmat_directed(13, nvec=5)
    rp, col, w = csr_of(g)
    n = g["n"]
    S = np.ascontiguousarray(np.stack(g["S"], axis=1))
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=True)
    Z, infos, st = G.solve_batch(S, eps=1e-6, omega=1.2, precision=precision)  # host memory
    assert st == capi.FJ_OK
    tol = FP64_TOL if precision == 0 else FP32_TOL
    _check_columns(n, rp, col, w, S, Z, infos, tol, truth_cols=[0, 4], omega_truth=1.0)
    mets = G.metrics_batch(S, Z)  # host memory, weighted directed
    for j in range(S.shape[1]):
        mo = oracle.metrics(n, rp, col, w, S[:, j], Z[:, j], directed=True)
        for key in ("P", "D", "I", "C", "mean_z"):
            assert abs(mets[j][key] - mo[key]) <= 1e-12 * abs(mo[key]) + 1e-15, (j, key)
    for j in (0, 3):
        z1, _, _ = G.solve(np.ascontiguousarray(S[:, j]), eps=1e-6, omega=1.2, precision=precision)
        assert rel_inf(Z[:, j], z1) <= 2 * tol


def test_batch_k1_and_repeat_deterministic(capi):
    g = W.ba_graph(5000, 3, seed_off=41)
    rp, col, w = csr_of(g)
    n = g["n"]
    S = np.ascontiguousarray(g["S"][0][:, None])
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    Z1, i1, _ = G.solve_batch(S, eps=1e-6, omega=1.0, precision=0, schedule=1)
    Z2, i2, _ = G.solve_batch(S, eps=1e-6, omega=1.0, precision=0, schedule=1)
    # Jacobi rounds have no intra-sweep races: bit-identical on repeat
    assert np.array_equal(Z1, Z2) and i1[0]["sweeps"] == i2[0]["sweeps"]
    z_star, _ = oracle.truth(n, rp, col, w, S[:, 0])
    assert rel_inf(Z1[:, 0], z_star) <= FP64_TOL


def test_batch_constant_columns(capi):
    """Constant s gives constant z = s (row sums of I + L are 1)."""
    g = W.ba_graph(3000, 4, seed_off=43)
    rp, col, w = csr_of(g)
    n = g["n"]
    S = np.ascontiguousarray(np.stack([np.full(n, 0.25), np.full(n, -2.0), np.zeros(n)], axis=1))
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    Z, infos, st = G.solve_batch(S, eps=1e-6, omega=1.5, precision=0)
    assert st == capi.FJ_OK
    for j in range(3):
        bound = infos[j]["eps_prime"] * (np.abs(S[:, j]).max() + infos[j]["c_eff"]) * 1.01
        assert np.max(np.abs(Z[:, j] - S[:, j])) <= bound


def test_batch_invalid_arguments(capi):
    g = W.ba_graph(2000, 3, seed_off=44)
    rp, col, w = csr_of(g)
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    for k in (65,):
        with pytest.raises(capi.FJError):
            G.solve_batch(np.zeros((n, k)), eps=1e-6)
    S = np.zeros((n, 2))
    S[5, 1] = np.nan
    with pytest.raises(capi.FJError):
        G.solve_batch(S, eps=1e-6)
    # a ragged handle (two disjoint graphs) takes one vector per graph: rejected
    rp2 = np.concatenate([rp, rp[1:] + rp[-1]]).astype(np.int64)
    col2 = np.concatenate([col, col + n]).astype(np.int32)
    R = capi.Graph.ragged(np.array([0, n, 2 * n], np.int64), rp2, col2, directed=False)
    with pytest.raises(capi.FJError):
        R.solve_batch(np.zeros((2 * n, 2)), eps=1e-6)


def test_autotuner_picks_a_certified_configuration(capi):
    g = W.ba_graph(20000, 5, nvec=4, seed_off=47)
    rp, col, w = csr_of(g)
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    s = g["S"][0]
    best, ms = G.tune(s, reps=1, eps=1e-6, precision=capi.FJ_PREC_FP32)
    assert ms > 0
    assert best["schedule"] in (capi.FJ_SCHED_JACOBI, capi.FJ_SCHED_MULTICOLOUR)
    if best["schedule"] == capi.FJ_SCHED_JACOBI:
        assert best["omega"] == 1.0
    else:
        # the fixed grid, or Eq. 17's omega from the same 200 power-iteration steps the tuner takes
        wopt = G.omega_opt(200)[1]
        assert best["palette"] in (4, 8, 16, 32) and best["omega"] in (1.2, 1.5, 1.6, 1.7, 1.8, wopt)
    z, info, st = G.solve(s, eps=1e-6, precision=capi.FJ_PREC_FP32, **best)
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    z_star, _ = oracle.truth(n, rp, col, w, s)
    assert rel_inf(z, z_star) <= FP32_TOL
    S = np.ascontiguousarray(np.stack(g["S"], axis=1))
    bb, bms = G.tune_batch(S, reps=1, eps=1e-6, precision=capi.FJ_PREC_FP32)
    Z, infos, st = G.solve_batch(S, eps=1e-6, precision=capi.FJ_PREC_FP32, **bb)
    assert st == capi.FJ_OK and all(i["converged"] == 1 for i in infos)


def test_replicas_on_two_streams_match_single_stream(capi):
    """Replicas: two handles solving disjoint sets of opinion vectors at the
    same time, each on its own CUDA stream from its own host thread, give
    bit for bit the results of the same solves run one after another."""
    import threading

    import torch

    g = W.rmat_multirhs(12, 4)
    rp, col, w = csr_of(g)
    n = g["n"]
    S = [np.ascontiguousarray(v) for v in g["S"]]
    opts = dict(eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    ref_h = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    want, bound = [], []
    for v in S:
        z, info, st = ref_h.solve(v, **opts)
        assert st == capi.FJ_OK
        want.append(np.array(z))
        # bit-identity holds when the atomics of the FP64 frontier cleanup did not run
        bound.append(0.0 if info[0]["frontier_rounds"] == 0 else 2 * info[0]["err_bound"])
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    handles = []
    for st_ in streams:
        with torch.cuda.stream(st_):
            handles.append(capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False, stream=st_.cuda_stream))
    got = [None] * len(S)
    got_rounds = [0] * len(S)
    got_bound = [0.0] * len(S)
    errors = []

    def replica(r):
        try:
            for j in range(r, len(S), 2):
                z, info, st = handles[r].solve(S[j], stream=streams[r].cuda_stream, **opts)
                got[j] = np.array(z)
                got_rounds[j] = info[0]["frontier_rounds"]
                got_bound[j] = info[0]["err_bound"]
        except Exception as e:  # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=replica, args=(r,)) for r in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for j in range(len(S)):
        if bound[j] == 0.0 and got_rounds[j] == 0:
            assert np.array_equal(got[j], want[j]), j
        else:
            assert np.max(np.abs(got[j] - want[j])) <= bound[j] + 2 * got_bound[j], j
