"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms
derived by hand from Lemma 1, the Neumann series of Lemma 2, a library sparse
solver, the bounds of Lemmas 3-5, the Gauss-Seidel equivalence of Theorem 2,
algebraic identities of the Table 1 measures, and Young's SOR theory.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from fjsynth import workloads as W


def csr(n, arcs, weights=None):
    src = np.array([a for a, _ in arcs], np.int32)
    dst = np.array([b for _, b in arcs], np.int32)
    w = None if weights is None else np.array(weights, np.float32)
    return oracle.csr_from_arcs(n, src, dst, w)


def undirected(n, edges, weights=None):
    arcs = []
    ws = []
    for i, (a, b) in enumerate(edges):
        arcs += [(a, b), (b, a)]
        if weights is not None:
            ws += [weights[i], weights[i]]
    return csr(n, arcs, ws if weights is not None else None)


def random_graph(n, p, directed, weighted, seed):
    rng = np.random.default_rng(seed)
    arcs, ws = [], []
    for u in range(n):
        for v in range(n):
            if u != v and (directed or u < v) and rng.random() < p:
                wt = float(np.float32(0.5 + rng.random()))
                arcs.append((u, v))
                ws.append(wt)
                if not directed:
                    arcs.append((v, u))
                    ws.append(wt)
    return csr(n, arcs, ws if weighted else None)


def all_solvers(n, rp, col, w, s):
    """z from LU, the certified SOR truth, and FIFO push at a tiny eps."""
    z_lu = oracle.lu_solve(n, rp, col, w, s)
    z_fifo = oracle.blisor_fifo(n, rp, col, w, s, 1e-13, 1.0)[0]
    z_sor = oracle.sor_ordered(n, rp, col, w, s, np.arange(n, dtype=np.int32), 1e-13, 1.0)[0]
    return z_lu, z_fifo, z_sor


# ------------------------------------------------------------ closed forms

def test_single_edge_closed_form():
    s = np.array([0.2, 0.9])
    rp, col, w = undirected(2, [(0, 1)])
    want = np.array([(2 * s[0] + s[1]) / 3, (s[0] + 2 * s[1]) / 3])
    for z in all_solvers(2, rp, col, w, s):
        np.testing.assert_allclose(z, want, rtol=0, atol=1e-11)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_undirected_star_closed_form(k):
    rng = np.random.default_rng(k)
    s = rng.random(k + 1)
    rp, col, w = undirected(k + 1, [(0, l) for l in range(1, k + 1)])
    z0 = (2 * s[0] + s[1:].sum()) / (k + 2)
    want = np.concatenate([[z0], (s[1:] + z0) / 2])
    for z in all_solvers(k + 1, rp, col, w, s):
        np.testing.assert_allclose(z, want, rtol=0, atol=1e-11)


@pytest.mark.parametrize("n", [2, 5, 9])
def test_complete_graph_closed_form(n):
    s = np.random.default_rng(n).random(n)
    rp, col, w = undirected(n, [(a, b) for a in range(n) for b in range(a + 1, n)])
    want = (s + s.sum()) / (n + 1)
    for z in all_solvers(n, rp, col, w, s):
        np.testing.assert_allclose(z, want, rtol=0, atol=1e-11)


def test_directed_arc_closed_form():
    # node 0 listens to node 1
    s = np.array([0.1, 0.7])
    rp, col, w = csr(2, [(0, 1)])
    want = np.array([(s[0] + s[1]) / 2, s[1]])
    for z in all_solvers(2, rp, col, w, s):
        np.testing.assert_allclose(z, want, rtol=0, atol=1e-11)


def test_directed_weighted_arc_closed_form():
    a = float(np.float32(1.37))
    s = np.array([0.25, 0.8])
    rp, col, w = csr(2, [(0, 1)], [a])
    want = np.array([(s[0] + a * s[1]) / (1 + a), s[1]])
    for z in all_solvers(2, rp, col, w, s):
        np.testing.assert_allclose(z, want, rtol=0, atol=1e-11)


@pytest.mark.parametrize("k", [1, 4])
def test_directed_stars_closed_form(k):
    s = np.random.default_rng(10 + k).random(k + 1)
    # leaves listen to the centre 0
    rp, col, w = csr(k + 1, [(l, 0) for l in range(1, k + 1)])
    want = np.concatenate([[s[0]], (s[1:] + s[0]) / 2])
    for z in all_solvers(k + 1, rp, col, w, s):
        np.testing.assert_allclose(z, want, rtol=0, atol=1e-11)
    # the centre listens to the leaves
    rp, col, w = csr(k + 1, [(0, l) for l in range(1, k + 1)])
    want = np.concatenate([[(s[0] + s[1:].sum()) / (k + 1)], s[1:]])
    for z in all_solvers(k + 1, rp, col, w, s):
        np.testing.assert_allclose(z, want, rtol=0, atol=1e-11)


def test_exact_rational_path():
    # path 0-1-2, s = (1, 0, 0): (I+L) z = s solved by hand in rationals
    # [[2,-1,0],[-1,3,-1],[0,-1,2]] z = (1,0,0)  ->  z = (5/8, 1/4, 1/8)
    rp, col, w = undirected(3, [(0, 1), (1, 2)])
    want = [Fraction(5, 8), Fraction(1, 4), Fraction(1, 8)]
    for z in all_solvers(3, rp, col, w, np.array([1.0, 0.0, 0.0])):
        np.testing.assert_allclose(z, [float(x) for x in want], rtol=0, atol=1e-11)


# ------------------------------------------------------- independent routes

@pytest.mark.parametrize("directed,weighted", [(False, False), (True, False), (True, True), (False, True)])
def test_neumann_series_matches_lu(directed, weighted):
    n = 9
    rp, col, w = random_graph(n, 0.35, directed, weighted, seed=3 + directed + 2 * weighted)
    s = np.random.default_rng(5).random(n)
    z_lu = oracle.lu_solve(n, rp, col, w, s)
    z_ns = oracle.neumann_series(n, rp, col, w, s)
    np.testing.assert_allclose(z_lu, z_ns, rtol=0, atol=1e-13)


@pytest.mark.parametrize("directed", [False, True])
def test_library_sparse_solve_matches_lu(directed):
    scipy_sparse = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    n = 300
    rp, col, w = random_graph(n, 0.03, directed, True, seed=11 + directed)
    s = np.random.default_rng(8).random(n)
    A = scipy_sparse.csr_matrix((np.asarray(w, np.float64), col, rp), shape=(n, n))
    d = np.asarray(A.sum(axis=1)).ravel()
    M = scipy_sparse.identity(n) + scipy_sparse.diags(d) - A
    z_lib = spla.spsolve(M.tocsc(), s)
    np.testing.assert_allclose(oracle.lu_solve(n, rp, col, w, s), z_lib, rtol=0, atol=1e-12)
    z_t, res = oracle.truth(n, rp, col, w, s)
    assert res < 1e-12


# ------------------------------------------------------------ truth oracle, sweep branch
#
# truth() solves by dense LU up to n = 2000 and by sequential SOR sweeps with
# an inline residual stop above that; the sweep branch is the reference of
# every GPU parity test on a larger graph (Lemma 1's z = (I + L)^{-1} s).  Its
# update and its stopping residual share the degree and weight code, so a
# slip common to both would go unseen by the residual alone: these pins judge
# it against LU and against a library sparse solve instead.

def weighted_ba(n, directed, seed):
    """BA graph with U(0.5, 1.5) FP32 weights; directed: each edge oriented at random."""
    g = W.ba_graph(n, 5, seed_off=seed)
    rng = np.random.default_rng(seed)
    a, b = g["src"].astype(np.int32), g["dst"].astype(np.int32)
    wt = (0.5 + rng.random(a.shape[0])).astype(np.float32)
    if directed:
        flip = rng.random(a.shape[0]) < 0.5
        a, b = np.where(flip, b, a), np.where(flip, a, b)
        return oracle.csr_from_arcs(n, a, b, wt)
    return oracle.csr_from_arcs(n, np.concatenate([a, b]), np.concatenate([b, a]), np.concatenate([wt, wt]))


@pytest.mark.parametrize("directed,omega", [(False, 1.0), (True, 1.0), (False, 1.5), (True, 1.2)])
def test_truth_sweep_branch_matches_lu(directed, omega):
    n = 1500
    rp, col, w = weighted_ba(n, directed, seed=31 + 2 * directed)
    s = np.random.default_rng(9).random(n)
    z_sor, res = oracle.truth(n, rp, col, w, s, omega=omega, force_sor=True)
    z_lu = oracle.lu_solve(n, rp, col, w, s)
    assert res <= 1e-12
    np.testing.assert_allclose(z_sor, z_lu, rtol=0, atol=1e-12)
    # the residual it reports is the residual of what it returns, up to the
    # rounding of its plain FP64 row sums: gamma_{deg+2} times the row's magnitudes
    r = oracle.residual_accurate(n, rp, col, w, s, z_sor)
    d = oracle.out_degree(n, rp, w)
    deg = np.diff(rp)
    rows = np.repeat(np.arange(n), deg)
    mag = (1 + d) * np.abs(z_sor) + np.bincount(rows, weights=np.asarray(w, np.float64) * np.abs(z_sor[col]),
                                                minlength=n) + np.abs(s)
    gam = (deg + 2) * 2.0 ** -53 / (1 - (deg + 2) * 2.0 ** -53)
    assert abs(float(np.max(np.abs(r))) - res) <= float(np.max(gam * mag))


def test_truth_sweep_branch_matches_library_solve_at_20k():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    n = 20000
    rp, col, w = weighted_ba(n, True, seed=47)
    s = np.random.default_rng(10).random(n)
    z_t, res = oracle.truth(n, rp, col, w, s)  # n > 2000: the sweep branch
    A = scipy_sparse.csr_matrix((np.asarray(w, np.float64), col, rp), shape=(n, n))
    d = np.asarray(A.sum(axis=1)).ravel()
    M = (scipy_sparse.identity(n) + scipy_sparse.diags(d) - A).tocsr()
    # a direct factorisation fills in badly on a power-law graph, so the library
    # side is Jacobi-preconditioned GMRES with a few steps of iterative refinement
    P = scipy_sparse.diags(1.0 / (1.0 + d))
    z_lib = np.zeros(n)
    for _ in range(4):
        dz, info = spla.gmres(M, s - M @ z_lib, rtol=1e-12, atol=0, restart=200, maxiter=50, M=P)
        assert info == 0
        z_lib = z_lib + dz
    dmax = float(np.max(d))
    tol = max(1e-13, 4e-15 * (1.0 + dmax))
    assert res <= tol
    # both are within their residual of z*: ||(I + L)^{-1}||_inf <= 1
    r_lib = float(np.max(np.abs(s - M @ z_lib)))
    np.testing.assert_allclose(z_t, z_lib, rtol=0, atol=tol + r_lib + 1e-14)
    r = oracle.residual_accurate(n, rp, col, w, s, z_t)
    assert float(np.max(np.abs(r))) <= tol * (1 + 1e-9)


def test_truth_sweep_branch_planted_degree_slip_is_caught():
    # the same sweeps with the in-degree in place of the out-degree (a slip the
    # inline residual would share) converge to another vector, which the LU
    # comparison above rejects; here the slip is made in numpy on the side
    n = 400
    rp, col, w = weighted_ba(n, True, seed=53)
    s = np.random.default_rng(11).random(n)
    z_lu = oracle.lu_solve(n, rp, col, w, s)
    rows = np.repeat(np.arange(n), np.diff(rp))
    wa = np.asarray(w, np.float64)
    din = np.bincount(col, weights=wa, minlength=n)
    z = np.zeros(n)
    for _ in range(400):
        for v in range(n):
            k0, k1 = rp[v], rp[v + 1]
            z[v] = (s[v] + float(np.dot(wa[k0:k1], z[col[k0:k1]]))) / (1.0 + din[v])
    assert np.max(np.abs(z - z_lu)) > 1e-6
    z_sor, _ = oracle.truth(n, rp, col, w, s, force_sor=True)
    assert np.max(np.abs(z_sor - z_lu)) <= 1e-12
    del rows


# ------------------------------------------------------------ push lemmas

def small_ba(n=1500, directed=False):
    g = W.ba_graph(n, 5, seed_off=90)
    if directed:
        rp, col, w = oracle.csr_from_arcs(n, g["src"], g["dst"])
    else:
        a, b, _ = W.symmetrize_arcs(g["src"], g["dst"])
        rp, col, w = oracle.csr_from_arcs(n, a, b)
    return n, rp, col, w, g["S"][0]


@pytest.mark.parametrize("directed", [False, True])
def test_lemma4_one_sided_bound(directed):
    n, rp, col, w, s = small_ba(directed=directed)
    eps = 1e-3
    z_star = oracle.lu_solve(n, rp, col, w, s)
    z, r, pushes, upd, ok = oracle.blisor_fifo(n, rp, col, w, s, eps, 1.0)
    c_eff, epsp = oracle.shift_params(s, eps)
    zp, zsp = z + c_eff, z_star + c_eff
    assert ok and np.all(r >= 0)
    assert np.all(zp <= zsp + 1e-14)
    assert np.all((1 - epsp) * zsp <= zp + 1e-14)
    # termination condition of Alg. 1
    assert np.all(r <= epsp * (s + c_eff))


@pytest.mark.parametrize("omega", [0.7, 1.5, 1.9])
def test_lemma5_two_sided_bound(omega):
    n, rp, col, w, s = small_ba()
    eps = 1e-4
    z_star = oracle.lu_solve(n, rp, col, w, s)
    z, r, pushes, upd, ok = oracle.blisor_fifo(n, rp, col, w, s, eps, omega)
    c_eff, epsp = oracle.shift_params(s, eps)
    assert ok
    assert np.all(np.abs(r) <= epsp * (s + c_eff))
    assert np.all(np.abs(z - z_star) <= epsp * (z_star + c_eff) + 1e-14)


@pytest.mark.parametrize("omega", [1.0, 1.4])
def test_lemma3_invariant(omega):
    n, rp, col, w, s = small_ba(directed=True)
    z, r, *_ = oracle.blisor_fifo(n, rp, col, w, s, 1e-5, omega)
    c_eff, _ = oracle.shift_params(s, 1e-5)
    resid = oracle.residual(n, rp, col, w, s + c_eff, z + c_eff)
    np.testing.assert_allclose(resid, r, rtol=0, atol=1e-12)
    # and the sign of an uncancelled mistake: flipping the residual breaks it
    assert np.max(np.abs(resid + r)) > 1e-9


@pytest.mark.parametrize("directed,weighted", [(False, False), (True, True)])
def test_theorem2_single_pass_is_one_gs_sweep(directed, weighted):
    n = 400
    rp, col, w = random_graph(n, 0.02, directed, weighted, seed=21)
    s = np.random.default_rng(2).random(n)
    # c = 0 and a single pass: Alg. 1 with the initial queue 0..n-1 and no appends
    z_push = oracle.blisor_fifo(n, rp, col, w, s, 0.5, 1.0, c=0.0, single_pass=True)[0]
    z_gs = oracle.gs_sweep_from_zero(n, rp, col, w, s)
    assert np.array_equal(z_push, z_gs)


def test_round_schedule_meets_same_bound():
    n, rp, col, w, s = small_ba()
    eps = 1e-5
    z_star = oracle.lu_solve(n, rp, col, w, s)
    c_eff, epsp = oracle.shift_params(s, eps)
    z, r, pushes, upd, rounds, ok = oracle.push_rounds(n, rp, col, w, s, eps, 1.0)
    assert ok and rounds > 1
    assert np.all(np.abs(r) <= epsp * (s + c_eff))
    assert np.all(np.abs(z - z_star) <= epsp * (z_star + c_eff) + 1e-14)


@pytest.mark.parametrize("directed,weighted", [(False, False), (True, True)])
@pytest.mark.parametrize("threads", [1, 2, 5, 16])
def test_threaded_rounds_equal_sequential_rounds(directed, weighted, threads):
    """The all-core baseline's threaded rounds are the sequential rounds: every
    row's arithmetic is the same, so z, r and the counts agree bit for bit
    (which also pins them to the LU-checked rounds above); more threads than
    rows and an empty graph included."""
    n = 700
    rp, col, w = random_graph(n, 0.01, directed, weighted, seed=31)
    s = np.random.default_rng(5).random(n)
    seq = oracle.push_rounds(n, rp, col, w, s, 1e-6, 1.0)
    thr = oracle.push_rounds_threads(n, rp, col, w, s, 1e-6, 1.0, threads=threads)
    assert np.array_equal(seq[0], thr[0]) and np.array_equal(seq[1], thr[1])
    assert seq[2:6] == thr[2:6] and thr[6] == threads
    z_star = oracle.lu_solve(n, rp, col, w, s)
    c_eff, epsp = oracle.shift_params(s, 1e-6)
    assert np.all(np.abs(thr[0] - z_star) <= epsp * (z_star + c_eff) + 1e-13)
    # three rows, more threads than rows; and no rows at all
    rp3 = np.array([0, 1, 2, 2], np.int64)
    col3 = np.array([1, 0], np.int32)
    s3 = np.array([0.2, 0.9, 0.5])
    a = oracle.push_rounds(3, rp3, col3, None, s3, 1e-6, 1.0)
    b = oracle.push_rounds_threads(3, rp3, col3, None, s3, 1e-6, 1.0, threads=threads)
    assert np.array_equal(a[0], b[0]) and a[2:6] == b[2:6]
    e = oracle.push_rounds_threads(0, np.zeros(1, np.int64), np.zeros(0, np.int32), None, np.zeros(0), 1e-6,
                                   1.0, threads=threads)
    assert e[0].shape == (0,) and e[2] == 0 and e[5]


def test_signed_opinions_shift():
    n, rp, col, w, s = small_ba(n=800)
    s = 2 * s - 1.0
    eps = 1e-4
    z_star = oracle.lu_solve(n, rp, col, w, s)
    c_eff, epsp = oracle.shift_params(s, eps)
    assert c_eff == pytest.approx(1e-5 - s.min())
    z, r, *_ = oracle.blisor_fifo(n, rp, col, w, s, eps, 1.2)
    assert np.all(np.abs(z - z_star) <= epsp * (z_star + c_eff) + 1e-13)


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("directed", [False, True])
def test_constant_opinions_give_constant_z(directed):
    n, rp, col, w, s = small_ba(n=700, directed=directed)
    s = np.full(n, 0.37)
    for z in (oracle.lu_solve(n, rp, col, w, s),
              oracle.blisor_fifo(n, rp, col, w, s, 1e-12, 1.0)[0]):
        np.testing.assert_allclose(z, 0.37, rtol=0, atol=1e-11)


@pytest.mark.parametrize("directed", [False, True])
def test_z_within_opinion_range(directed):
    n, rp, col, w, s = small_ba(n=900, directed=directed)
    z = oracle.lu_solve(n, rp, col, w, s)
    assert z.min() >= s.min() - 1e-14 and z.max() <= s.max() + 1e-14


def test_undirected_total_opinion_preserved():
    n, rp, col, w, s = small_ba(n=900)
    z = oracle.lu_solve(n, rp, col, w, s)
    assert abs(z.sum() - s.sum()) < 1e-10
    n2, rp2, col2, w2, _ = small_ba(n=900, directed=True)
    z2 = oracle.lu_solve(n2, rp2, col2, w2, s)
    assert abs(z2.sum() - s.sum()) > 1e-6  # fails for directed graphs, as expected


def test_isolated_nodes_keep_their_opinion():
    rp, col, w = csr(5, [(0, 1), (1, 0)])
    s = np.array([0.1, 0.9, 0.3, 0.5, 0.7])
    for z in all_solvers(5, rp, col, w, s):
        np.testing.assert_allclose(z[2:], s[2:], rtol=0, atol=1e-12)


# ------------------------------------------------------------ metrics

def test_metric_identities_undirected():
    n, rp, col, w, s = small_ba()
    z = oracle.lu_solve(n, rp, col, w, s)
    m = oracle.metrics(n, rp, col, w, s, z, directed=False)
    # s = (I+L) z with D = z^T L z and I = ||L z||^2
    assert abs(s @ s - (m["C"] + 2 * m["D"] + m["I"])) < 1e-9
    assert abs(s @ z - (m["C"] + m["D"])) < 1e-9
    assert abs(m["P"] - (m["C"] - n * m["mean_z"] ** 2)) < 1e-9
    assert abs(m["mean_z"] - s.mean()) < 1e-12


def test_metrics_single_edge_closed_form():
    s = np.array([0.2, 0.9])
    rp, col, w = undirected(2, [(0, 1)])
    z = oracle.lu_solve(2, rp, col, w, s)
    m = oracle.metrics(2, rp, col, w, s, z, directed=False)
    g = (s[1] - s[0]) / 3
    assert abs(m["D"] - g * g) < 1e-15
    assert abs(m["I"] - 2 * g * g) < 1e-15
    assert abs(m["C"] - (z[0] ** 2 + z[1] ** 2)) < 1e-15
    assert abs(m["P"] - 2 * (0.5 * (s[1] - s[0]) / 3) ** 2) < 1e-15
    mdir = oracle.metrics(2, rp, col, w, s, z, directed=True)
    assert abs(mdir["D"] - 2 * g * g) < 1e-15


# ------------------------------------------------------------ SOR theory

def cycle_red_black(n):
    rp, col, w = undirected(n, [(i, (i + 1) % n) for i in range(n)])
    order = np.concatenate([np.arange(0, n, 2), np.arange(1, n, 2)]).astype(np.int32)
    return rp, col, w, order


@pytest.mark.parametrize("omega", [1.0, 1.3, 1.6])
def test_sor_rate_on_consistently_ordered_cycle(omega):
    # 2-regular bipartite: mu = rho((I+D)^{-1} A) = 2/3.  For a red-black order
    # Young's theory gives the asymptotic rate mu^2 at omega = 1 and omega - 1
    # for omega >= omega_opt = 1 + (mu / (1 + sqrt(1 - mu^2)))^2 (Eq. 17).
    n = 64
    rp, col, w, order = cycle_red_black(n)
    s = np.random.default_rng(4).random(n)
    z_star = oracle.lu_solve(n, rp, col, w, s)
    mu = 2.0 / 3.0
    omega_opt = 1 + (mu / (1 + np.sqrt(1 - mu * mu))) ** 2
    want = mu * mu if omega == 1.0 else omega - 1.0
    assert omega == 1.0 or omega >= omega_opt
    # windows inside the asymptotic regime and above the FP64 error floor
    k0, k1 = {1.0: (10, 30), 1.3: (8, 24), 1.6: (10, 50)}[omega]
    errs = []
    for k in (k0, k1):
        z = oracle.sor_ordered(n, rp, col, w, s, order, 1e-300, omega, c=0.0, max_sweeps=k)[0]
        errs.append(np.linalg.norm(z - z_star))
    rate = (errs[1] / errs[0]) ** (1 / (k1 - k0))
    assert abs(rate - want) < 0.02 * want + 0.01


# ------------------------------------------------------------ colouring

def test_greedy_colouring_properties():
    g = W.rmat_directed(12)
    rp, col, w = oracle.csr_from_arcs(g["n"], g["src"], g["dst"], g["w"])
    colour, k = oracle.greedy_colour(g["n"], rp, col)
    rows = np.repeat(np.arange(g["n"]), np.diff(rp))
    assert np.all(colour[rows] != colour[col])  # proper on every arc
    sp, sc = oracle.symmetric_pattern(g["n"], rp, col)
    assert k <= np.diff(sp).max() + 1
    assert colour.min() == 0 and colour.max() == k - 1


def test_greedy_colour_counts_on_known_graphs():
    n = 6
    rp, col, w = undirected(n, [(a, b) for a in range(n) for b in range(a + 1, n)])
    assert oracle.greedy_colour(n, rp, col)[1] == n
    # even cycle coloured greedily in natural order needs exactly 2 colours
    rp, col, w = undirected(10, [(i, (i + 1) % 10) for i in range(10)])
    sp, sc = oracle.symmetric_pattern(10, rp, col)
    colour = np.empty(10, np.int32)
    k = oracle._lib().oracle_greedy_colour(10, oracle._p(np.ascontiguousarray(sp)),
                                           oracle._p(np.ascontiguousarray(sc)),
                                           oracle._p(np.arange(10, dtype=np.int32)),
                                           oracle._p(colour))
    assert k == 2 and list(colour) == [0, 1] * 5


def test_priority_hash_is_splitmix64():
    # published SplitMix64 test vector: state 0 gives 0xE220A8397B1DCDAF as first output
    assert int(oracle.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF


# ------------------------------------------------------------ graph ingest

def test_csr_from_arcs_brute_force():
    rng = np.random.default_rng(7)
    n = 50
    src = rng.integers(0, n, 3000).astype(np.int32)
    dst = rng.integers(0, n, 3000).astype(np.int32)
    w = rng.random(3000).astype(np.float32)
    rp, col, wc = oracle.csr_from_arcs(n, src, dst, w)
    first = {}
    for e in range(3000):
        if src[e] != dst[e] and (src[e], dst[e]) not in first:
            first[(src[e], dst[e])] = w[e]
    keys = sorted(first)
    assert rp[-1] == len(keys)
    for u in range(n):
        row = [(u, int(c)) for c in col[rp[u]:rp[u + 1]]]
        assert row == [k for k in keys if k[0] == u]
        assert list(wc[rp[u]:rp[u + 1]]) == [first[k] for k in row]


@pytest.mark.parametrize("weighted", [False, True])
def test_csr_build_routes_agree(weighted):
    """The C and numpy constructions of the same definition agree bit for bit on
    arc lists with many repeats and self-loops (R-MAT at scale 13)."""
    g = W.rmat_directed(13)
    w = g["w"] if weighted else None
    a = oracle.csr_from_arcs(g["n"], g["src"], g["dst"], w)
    b = oracle.csr_from_arcs_np(g["n"], g["src"], g["dst"], w)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    if weighted:
        assert np.array_equal(a[2], b[2])
    assert a[0][-1] < g["src"].shape[0]  # repeats were dropped


def test_transpose_brute_force():
    rng = np.random.default_rng(9)
    n = 40
    rp, col, w = oracle.csr_from_arcs(n, rng.integers(0, n, 500), rng.integers(0, n, 500),
                                      rng.random(500).astype(np.float32))
    tp, tc, tw = oracle.transpose(n, rp, col, w)
    for v in range(n):
        want = [(u, w[k]) for u in range(n) for k in range(rp[u], rp[u + 1]) if col[k] == v]
        assert list(zip(tc[tp[v]:tp[v + 1]].tolist(), tw[tp[v]:tp[v + 1]].tolist())) == want


def test_degree_sums_are_exact_in_fp64():
    g = W.rmat_directed(14)
    rp, col, w = oracle.csr_from_arcs(g["n"], g["src"], g["dst"], g["w"])
    d = oracle.out_degree(g["n"], rp, w)
    # FP32 weights in [0.5, 1.5] are multiples of 2^-24: every partial sum is exact
    assert np.all(d * 2.0 ** 24 == np.round(d * 2.0 ** 24))
    rev = np.array([np.sum(w[rp[u]:rp[u + 1]][::-1].astype(np.float64)) for u in range(0, g["n"], 97)])
    assert np.array_equal(rev, d[::97])


def _exact_residual(n, rp, col, w, s, z):
    """s - (I + L) z over the rationals (every FP64 input is an exact rational)."""
    out = []
    for v in range(n):
        acc = Fraction(float(s[v])) - Fraction(float(z[v]))
        for k in range(int(rp[v]), int(rp[v + 1])):
            a = Fraction(float(w[k])) if w is not None else Fraction(1)
            acc += a * (Fraction(float(z[int(col[k])])) - Fraction(float(z[v])))
        out.append(acc)
    return out


@pytest.mark.parametrize("weighted", [False, True])
def test_accurate_residual_matches_rational_arithmetic(weighted):
    """Dot2 residual = the exact residual rounded, within 2 ulp, even where a plain
    FP64 row sum loses every digit (s built so that the residual is one rounding)."""
    rng = np.random.default_rng(7)
    n = 40
    arcs, ws = [], []
    for u in range(n):
        deg = 400 if u == 0 else int(rng.integers(0, 6))  # one hub row
        for v in rng.choice(np.arange(1, n), size=min(deg, n - 1), replace=deg > n - 1):
            if v != u:
                arcs.append((u, int(v)))
                ws.append(float(np.float32(0.5 + rng.random())))
    src = np.array([a for a, _ in arcs], np.int32)
    dst = np.array([b for _, b in arcs], np.int32)
    rp, col, w = oracle.csr_from_arcs(n, src, dst, np.array(ws, np.float32) if weighted else None)
    # hub rows repeat columns only through the arc list; csr_from_arcs keeps one copy each
    z = 1.0 + rng.random(n) * 1e-3
    # s_v = round((I + L) z)_v: the exact residual is only s's rounding error
    exact_lz = _exact_residual(n, rp, col, w, np.zeros(n), z)
    s = np.array([float(-x) for x in exact_lz])
    want = _exact_residual(n, rp, col, w, s, z)
    got = oracle.residual_accurate(n, rp, col, w, s, z)
    plain = oracle.residual(n, rp, col, w, s, z)
    u = 2.0 ** -53
    for v in range(n):
        wv = float(want[v])
        assert abs(got[v] - wv) <= 4 * u * abs(wv) + 1e-300, (v, got[v], wv)
    # the plain sum is off by far more than the residual itself at the hub
    assert abs(plain[0] - float(want[0])) > 10 * abs(float(want[0])) or float(want[0]) == 0.0
    # generic inputs: also within 2 ulp of the rational value
    s2 = rng.random(n)
    want2 = _exact_residual(n, rp, col, w, s2, z)
    got2 = oracle.residual_accurate(n, rp, col, w, s2, z)
    for v in range(n):
        assert abs(got2[v] - float(want2[v])) <= 4 * u * abs(float(want2[v])) + 1e-300


def test_empty_and_edgeless_graphs():
    rp = np.zeros(4, np.int64)
    col = np.zeros(0, np.int32)
    s = np.array([0.3, 0.0, 1.0])
    z, r, p, u, ok = oracle.blisor_fifo(3, rp, col, None, s, 1e-6, 1.0)
    np.testing.assert_allclose(z, s, atol=1e-15)
    assert oracle.metrics(3, rp, col, None, s, z, False)["D"] == 0.0


# ------------------------------------------------------------ palette colouring

def test_palette_colouring_reduces_to_greedy_and_constant():
    g = W.rmat_directed(11)
    rp, col, w = oracle.csr_from_arcs(g["n"], g["src"], g["dst"], g["w"])
    c0, k0 = oracle.greedy_colour(g["n"], rp, col)
    c1, k1, din = oracle.palette_colour(g["n"], rp, col, w, True, 32 if k0 <= 32 else k0)
    assert k1 == k0 and np.array_equal(c0, c1) and np.all(din == 0)
    c2, k2, din2 = oracle.palette_colour(g["n"], rp, col, w, True, 1)
    assert k2 == 1 and np.all(c2 == 0)
    # with one colour every neighbour is in class: the in-class weight is the whole symmetric degree
    sp_, sc_, sw_, sq_ = oracle.symmetric_weights(g["n"], rp, col, w, True)
    rows = np.repeat(np.arange(g["n"]), np.diff(sp_))
    np.testing.assert_allclose(din2, np.bincount(rows, weights=sw_, minlength=g["n"]))


def test_palette_colouring_least_conflict_rule_brute_force():
    rng = np.random.default_rng(5)
    n = 60
    rp, col, w = random_graph(n, 0.25, True, True, seed=8)
    K = 3
    colour, k, din = oracle.palette_colour(n, rp, col, w, True, K)
    sp_, sc_, sw_, sq_ = oracle.symmetric_weights(n, rp, col, w, True)
    order = oracle.colour_priority_order(n, sp_)
    pos = np.empty(n, np.int64)
    pos[order] = np.arange(n)
    for v in range(n):
        conf = np.zeros(K, np.int64)
        for kk in range(sp_[v], sp_[v + 1]):
            u = sc_[kk]
            if pos[u] < pos[v]:
                conf[colour[u]] += sq_[kk]
        zero = np.flatnonzero(conf == 0)
        want = zero[0] if len(zero) else int(np.argmin(conf))
        assert colour[v] == want
    # fixed-point weights of a pair sum both arcs
    assert np.all(sq_ == np.rint(sw_ * 2.0 ** 32).astype(np.int64))


def test_safe_omega_keeps_split_diagonally_dominant():
    d = np.array([0.0, 3.0, 10.0, 5.0])
    din = np.array([0.0, 3.0, 2.0, 0.0])
    om = oracle.safe_omega(1.8, d, din)
    assert om[0] == 1.8 and om[3] == 1.8
    assert np.all((2 / om - 1) * (1 + d) >= din - 1e-12)


# ------------------------------------------------------------ spectral radius for Eq. 17

def test_jacobi_radius_complete_graph_closed_form():
    # K_m, unit weights: M = (J - I) / m, whose spectral radius is (m - 1) / m
    m = 9
    rp, col, w = undirected(m, [(i, j) for i in range(m) for j in range(i + 1, m)])
    assert abs(oracle.jacobi_radius_power(m, rp, col, w, 5) - (m - 1) / m) < 1e-14


@pytest.mark.parametrize("directed", [False, True])
def test_jacobi_radius_matches_dense_eigenvalues(directed):
    rng = np.random.default_rng(21 if directed else 22)
    n = 60
    arcs = {(int(u), int(v)) for u, v in rng.integers(0, n, (400, 2)) if u != v}
    if not directed:
        arcs |= {(v, u) for u, v in arcs}
    arcs = sorted(arcs)
    src = np.array([a for a, _ in arcs], np.int32)
    dst = np.array([b for _, b in arcs], np.int32)
    wt = (0.5 + rng.random(len(arcs))).astype(np.float32)
    if not directed:
        wt = np.array([wt[min(i, arcs.index((b, a)))] for i, (a, b) in enumerate(arcs)], np.float32)
    rp, col, w = oracle.csr_from_arcs(n, src, dst, wt)
    dense = oracle.dense_i_plus_l(n, rp, col, w)
    dg = np.diag(dense)
    m = (np.diag(dg) - dense) / dg[:, None]  # (I + D)^{-1} A
    mu = max(abs(np.linalg.eigvals(m)))
    assert abs(oracle.jacobi_radius_power(n, rp, col, w, 3000) - mu) < 1e-9


def test_jacobi_radius_bipartite_path():
    # a path is bipartite, so M's spectrum is symmetric (+-mu) and plain power
    # iteration on M would alternate; the shifted iteration converges to mu
    n = 12
    rp, col, w = undirected(n, [(i, i + 1) for i in range(n - 1)])
    dense = oracle.dense_i_plus_l(n, rp, col, w)
    dg = np.diag(dense)
    ev = np.linalg.eigvals((np.diag(dg) - dense) / dg[:, None])
    mu = max(abs(ev))
    assert np.min(np.abs(ev + mu)) < 1e-12  # -mu is an eigenvalue too
    assert abs(oracle.jacobi_radius_power(n, rp, col, w, 4000) - mu) < 1e-10


def test_omega_opt_is_youngs_formula():
    # Eq. 17 written as 1 + (mu / (1 + sqrt(1 - mu^2)))^2 equals 2 / (1 + sqrt(1 - mu^2))
    for mu in (0.0, 0.3, 2.0 / 3.0, 0.9, 0.999):
        assert abs(oracle.omega_opt(mu) - 2.0 / (1.0 + np.sqrt(1.0 - mu * mu))) < 1e-15


# ------------------------------------------------------------ multicolour row order

@pytest.mark.parametrize("cap", [5, 12, 1000])
def test_sweep_order_brute_force(monkeypatch, cap):
    """The row order against a brute-force restatement: the hub set is the
    largest in-degree threshold set of at most cap nodes, and every range is
    sorted by (colour, in-degree descending, id)."""
    monkeypatch.setattr(oracle, "HUB_CAPACITY", cap)
    rng = np.random.default_rng(17)
    n = 40
    arcs = [(int(a), int(b)) for a, b in rng.integers(0, n, (160, 2)) if a != b]
    rp, col, _ = csr(n, arcs)
    colour = rng.integers(0, 4, n).astype(np.int32)
    perm, nhub, hub_row, class_row = oracle.sweep_order(n, rp, col, colour, hubs=True)
    indeg = [int(np.sum(col == v)) for v in range(n)]
    assert sorted(perm.tolist()) == list(range(n))
    if n <= cap:
        hubs = set(range(n))
    else:
        hubs = None
        for t in sorted(set(indeg)) + [max(indeg) + 1]:
            cand = {v for v in range(n) if indeg[v] >= t}
            if len(cand) <= cap:
                hubs = cand
                break
    assert nhub == len(hubs) and set(perm[:nhub].tolist()) == hubs
    key = lambda v: (colour[v], -indeg[v], v)
    assert perm[:nhub].tolist() == sorted(hubs, key=key)
    assert perm[nhub:].tolist() == sorted(set(range(n)) - hubs, key=key)
    K = int(colour.max()) + 1
    for c in range(K):
        assert all(colour[v] == c for v in perm[hub_row[c]:hub_row[c + 1]])
        assert all(colour[v] == c for v in perm[class_row[c]:class_row[c + 1]])
    assert hub_row[K] == nhub == class_row[0] and class_row[K] == n
