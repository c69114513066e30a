"""GPU paths beyond the plain solve, each checked against the FP64 oracle.

- The zero start judges a warm start and is its fallback (single vector and
  per vector of a batch): a start whose exact residual sum is not below the
  zero start's is dropped, and the solve certifies as from zero.
- fj_solve_trace: a row's relative residual max_v |r_v| / s'_v equals the
  oracle's, evaluated with compensated sums on the estimate the solve held at
  that point (taken from a solve capped at the same sweep count).
- The FP64 frontier cleanup (scatter-form push rounds on the few entries the
  certificate leaves above threshold) runs and still certifies against truth,
  also when long in-neighbour lists are scattered by a block each.
- Update counts of the GPU schedules against the FIFO push of Alg. 1-3 at
  the same omega (Fig. 2's axis): the same order of magnitude; the counts
  themselves are not pinned (the GPU order differs from the FIFO on purpose).
"""
import numpy as np
import pytest

import oracle
from fjsynth import workloads as W
from gpu_common import FP32_TOL, FP64_TOL, certificate_holds, csr_of, rel_inf, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi as c
    return c


@pytest.fixture(scope="module")
def ba6k():
    g = W.ba_graph(6000, 5, seed_off=71)
    rp, col, w = csr_of(g)
    s = g["S"][0]
    z_star, _ = oracle.truth(g["n"], rp, col, w, s)
    return g, rp, col, w, s, z_star


# ------------------------------------------------------------ warm start and its judge

def test_warm_start_judged_by_zero_start(capi, ba6k):
    g, rp, col, w, s, z_star = ba6k
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    (s_d,) = to_dev(s)
    opts = dict(eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    z_c, ic, _ = G.solve(s_d, **opts)
    assert ic[0]["warm_start"] == -1
    # a good start is kept and saves sweeps
    good = z_star + 1e-4 * np.random.default_rng(1).standard_normal(n)
    z_g, ig, st = G.solve(s_d, z0=to_dev(good)[0], **opts)
    assert st == capi.FJ_OK and ig[0]["warm_start"] == 1 and ig[0]["converged"] == 1
    assert ig[0]["sweeps"] < ic[0]["sweeps"]
    assert rel_inf(z_g.cpu().numpy(), z_star) <= FP32_TOL
    # a bad start (a network with wild output) loses to the zero start: the
    # solve is the zero-start solve, bit for bit
    bad = 40.0 * (np.random.default_rng(2).random(n) - 0.5)
    z_b, ib, st = G.solve(s_d, z0=to_dev(bad)[0], **opts)
    assert st == capi.FJ_OK and ib[0]["warm_start"] == 0 and ib[0]["converged"] == 1
    assert ib[0]["sweeps"] == ic[0]["sweeps"]
    assert np.array_equal(z_b.cpu().numpy(), z_c.cpu().numpy())
    ok, r = certificate_holds(n, rp, col, w, s, z_b.cpu().numpy(), ib[0]["c_eff"], ib[0]["eps_prime"])
    assert ok


def test_warm_start_with_bad_network_falls_back(capi, ba6k):
    """A network with huge random weights: its clamped output jumps between the
    opinion bounds from node to node, a start far worse than zero, so the solve
    falls back and costs what the zero start costs."""
    from oracle import mpnn as ref

    g, rp, col, w, s, z_star = ba6k
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    (s_d,) = to_dev(s)
    theta = (300.0 * ref.init_params(5)).astype(np.float32)
    net = capi.MPNN(theta)
    z0 = net.predict(G, s)
    opts = dict(eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    z_c, ic, _ = G.solve(s_d, **opts)
    z, iw, st = G.solve(s_d, z0=to_dev(z0)[0], **opts)
    assert st == capi.FJ_OK and iw[0]["converged"] == 1
    assert rel_inf(z.cpu().numpy(), z_star) <= FP32_TOL
    # the judge, recomputed by the oracle: residual sums of the two starts
    r0 = oracle.residual_accurate(n, rp, col, w, s, z0)
    assert np.sum(np.abs(r0)) > 2.0 * np.sum(s + iw[0]["c_eff"])  # the start is clearly bad
    assert iw[0]["warm_start"] == 0
    assert iw[0]["sweeps"] == ic[0]["sweeps"]
    assert np.array_equal(z.cpu().numpy(), z_c.cpu().numpy())


def test_batch_warm_start_judged_per_vector(capi):
    g = W.rmat_multirhs(12, 4)
    rp, col, w = csr_of(g)
    n = g["n"]
    S = np.ascontiguousarray(np.stack(g["S"], axis=1))
    Zs = np.stack([oracle.truth(n, rp, col, w, np.ascontiguousarray(S[:, j]))[0] for j in range(4)], axis=1)
    Z0 = Zs + 1e-4 * np.random.default_rng(3).standard_normal(Zs.shape)
    Z0[:, 1] = 30.0 * (np.random.default_rng(4).random(n) - 0.5)  # columns 1 and 3 lose
    Z0[:, 3] = -25.0
    Z0 = np.ascontiguousarray(Z0)
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    opts = dict(eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    Sd, Z0d = to_dev(S, Z0)
    Z, infos, st = G.solve_batch(Sd, Z0=Z0d, **opts)
    assert st == capi.FJ_OK
    assert [i["warm_start"] for i in infos] == [1, 0, 1, 0]
    Z = Z.cpu().numpy()
    for j in range(4):
        assert infos[j]["converged"] == 1
        assert rel_inf(Z[:, j], Zs[:, j]) <= FP32_TOL, j


# ------------------------------------------------------------ trace rows against the oracle

def test_trace_rows_match_oracle_residual(capi):
    """Rows after 8 and 16 sweeps: the relative residual of the estimate at that
    point, recomputed by the oracle from the z of a solve capped there."""
    g = W.rmat_directed(12, seed_off=73)
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=True)
    (s_d,) = to_dev(s)
    opts = dict(eps=1e-6, omega=1.5, palette=8, precision=capi.FJ_PREC_FP64, check_every=8)
    _, info, st, tr = G.solve_trace(s_d, **opts)
    assert st == capi.FJ_OK
    rows0 = tr[tr[:, 3] == 0.0]
    checked = 0
    for sw in (8, 16):
        row = rows0[rows0[:, 1] == sw]
        if row.shape[0] == 0:
            continue
        z, inf, st = G.solve(s_d, max_sweeps=sw, max_refine=0, allow_unconverged=True, **opts)
        if inf[0]["frontier_rounds"] > 0:
            continue  # the capped solve went on to the cleanup: not the state of the row
        zc = z.cpu().numpy()
        ce = inf[0]["c_eff"]
        r = oracle.residual_accurate(n, rp, col, w, s, zc)
        rel = float(np.max(np.abs(r) / (s + ce)))
        assert row[0, 2] == pytest.approx(rel, rel=1e-6, abs=1e-12), (sw, row[0, 2], rel)
        checked += 1
    assert checked >= 1
    # the last row is the final certificate of the returned z
    z, inf, _ = G.solve(s_d, **opts)
    r = oracle.residual_accurate(n, rp, col, w, s, z.cpu().numpy())
    rel = float(np.max(np.abs(r) / (s + inf[0]["c_eff"])))
    assert tr[-1, 3] == 1.0 and tr[-1, 2] == pytest.approx(rel, rel=1e-6, abs=1e-15)


# ------------------------------------------------------------ FP64 frontier cleanup

def test_frontier_cleanup_runs_and_certifies(capi):
    """Small graphs end their FP32 pass with few entries above the FP64
    threshold, which the scatter-form FP64 push clears."""
    ran = 0
    for seed_off, n in ((81, 1500), (82, 3000), (83, 5000)):
        g = W.ba_graph(n, 4, seed_off=seed_off)
        rp, col, w = csr_of(g)
        s = g["S"][0]
        z_star, _ = oracle.truth(n, rp, col, w, s)
        G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
        (s_d,) = to_dev(s)
        for prec, tol in ((capi.FJ_PREC_FP32, FP32_TOL), (capi.FJ_PREC_FP64, FP64_TOL)):
            z, info, st = G.solve(s_d, eps=1e-6, omega=1.5, precision=prec)
            i0 = info[0]
            assert st == capi.FJ_OK and i0["converged"] == 1
            assert rel_inf(z.cpu().numpy(), z_star) <= tol
            ok, _ = certificate_holds(n, rp, col, w, s, z.cpu().numpy(), i0["c_eff"], i0["eps_prime"])
            assert ok
            if i0["frontier_rounds"] > 0:
                assert i0["frontier_pushes"] > 0 and i0["frontier_edges"] > 0
                ran += 1
    assert ran >= 1, "no solve reached the frontier cleanup"


def _hub_graph(n, hubs, seed_off):
    """BA(n, 4) plus `hubs` extra nodes joined to every BA node: each hub's
    in-neighbour list (n entries) is longer than the block-scatter threshold."""
    g = W.ba_graph(n, 4, seed_off=seed_off)
    hs = np.repeat(np.arange(n, n + hubs, dtype=np.int32), n)
    hd = np.tile(np.arange(n, dtype=np.int32), hubs)
    src = np.concatenate([g["src"], hs])
    dst = np.concatenate([g["dst"], hd])
    a, b, c = W.symmetrize_arcs(src, dst, None)
    nt = n + hubs
    rp, col, w = oracle.csr_from_arcs(nt, a, b, c)
    rng = np.random.default_rng(9000 + seed_off)
    s = np.concatenate([g["S"][0], rng.uniform(0.0, 1.0, hubs)])
    return nt, rp, col, w, s


@pytest.mark.parametrize("long_min", ["0", None])
def test_frontier_long_scatter(capi, monkeypatch, long_min):
    """The frontier round's long in-neighbour lists go to one block each
    (FJ_FRONTIER_LONG=0 sends every entry there, and these solves must reach
    the cleanup; under the default the hubs of these graphs would go there if
    a frontier holds them); results still certify and match truth."""
    if long_min is None:
        monkeypatch.delenv("FJ_FRONTIER_LONG", raising=False)
    else:
        monkeypatch.setenv("FJ_FRONTIER_LONG", long_min)
    ran = 0
    cases = [(85, 5000, 3), (86, 6000, 2)] if long_min is None else [(81, 1500, 0), (83, 5000, 0), (85, 5000, 3)]
    for seed_off, n, hubs in cases:
        if hubs:
            nt, rp, col, w, s = _hub_graph(n, hubs, seed_off)
        else:
            g = W.ba_graph(n, 4, seed_off=seed_off)
            rp, col, w = csr_of(g)
            nt, s = n, g["S"][0]
        z_star, _ = oracle.truth(nt, rp, col, w, s)
        G = capi.Graph.from_csr(nt, *to_dev(rp, col, w), directed=False)
        (s_d,) = to_dev(s)
        for prec, tol in ((capi.FJ_PREC_FP32, FP32_TOL), (capi.FJ_PREC_FP64, FP64_TOL)):
            for omega in (1.0, 1.5):
                z, info, st = G.solve(s_d, eps=1e-6, omega=omega, precision=prec)
                i0 = info[0]
                assert st == capi.FJ_OK and i0["converged"] == 1
                assert rel_inf(z.cpu().numpy(), z_star) <= tol
                ok, _ = certificate_holds(nt, rp, col, w, s, z.cpu().numpy(), i0["c_eff"], i0["eps_prime"])
                assert ok
                ran += i0["frontier_rounds"] > 0
    if long_min == "0":  # the hub graphs need not leave a frontier at all
        assert ran >= 1, "no solve reached the frontier cleanup"


# ------------------------------------------------------------ certificate against the exact residual

def _oracle_stats(n, rp, col, w, s, z):
    """max_v |r_v| and max_v |r_v| / s'_v of the exact residual of z."""
    ce = oracle.shift_params(s, 1e-6)[0]
    r = oracle.residual_accurate(n, rp, col, w, s, z)
    return float(np.max(np.abs(r))), float(np.max(np.abs(r) / (s + ce)))


@pytest.mark.parametrize("kind", ["hubs", "weighted"])
def test_certificate_statistics_equal_exact_residual(capi, kind):
    """The certificate's reported max |r| and max |r|/s' equal the oracle's
    compensated residual of the returned z, on solves stopped early (large
    residuals, decided mostly far from the threshold).  The hub graph's rows of
    5000 nonzeros and the weighted R-MAT's long rows are summed by the
    certificate's 128-bit fixed-point chunks (with the product's FMA error on
    the weighted graph); the hub rows carry the largest residuals."""
    if kind == "hubs":
        n, rp, col, w, s = _hub_graph(5000, 3, 87)
        directed = False
    else:
        g = W.rmat_directed(13, seed_off=88)
        rp, col, w = csr_of(g)
        n, s, directed = g["n"], g["S"][0], True
    assert int(np.max(np.diff(rp))) > 512  # long rows present
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=directed)
    (s_d,) = to_dev(s)
    for prec in (capi.FJ_PREC_FP32, capi.FJ_PREC_FP64):
        for sw in (2, 6, 12):
            z, inf, st = G.solve(s_d, eps=1e-6, omega=1.5, precision=prec, max_sweeps=sw, max_refine=0,
                                 allow_unconverged=True)
            a, rel = _oracle_stats(n, rp, col, w, s, z.cpu().numpy())
            i0 = inf[0]
            assert i0["resid_inf"] == pytest.approx(a, rel=1e-9, abs=1e-15), (prec, sw)
            assert i0["resid_rel_max"] == pytest.approx(rel, rel=2e-6), (prec, sw)
    # the batch certificate, per vector
    rng = np.random.default_rng(89)
    k = 4
    S = np.stack([s, rng.random(n), 1.0 - s, rng.random(n) ** 3], axis=1)
    (S_d,) = to_dev(np.ascontiguousarray(S))
    Z, infos, st = G.solve_batch(S_d, eps=1e-6, omega=1.5, max_sweeps=6, max_refine=0, allow_unconverged=True)
    Zh = Z.cpu().numpy()
    for j in range(k):
        a, rel = _oracle_stats(n, rp, col, w, S[:, j], Zh[:, j])
        assert infos[j]["resid_inf"] == pytest.approx(a, rel=1e-9, abs=1e-15), j
        assert infos[j]["resid_rel_max"] == pytest.approx(rel, rel=2e-6), j


# ------------------------------------------------------------ update counts (Fig. 2's axis)

@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_update_counts_track_the_fifo_push(capi, ba6k, omega):
    g, rp, col, w, s, _ = ba6k
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    (s_d,) = to_dev(s)
    _, info, st = G.solve(s_d, eps=1e-6, omega=omega, precision=capi.FJ_PREC_FP64)
    assert st == capi.FJ_OK
    _, _, pushes, updates, ok = oracle.blisor_fifo(n, rp, col, w, s, 1e-6, omega)
    assert ok
    ratio = info[0]["edges"] / updates
    assert 0.5 <= ratio <= 2.0, (info[0]["edges"], updates)


# ------------------------------------------------------------ row order (locality) and relabelling

@pytest.mark.parametrize("name,K", [("rmat16_dir", 8), ("rmat16_und", 16), ("ba3k", 16), ("rmat12_und", 0)])
def test_sweep_order_matches_oracle(capi, name, K):
    """The multicolour row order with its hub prefix, bit for bit."""
    if name == "rmat16_dir":
        g = W.rmat_directed(16)
    elif name == "rmat16_und":
        g = W.rmat_undirected(16)
    elif name == "rmat12_und":
        g = W.rmat_undirected(12)
    else:
        g = W.ba_graph(3000, 4, seed_off=84)
    rp, col, w = csr_of(g)
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=g["directed"])
    perm, nhub, hub_row, class_row = G.order(K)
    if K > 0:
        colour, _, _ = oracle.palette_colour(n, rp, col, w, g["directed"], K)
    else:
        colour, _ = oracle.greedy_colour(n, rp, col)
    perm_o, nhub_o, hr_o, cr_o = oracle.sweep_order(n, rp, col, colour, hubs=K > 0)
    assert nhub == nhub_o
    assert np.array_equal(perm, perm_o)
    assert np.array_equal(hub_row, hr_o) and np.array_equal(class_row, cr_o)


def test_relabelled_graph_gives_permuted_solution(capi):
    """Solving the same graph under a random relabelling changes the row order
    (ties are broken by id) but not the result: z is the relabelled z*."""
    g = W.rmat_directed(13, seed_off=85)
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    z_star, _ = oracle.truth(n, rp, col, w, s)
    pi = np.random.default_rng(5).permutation(n).astype(np.int32)  # new id of node v is pi[v]
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))
    rp2, col2, w2 = oracle.csr_from_arcs(n, pi[src], pi[col], w)
    s2 = np.empty(n)
    s2[pi] = s
    opts = dict(eps=1e-6, omega=1.5, palette=8, precision=capi.FJ_PREC_FP32)
    G1 = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=True)
    G2 = capi.Graph.from_csr(n, *to_dev(rp2, col2, w2), directed=True)
    z1, i1, _ = G1.solve(to_dev(s)[0], **opts)
    z2, i2, _ = G2.solve(to_dev(s2)[0], **opts)
    assert i1[0]["converged"] == 1 and i2[0]["converged"] == 1
    z1 = z1.cpu().numpy()
    z2 = z2.cpu().numpy()[pi]  # back to the first labelling
    assert rel_inf(z1, z_star) <= FP32_TOL and rel_inf(z2, z_star) <= FP32_TOL
    # the two row orders, in the first labelling, differ (the sweep order moved)
    o1 = G1.order(8)[0]
    inv_pi = np.empty(n, np.int32)
    inv_pi[pi] = np.arange(n, dtype=np.int32)
    o2 = inv_pi[G2.order(8)[0]]
    assert not np.array_equal(o1, o2)
