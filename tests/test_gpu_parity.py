"""GPU path against the FP64 oracle, through the C ABI.

Bit-exact: graph ingest (CSR from arcs, transpose, FP64 degrees), the push
frontier F = {v : |r_v| > h_v}, the greedy colouring.  Within tolerance: z
against the oracle's certified truth (1e-6 FP64 path, 1e-5 FP32 paths, as the
relative max-norm error), the metrics (1e-5 relative against the oracle's
metrics of the exact z; 1e-12 against the oracle's metrics of the same z).
"""
import numpy as np
import pytest

import oracle
from fjsynth import workloads as W
from gpu_common import FP32_TOL, FP64_TOL, METRIC_TOL, certificate_holds, csr_of, rel_inf, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi as c
    return c


# ------------------------------------------------------------ graph ingest

@pytest.mark.parametrize("scale,directed", [(12, True), (13, False)])
def test_ingest_from_arcs_bit_exact(capi, scale, directed):
    if directed:
        g = W.rmat_directed(scale)
        src, dst, w = g["src"], g["dst"], g["w"]
    else:
        g = W.rmat_undirected(scale)
        src, dst, w = W.symmetrize_arcs(g["src"], g["dst"], None)
    n = g["n"]
    rp, col, wc = oracle.csr_from_arcs(n, src, dst, w)
    G = capi.Graph.from_arcs(n, *to_dev(src, dst, w), directed=directed)
    grp, gcol, gw, gdeg = G.export(weights=w is not None)
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    if w is not None:
        assert np.array_equal(gw, wc)
    assert np.array_equal(gdeg, oracle.out_degree(n, rp, wc))
    if directed:
        tp, tc, tw = oracle.transpose(n, rp, col, wc)
        trp, tcol, tww, _ = G.export(transposed=True)
        assert np.array_equal(trp, tp) and np.array_equal(tcol, tc) and np.array_equal(tww, tw)


def test_ingest_from_csr_roundtrip_host_memory(capi):
    g = W.ba_graph(3000, 5, seed_off=31)
    rp, col, w = csr_of(g)
    G = capi.Graph.from_csr(g["n"], rp, col, None, directed=False)
    grp, gcol, _, gdeg = G.export(weights=False)
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    assert np.array_equal(gdeg, np.diff(rp).astype(np.float64))


# ------------------------------------------------------------ frontier

@pytest.mark.parametrize("n", [1, 2047, 2048, 2049, 100003])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_frontier_bit_exact(capi, n, dtype):
    import torch

    rng = np.random.default_rng(n)
    h = rng.random(n).astype(dtype)
    r = (rng.random(n) * 2 - 1).astype(dtype) * 1.5
    ties = rng.random(n) < 0.1
    r[ties] = np.where(rng.random(ties.sum()) < 0.5, h[ties], -h[ties])  # |r| == h is not in F
    want = oracle.frontier(r, h)
    lst, cnt = capi.frontier(torch.from_numpy(r).cuda(), torch.from_numpy(h).cuda())
    assert cnt == want.shape[0]
    assert np.array_equal(lst.cpu().numpy(), want)


# ------------------------------------------------------------ colouring

@pytest.mark.parametrize("kind", ["ba", "rmat_dir"])
def test_colouring_matches_greedy_oracle(capi, kind):
    g = W.ba_graph(5000, 5, seed_off=41) if kind == "ba" else W.rmat_directed(12)
    rp, col, w = csr_of(g)
    G = capi.Graph.from_csr(g["n"], *to_dev(rp, col, w), directed=g["directed"])
    colour, k = G.colour()
    want, kw = oracle.greedy_colour(g["n"], rp, col)
    assert k == kw and np.array_equal(colour, want)


@pytest.mark.parametrize("kind,K", [("rmat_dir", 8), ("rmat_und", 4), ("ba", 3)])
def test_palette_colouring_matches_oracle(capi, kind, K):
    g = {"rmat_dir": lambda: W.rmat_directed(12), "rmat_und": lambda: W.rmat_undirected(12),
         "ba": lambda: W.ba_graph(4000, 5, seed_off=43)}[kind]()
    rp, col, w = csr_of(g)
    G = capi.Graph.from_csr(g["n"], *to_dev(rp, col, w), directed=g["directed"])
    colour, k = G.colour(palette=K)
    want, kw, din = oracle.palette_colour(g["n"], rp, col, w, g["directed"], K)
    assert k == kw and np.array_equal(colour, want)


# ------------------------------------------------------------ solve parity

@pytest.fixture(scope="module")
def ba20k():
    g = W.ba_graph(20000, 5)
    rp, col, w = csr_of(g)
    s = g["S"][0]
    z_star, res = oracle.truth(g["n"], rp, col, w, s, omega=1.5)
    return g, rp, col, w, s, z_star


@pytest.mark.parametrize("omega,schedule", [(1.0, 1), (1.0, 2), (1.2, 2), (1.5, 2), (1.8, 2), (0.8, 1)])
def test_fp64_ba20k(capi, ba20k, omega, schedule):
    g, rp, col, w, s, z_star = ba20k
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    (s_d,) = to_dev(s)
    z_d, info, st = G.solve(s_d, eps=1e-6, omega=omega, precision=capi.FJ_PREC_FP64, schedule=schedule)
    z = z_d.cpu().numpy()
    inf = info[0]
    assert st == capi.FJ_OK and inf["converged"] == 1
    assert rel_inf(z, z_star) <= FP64_TOL
    ok, r = certificate_holds(n, rp, col, w, s, z, inf["c_eff"], inf["eps_prime"])
    assert ok, np.max(np.abs(r) / (s + inf["c_eff"]))
    assert inf["resid_rel_max"] <= inf["eps_prime"]
    m = G.metrics(s_d, z_d)
    mo_same = oracle.metrics(n, rp, col, w, s, z, directed=False)
    mo_true = oracle.metrics(n, rp, col, w, s, z_star, directed=False)
    for k in ("P", "D", "I", "C", "mean_z"):
        assert abs(m[k] - mo_same[k]) <= 1e-12 * abs(mo_same[k]) + 1e-15
        assert abs(m[k] - mo_true[k]) <= METRIC_TOL * abs(mo_true[k])


@pytest.mark.parametrize("kind", ["exp", "pareto"])
def test_fp32_rmat_directed_heavy_tailed_opinions(capi, kind):
    """The paper's exponential and power-law (alpha = 2.5) opinion laws, each
    normalised by its maximum: most s_v are small, so the thresholds eps' s'_v
    are too; the certificate and the truth agree all the same."""
    g = W.rmat_directed(13, kind=W.OP_EXP if kind == "exp" else W.OP_PARETO)
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=True)
    (s_d,) = to_dev(s)
    z_d, info, st = G.solve(s_d, eps=1e-6, omega=1.6, palette=8, precision=capi.FJ_PREC_FP32)
    z = z_d.cpu().numpy()
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    ok, _ = certificate_holds(n, rp, col, w, s, z, info[0]["c_eff"], info[0]["eps_prime"])
    assert ok
    z_star, _ = oracle.truth(n, rp, col, w, s)
    assert rel_inf(z, z_star) <= FP32_TOL


@pytest.mark.parametrize("omega", [1.0, 1.2, 1.5])
def test_fp32_rmat_directed(capi, omega):
    g = W.rmat_directed(14)
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    z_star, _ = oracle.truth(n, rp, col, w, s)
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=True)
    (s_d,) = to_dev(s)
    z_d, info, st = G.solve(s_d, eps=1e-6, omega=omega, precision=capi.FJ_PREC_FP32)
    z = z_d.cpu().numpy()
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    assert rel_inf(z, z_star) <= FP32_TOL
    ok, _ = certificate_holds(n, rp, col, w, s, z, info[0]["c_eff"], info[0]["eps_prime"])
    assert ok
    m = G.metrics(s_d, z_d)
    mo = oracle.metrics(n, rp, col, w, s, z_star, directed=True)
    for k in ("P", "D", "I", "C"):
        assert abs(m[k] - mo[k]) <= METRIC_TOL * abs(mo[k])


@pytest.mark.parametrize("omega,schedule", [(1.0, 1), (1.5, 2), (1.8, 2)])
def test_fp32_rmat_undirected_beta_mix(capi, omega, schedule):
    g = W.rmat_undirected(14)
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    z_star, _ = oracle.truth(n, rp, col, w, s, omega=1.5)
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    (s_d,) = to_dev(s)
    z_d, info, st = G.solve(s_d, eps=1e-6, omega=omega, precision=capi.FJ_PREC_FP32, schedule=schedule)
    z = z_d.cpu().numpy()
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    assert rel_inf(z, z_star) <= FP32_TOL
    assert abs(z.sum() - s.sum()) <= 1e-6 * s.sum()  # undirected: 1^T z = 1^T s
    m = G.metrics(s_d, z_d)
    mo = oracle.metrics(n, rp, col, w, s, z_star, directed=False)
    for k in ("P", "D", "I", "C"):
        assert abs(m[k] - mo[k]) <= METRIC_TOL * abs(mo[k])


def test_host_and_device_memory_agree(capi, ba20k):
    g, rp, col, w, s, z_star = ba20k
    G = capi.Graph.from_csr(g["n"], rp, col, w, directed=False)
    z_h, info_h, _ = G.solve(s, eps=1e-6, omega=1.5)
    (s_d,) = to_dev(s)
    z_d, info_d, _ = G.solve(s_d, eps=1e-6, omega=1.5)
    assert np.array_equal(z_h, z_d.cpu().numpy())  # same kernels, same order: identical
    m_h = G.metrics(s, z_h)
    m_d = G.metrics(s_d, z_d)
    assert m_h == m_d


def test_repeat_solve_is_deterministic(capi, ba20k):
    g, rp, col, w, s, _ = ba20k
    G = capi.Graph.from_csr(g["n"], *to_dev(rp, col, w), directed=False)
    (s_d,) = to_dev(s)
    za, ia, _ = G.solve(s_d, eps=1e-6, omega=1.2, precision=capi.FJ_PREC_FP32)
    a = za.cpu().numpy()
    zb, ib, _ = G.solve(s_d, eps=1e-6, omega=1.2, precision=capi.FJ_PREC_FP32)
    b = zb.cpu().numpy()
    if ia[0]["frontier_rounds"] == 0 and ib[0]["frontier_rounds"] == 0:
        assert np.array_equal(a, b)  # sweeps and certificate sum in a fixed order
    else:
        # the FP64 frontier cleanup adds with atomics: equal to within the certificate
        assert np.max(np.abs(a - b)) <= ia[0]["err_bound"] + ib[0]["err_bound"]


# ------------------------------------------------------------ ragged batch

def test_ragged_batch_matches_per_graph(capi):
    r = W.ragged_ba(count=12, lo=300, hi=6000)
    offs = [0]
    rps, cols, ss, parts = [], [], [], []
    for gr in r["graphs"]:
        a, b, _ = W.symmetrize_arcs(gr["src"], gr["dst"])
        rp, col, _ = oracle.csr_from_arcs(gr["n"], a, b)
        parts.append((gr["n"], rp, col, gr["s"]))
        rps.append(rp[1:] + (rps[-1][-1] if rps else 0))
        cols.append(col + offs[-1])
        ss.append(gr["s"])
        offs.append(offs[-1] + gr["n"])
    row_ptr = np.concatenate([[0], *rps]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32)
    s = np.concatenate(ss)
    node_off = np.array(offs, np.int64)
    G = capi.Graph.ragged(*to_dev(node_off, row_ptr, col), directed=False)
    (s_d,) = to_dev(s)
    z_d, infos, st = G.solve(s_d, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    z = z_d.cpu().numpy()
    mets = G.metrics(s_d, z_d)
    assert len(infos) == 12 and len(mets) == 12
    for i, (n, rp, c, sg) in enumerate(parts):
        zs, _ = oracle.truth(n, rp, c, None, sg)
        zi = z[offs[i]:offs[i + 1]]
        assert infos[i]["converged"] == 1
        assert rel_inf(zi, zs) <= FP32_TOL
        mo = oracle.metrics(n, rp, c, None, sg, zs, directed=False)
        for k in ("P", "D", "I", "C"):
            assert abs(mets[i][k] - mo[k]) <= METRIC_TOL * abs(mo[k])


# ------------------------------------------------------------ warm start

def test_warm_start_converges_faster(capi, ba20k):
    g, rp, col, w, s, z_star = ba20k
    G = capi.Graph.from_csr(g["n"], *to_dev(rp, col, w), directed=False)
    (s_d,) = to_dev(s)
    z_cold, ic, _ = G.solve(s_d, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    z0 = z_star + 1e-4 * np.random.default_rng(0).standard_normal(g["n"])
    (z0_d,) = to_dev(z0)
    z_warm, iw, st = G.solve(s_d, z0=z0_d, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    assert st == capi.FJ_OK and iw[0]["converged"] == 1
    assert rel_inf(z_warm.cpu().numpy(), z_star) <= FP32_TOL
    assert iw[0]["sweeps"] < ic[0]["sweeps"]


# ------------------------------------------------------------ edge cases

def test_single_node_and_edgeless(capi):
    rp = np.zeros(2, np.int64)
    col = np.zeros(0, np.int32)
    G = capi.Graph.from_csr(1, rp, col, None, directed=True)
    z, info, st = G.solve(np.array([0.42]), eps=1e-6, omega=1.0)
    assert st == 0 and abs(z[0] - 0.42) <= 1e-12
    n = 5000
    G = capi.Graph.from_csr(n, np.zeros(n + 1, np.int64), col, None, directed=False)
    s = np.random.default_rng(1).random(n)
    z, info, st = G.solve(s, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    assert np.max(np.abs(z - s)) <= 1e-6 * s.max()
    m = G.metrics(s, z)
    assert m["D"] == 0.0


def test_constant_and_signed_opinions(capi, ba20k):
    g, rp, col, w, s, _ = ba20k
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    z, info, _ = G.solve(np.full(n, 0.3), eps=1e-6, omega=1.5)
    err = np.max(np.abs(z - 0.3))
    assert err <= 1e-6 * 0.3
    m = G.metrics(np.full(n, 0.3), z)
    # each edge term is at most (2 err)^2 and each node term at most (2 err)^2
    assert m["D"] <= (rp[-1] // 2) * (2 * err) ** 2 and m["P"] <= n * (2 * err) ** 2
    mo = oracle.metrics(n, rp, col, w, np.full(n, 0.3), z, directed=False)
    for k in ("P", "D", "I", "C"):
        assert abs(m[k] - mo[k]) <= 1e-9 * abs(mo[k]) + 1e-18
    sg = np.where(np.random.default_rng(3).random(n) < 0.5, -1.0, 1.0)
    z, info, st = G.solve(sg, eps=1e-6, omega=1.5)
    zs, _ = oracle.truth(n, rp, col, w, sg, omega=1.5)
    c_eff, epsp = info[0]["c_eff"], info[0]["eps_prime"]
    assert abs(c_eff - (1.0 + 1e-5)) < 1e-15
    # Alg. 2 guarantee relative to z + c_eff
    assert np.all(np.abs(z - zs) <= epsp * (zs + c_eff) + 1e-12)


def test_invalid_arguments_rejected(capi):
    rp = np.array([0, 1, 2], np.int64)
    with pytest.raises(capi.FJError) as e:
        capi.Graph.from_csr(2, rp, np.array([0, 0], np.int32), None)  # self-loop in row 0
    assert e.value.status == capi.FJ_ERR_INVALID_ARG
    with pytest.raises(capi.FJError):
        capi.Graph.from_csr(2, rp, np.array([1, 5], np.int32), None)  # column out of range
    with pytest.raises(capi.FJError):
        capi.Graph.from_csr(2, rp, np.array([1, 0], np.int32), np.array([1.0, -1.0], np.float32))
    with pytest.raises(capi.FJError):
        capi.Graph.from_csr(3, np.array([0, 2, 2, 2], np.int64), np.array([2, 1], np.int32), None)  # unsorted
    with pytest.raises(capi.FJError):
        capi.Graph.from_csr(2, np.array([0, 2, 1], np.int64), np.array([1, 0], np.int32), None)
    G = capi.Graph.from_csr(2, rp, np.array([1, 0], np.int32), None)
    for bad in (dict(omega=2.0), dict(omega=0.0), dict(eps=0.0), dict(eps=1.0),
                dict(omega=1.5, schedule=capi.FJ_SCHED_JACOBI), dict(precision=7)):
        with pytest.raises(capi.FJError) as e:
            G.solve(np.array([0.1, 0.2]), **bad)
        assert e.value.status == capi.FJ_ERR_INVALID_ARG
    with pytest.raises(capi.FJError):
        G.solve(np.array([0.1, np.nan]))


def test_sweep_cap_reports_not_converged(capi, ba20k):
    g, rp, col, w, s, _ = ba20k
    G = capi.Graph.from_csr(g["n"], *to_dev(rp, col, w), directed=False)
    z, info, st = G.solve(s, eps=1e-6, omega=1.0, max_sweeps=3, max_refine=0, check_every=1,
                          allow_unconverged=True)
    assert st == capi.FJ_ERR_NOT_CONVERGED and info[0]["converged"] == 0
    assert np.all(np.isfinite(z))


def test_auto_schedule_recovers_from_divergence(capi):
    """Directed, randomly oriented, weighted BA graph (a warm-start training graph):
    SOR over colour classes at omega 1.5 is not covered by the symmetric theory.
    Under the explicit multicolour schedule a diverging solve reports
    FJ_ERR_DIVERGED; under AUTO it restarts at omega 1 and certifies."""
    gd = W.warm_training_set()[1]  # ba_dir_n30000
    rp, col, w = oracle.csr_from_arcs(gd["n"], gd["src"], gd["dst"], gd["w"])
    n, s = gd["n"], gd["S"][0]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=True)
    (s_d,) = to_dev(s)
    _, _, st_mc = G.solve(s_d, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32,
                          schedule=capi.FJ_SCHED_MULTICOLOUR, allow_unconverged=True)
    z_d, info, st = G.solve(s_d, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32, schedule=capi.FJ_SCHED_AUTO)
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    if st_mc == capi.FJ_ERR_DIVERGED:
        assert info[0]["omega_used"] == 1.0
    else:
        assert info[0]["omega_used"] == 1.5
    z_star, _ = oracle.truth(n, rp, col, w, s)
    assert rel_inf(z_d.cpu().numpy(), z_star) <= FP32_TOL


def test_ragged_from_arcs_matches_separate_handles(capi):
    """The ragged handle the batch bench builds (each graph through the library's
    own ingest, laid out block-diagonally) gives per graph the same certified z
    and metrics as that graph's own handle."""
    r = W.ragged_ba(count=9, lo=200, hi=5000)
    parts, svecs = [], []
    for gr in r["graphs"]:
        a, b, _ = W.symmetrize_arcs(gr["src"], gr["dst"])
        parts.append((gr["n"], a, b, None))
        svecs.append(gr["s"])
    R = capi.Graph.ragged_from_arcs(parts, directed=False)
    s = np.concatenate(svecs)
    z, infos, st = R.solve(s, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP64)
    mets = R.metrics(s, z)
    assert st == capi.FJ_OK and len(infos) == 9
    off = 0
    for i, (n, a, b, _) in enumerate(parts):
        rp, col, _ = oracle.csr_from_arcs(n, a, b)
        zs, _ = oracle.truth(n, rp, col, None, svecs[i])
        assert infos[i]["converged"] == 1
        assert rel_inf(z[off:off + n], zs) <= FP64_TOL
        mo = oracle.metrics(n, rp, col, None, svecs[i], zs, directed=False)
        for k in ("P", "D", "I", "C"):
            assert abs(mets[i][k] - mo[k]) <= METRIC_TOL * abs(mo[k])
        off += n


@pytest.mark.parametrize("name", ["ba2k", "rmat12_dir", "rmat12_und", "path"])
def test_omega_opt_matches_oracle_power_iteration(capi, name):
    """fj_graph_omega_opt: mu after the same number of power-iteration steps as
    the oracle's (FP64, different summation order), and Eq. 17 from it."""
    if name == "ba2k":
        g = W.ba_graph(2000, 5, seed_off=51)
        directed = False
    elif name == "path":
        n = 300
        src = np.arange(n - 1, dtype=np.int32)
        g = {"n": n, "src": src, "dst": src + 1, "w": None, "directed": False}
        directed = False
    else:
        g = W.rmat_directed(12) if name.endswith("dir") else W.rmat_undirected(12)
        directed = name.endswith("dir")
    rp, col, w = csr_of(g)
    n = g["n"]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=directed)
    for iters in (1, 7, 300):
        mu, om = G.omega_opt(iters)
        mu_o = oracle.jacobi_radius_power(n, rp, col, w, iters)
        assert abs(mu - mu_o) <= 1e-11, (iters, mu, mu_o)
        assert abs(om - oracle.omega_opt(min(max(mu_o, 0.0), 1.0))) <= 1e-9


def test_solve_trace_records_convergence(capi):
    """fj_solve_trace: the same z as fj_solve; rows with nondecreasing time and
    sweeps; the last row is a certificate (kind 1) at or below eps'."""
    g = W.rmat_directed(13)
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=True)
    (s_d,) = to_dev(s)
    opts = dict(eps=1e-6, omega=1.6, palette=8, precision=capi.FJ_PREC_FP32)
    z_ref, info_ref, _ = G.solve(s_d, **opts)
    z, info, st, tr = G.solve_trace(s_d, **opts)
    assert st == capi.FJ_OK
    assert np.array_equal(z.cpu().numpy(), z_ref.cpu().numpy())  # the trace changes nothing
    assert tr.shape[0] >= 2 and tr.shape[1] == 4
    assert np.all(np.diff(tr[:, 0]) >= 0) and np.all(np.diff(tr[:, 1]) >= 0)
    assert tr[-1, 3] == 1.0 and tr[-1, 2] <= info[0]["eps_prime"]
    assert tr[-1, 2] == pytest.approx(info[0]["resid_rel_max"], rel=1e-6)
    push = tr[tr[:, 3] == 0.0]
    assert push.shape[0] >= 1 and push[0, 2] > push[-1, 2]  # the push residual came down
