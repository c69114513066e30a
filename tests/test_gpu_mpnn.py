"""Learned warm start on the GPU against the FP64 reference network (oracle/mpnn.py).

The network's forward pass, gradient and Adam step are compared with the
oracle on the same parameters and inputs:
  - against the oracle with bfloat16 rounding at the kernels' rounding points
    (tight: median 1e-5 and 99th percentile 1e-2 relative for z0, 1e-2 per
    gradient block; what remains is FP32 vs FP64 arithmetic between those
    points and the rare rounding-boundary flips it causes),
  - against the plain FP64 oracle (5e-2 relative: eight significant bits at
    every stored activation, weight and pre-activation gradient, compounded
    over three layers of random weights).
Sizes span many 128-row tiles with a ragged tail, weighted directed and
unweighted undirected graphs, and nodes with no out-neighbours.  A training
run shows what the network gains: fewer sweeps from its z0 than from zero on
held-out graphs, to the same certificate.
"""
import numpy as np
import pytest

import oracle
from oracle import mpnn as ref
from fjsynth import workloads as W
from gpu_common import FP32_TOL, certificate_holds, csr_of, rel_inf, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi as c
    return c


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in ref.layer_dims():
        lim = scale / np.sqrt(2 * fi)
        out.append((rng.uniform(-lim, lim, (fi, fo)), rng.uniform(-lim, lim, (fi, fo)), rng.uniform(-0.1, 0.1, fo)))
    wo = rng.uniform(-0.2, 0.2, ref.HIDDEN)
    return ref.pack(out, wo, 0.05).astype(np.float32)


def graphs():
    g1 = W.rmat_directed(12, seed_off=61)          # weighted, directed, sinks present
    g2 = W.ba_graph(3000, 4, seed_off=62)           # unweighted, undirected, 3000 = 23 tiles + 56
    return [g1, g2]


def block_errors(got, want):
    """Relative norm error per parameter block (layer matrices, biases, head)."""
    errs = []
    at = 0
    for fi, fo in ref.layer_dims():
        for size in (fi * fo, fi * fo, fo):
            a, b = got[at:at + size], want[at:at + size]
            errs.append(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
            at += size
    for size in (ref.HIDDEN, 1):
        a, b = got[at:at + size], want[at:at + size]
        errs.append(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
        at += size
    return np.array(errs)


@pytest.mark.parametrize("gi", [0, 1])
def test_forward_matches_oracle(capi, gi):
    g = graphs()[gi]
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    theta = random_params(7 + gi, scale=2.0)
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=g["directed"])
    net = capi.MPNN(theta)
    z0 = net.predict(G, s)
    lo, hi = s.min(), s.max()
    zb, _ = ref.forward(theta.astype(np.float64), n, rp, col, w, s, bf16=True)
    zf, _ = ref.forward(theta.astype(np.float64), n, rp, col, w, s, bf16=False)
    d = oracle.out_degree(n, rp, w)
    zb = np.where(d > 0, np.clip(zb, lo, hi), s)  # nodes that listen to nobody keep z = s
    zf = np.where(d > 0, np.clip(zf, lo, hi), s)
    scale = np.max(np.abs(zf)) + 1e-30
    # against the bfloat16-emulating oracle: the bulk agrees to FP32-vs-FP64
    # arithmetic; a value that lands on the other side of a bfloat16 rounding
    # boundary (FP32 on the GPU, FP64 here) moves a few nodes by about one
    # bfloat16 unit of an activation, and those must stay rare
    d = np.abs(z0 - zb) / scale
    assert np.median(d) <= 1e-5
    assert np.quantile(d, 0.99) <= 1e-2
    assert d.max() <= 3e-2
    assert np.max(np.abs(z0 - zf)) <= 5e-2 * scale
    assert np.all(z0 >= lo) and np.all(z0 <= hi)


@pytest.mark.parametrize("gi", [0, 1])
def test_gradient_matches_oracle(capi, gi):
    g = graphs()[gi]
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    z, _ = oracle.truth(n, rp, col, w, s)
    theta = random_params(17 + gi, scale=2.0)
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=g["directed"])
    net = capi.MPNN(theta)
    loss, grad = net.grad(G, s, z)
    lb, gb = ref.loss_and_grad(theta.astype(np.float64), n, rp, col, w, s, z, bf16=True)
    lf, gf = ref.loss_and_grad(theta.astype(np.float64), n, rp, col, w, s, z, bf16=False)
    assert abs(loss - lb) <= 1e-3 * lb
    assert abs(loss - lf) <= 5e-2 * lf
    eb = block_errors(grad.astype(np.float64), gb)
    ef = block_errors(grad.astype(np.float64), gf)
    assert np.all(eb <= 1e-2), eb
    assert np.all(ef <= 5e-2), ef


def test_adam_step_matches_oracle(capi):
    g = graphs()[1]
    rp, col, w = csr_of(g)
    n, s = g["n"], g["S"][0]
    z, _ = oracle.truth(n, rp, col, w, s)
    theta = random_params(29)
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    net = capi.MPNN(theta)
    m = np.zeros(theta.shape[0])
    v = np.zeros(theta.shape[0])
    t = theta.astype(np.float64)
    for step in (1, 2, 3):
        _, grad = net.grad(G, s, z)
        net.adam_step(1e-3)
        t, m, v = ref.adam_step(t, m, v, grad.astype(np.float64), step, 1e-3)
        got = net.params().astype(np.float64)
        assert np.max(np.abs(got - t)) <= 1e-6 + 1e-5 * np.max(np.abs(t))
        t = got


def test_trained_network_saves_sweeps(capi):
    """Train on BA and SBM graphs (targets from the GPU plain solver, certified),
    then start held-out solves from z0: same certificate, fewer sweeps."""
    train = []
    for i in range(6):
        g = W.ba_graph(4000 + 1000 * i, 4, seed_off=100 + i) if i % 2 == 0 else W.sbm_graph(5000 + 500 * i, 4, index=i)
        rp, col, w = csr_of(g)
        G = capi.Graph.from_csr(g["n"], *to_dev(rp, col, w), directed=False)
        s = g["S"][0]
        z, info, _ = G.solve(s, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP64)
        train.append((G, s, z))
    net = capi.MPNN(ref.init_params(3).astype(np.float32))
    first = None
    for it in range(300):
        G, s, z = train[it % len(train)]
        loss = net.train_step(G, s, z, 3e-3)
        if first is None:
            first = loss
    assert loss < 0.2 * first
    gains = []
    for i in range(2):
        g = W.ba_graph(6000, 4, seed_off=200 + i)
        rp, col, w = csr_of(g)
        n, s = g["n"], g["S"][0]
        G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
        z0 = net.predict(G, s)
        zc, ic, _ = G.solve(s, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
        zw, iw, _ = G.solve(s, z0=z0, eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
        assert ic[0]["converged"] == 1 and iw[0]["converged"] == 1
        z_star, _ = oracle.truth(n, rp, col, w, s)
        assert rel_inf(zw, z_star) <= FP32_TOL
        ok, _ = certificate_holds(n, rp, col, w, s, zw, iw[0]["c_eff"], iw[0]["eps_prime"])
        assert ok
        # the start is closer than zero
        assert np.max(np.abs(z0 - z_star)) < 0.5 * np.max(np.abs(z_star))
        gains.append(ic[0]["sweeps"] - iw[0]["sweeps"])
    assert min(gains) > 0, gains
