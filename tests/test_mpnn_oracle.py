"""Pins of the FP64 reference network (oracle/mpnn.py) against facts that do not
come from the network's own code: finite differences, hand-computed forward
values on a small weighted digraph, the adjoint identity of the aggregation,
bfloat16 rounding of known values and the first Adam step's closed form."""
import numpy as np
import pytest

import oracle
from oracle import mpnn


def small_digraph():
    # arcs (u listens to v, weight): 0->1 (1), 0->2 (3), 1->2 (2); node 2 listens to nobody
    src = np.array([0, 0, 1], np.int32)
    dst = np.array([1, 2, 2], np.int32)
    w = np.array([1.0, 3.0, 2.0], np.float32)
    rp, col, wc = oracle.csr_from_arcs(3, src, dst, w)
    return 3, rp, col, wc


def zero_params():
    layers = [(np.zeros((fi, fo)), np.zeros((fi, fo)), np.zeros(fo)) for fi, fo in mpnn.layer_dims()]
    return layers, np.zeros(mpnn.HIDDEN), 0.0


def test_param_count():
    assert mpnn.param_count() == (2 * 4 * 64 + 64) + 2 * (2 * 64 * 64 + 64) + 65


def test_features_by_hand():
    n, rp, col, w = small_digraph()
    s = np.array([0.2, 0.6, 1.0])
    x = mpnn.features(n, rp, col, w, s)
    # d = (4, 2, 0); din = (0, 1, 2); m_0 = (1*0.6 + 3*1.0)/4, m_1 = 1.0, m_2 = 0
    np.testing.assert_allclose(x[:, 0], s)
    np.testing.assert_allclose(x[:, 1], np.log([5.0, 3.0, 1.0]))
    np.testing.assert_allclose(x[:, 2], np.log([1.0, 2.0, 3.0]))
    np.testing.assert_allclose(x[:, 3], [0.9, 1.0, 0.0])


def _base_by_hand(s):
    # d = (4, 2, 0), m = (0.9, 1.0, 0): b = (s + d m) / (1 + d)
    return np.array([(s[0] + 4 * 0.9) / 5, (s[1] + 2 * 1.0) / 3, s[2]])


def test_base_term_is_one_jacobi_step():
    n, rp, col, w = small_digraph()
    s = np.array([0.2, 0.6, 1.0])
    np.testing.assert_allclose(mpnn.base_term(n, rp, col, w, s), _base_by_hand(s), rtol=0, atol=1e-15)
    # the Jacobi update of (I + L) z = s from z = s: b = (I + D)^{-1} (s + A s)
    dense = oracle.dense_i_plus_l(n, rp, col, w)
    dgl = np.diag(dense)
    a = np.diag(dgl) - dense
    np.testing.assert_allclose(mpnn.base_term(n, rp, col, w, s), (s + a @ s) / dgl, rtol=0, atol=1e-15)


@pytest.mark.parametrize("route", ["copy_s", "copy_m", "aggregate_in_layer2", "bias_only"])
def test_forward_by_hand(route):
    n, rp, col, w = small_digraph()
    s = np.array([0.2, 0.6, 1.0])
    layers, wo, bo = zero_params()
    (w1s, w1n, b1), (w2s, w2n, b2), (w3s, w3n, b3) = layers
    if route == "copy_s":
        w1s[0, 0] = w2s[0, 0] = w3s[0, 0] = 1.0
        wo[0] = 1.0
        want = s
    elif route == "copy_m":
        w1s[3, 0] = w2s[0, 0] = w3s[0, 0] = 1.0
        wo[0] = 1.0
        want = np.array([0.9, 1.0, 0.0])
    elif route == "aggregate_in_layer2":
        # h1_0 = s, h2_0 = mean over out-neighbours of h1_0 = m, h3_0 = h2_0
        w1s[0, 0] = w2n[0, 0] = w3s[0, 0] = 1.0
        wo[0] = 2.0
        want = 2.0 * np.array([0.9, 1.0, 0.0])
    else:
        b3[5] = 0.3
        wo[5] = 2.0
        bo = 0.1
        want = np.full(3, 0.7)
    theta = mpnn.pack(layers, wo, bo)
    z0, _ = mpnn.forward(theta, n, rp, col, w, s)
    np.testing.assert_allclose(z0, _base_by_hand(s) + want, rtol=0, atol=1e-15)


def test_relu_cuts_negative_path():
    n, rp, col, w = small_digraph()
    s = np.array([0.2, 0.6, 1.0])
    layers, wo, bo = zero_params()
    layers[0][0][0, 0] = -1.0  # h1_0 = relu(-s) = 0
    layers[1][0][0, 0] = layers[2][0][0, 0] = 1.0
    wo[0] = 1.0
    z0, _ = mpnn.forward(mpnn.pack(layers, wo, bo), n, rp, col, w, s)
    np.testing.assert_allclose(z0, _base_by_hand(s), rtol=0, atol=1e-15)


def test_aggregation_adjoint_identity():
    rng = np.random.default_rng(3)
    n = 40
    src = rng.integers(0, n, 300).astype(np.int32)
    dst = rng.integers(0, n, 300).astype(np.int32)
    w = (0.5 + rng.random(300)).astype(np.float32)
    rp, col, wc = oracle.csr_from_arcs(n, src, dst, w)
    fwd, adj, _ = mpnn._mean_op(n, rp, col, wc)
    h = rng.standard_normal((n, 5))
    y = rng.standard_normal((n, 5))
    assert abs(np.sum(fwd(h) * y) - np.sum(h * adj(y))) <= 1e-12 * np.sum(np.abs(fwd(h) * y))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(11)
    n = 18
    src = rng.integers(0, n, 70).astype(np.int32)
    dst = rng.integers(0, n, 70).astype(np.int32)
    w = (0.5 + rng.random(70)).astype(np.float32)
    rp, col, wc = oracle.csr_from_arcs(n, src, dst, w)
    s = rng.random(n)
    z = rng.random(n)
    theta = mpnn.init_params(5) * 3.0
    loss, g = mpnn.loss_and_grad(theta, n, rp, col, wc, s, z)
    _, sv = mpnn.forward(theta, n, rp, col, wc, s)
    assert min(np.min(np.abs(p)) for p in sv["pre"]) > 1e-5  # no kink within the step
    idx = rng.choice(theta.shape[0], 80, replace=False)
    idx = np.concatenate([idx, [theta.shape[0] - 1, theta.shape[0] - 2]])
    h = 1e-7
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (mpnn.loss_and_grad(tp, n, rp, col, wc, s, z)[0] - mpnn.loss_and_grad(tm, n, rp, col, wc, s, z)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_bf16_round_known_values():
    one = 1.0
    u = 2.0 ** -8
    vals = np.array([one, one + u, one + 3 * u, one + u + 2.0 ** -20, -2.5, 0.0, 3.0e38])
    want = np.array([one, one, one + 4 * u, one + 2 * u, -2.5, 0.0, np.float64(np.float32(3.0e38))])
    got = mpnn.bf16_round(vals)
    # 3e38 rounds to a bfloat16 neighbour: check it is representable (low 16 bits zero)
    assert np.all(got[:6] == want[:6])
    assert (np.float32(got[6]).view(np.uint32) & 0xFFFF) == 0


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    theta = np.array([1.0, 1.0, 1.0, 1.0])
    t1, m, v = mpnn.adam_step(theta, np.zeros(4), np.zeros(4), g, 1, lr=0.01)
    # first step: m/(1-b1) = g, v/(1-b2) = g^2, so the step is lr * g / (|g| + eps)
    np.testing.assert_allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
