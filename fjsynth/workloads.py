"""Named synthetic workloads: graph edge lists plus innate-opinion vectors.

Each workload fixes its generator, sizes and seed.  The five full-size ones
stand in for the paper's KONECT/SNAP graphs (power-law degree, up to tens of
millions of nodes); small ones of the same shape serve the parity tests.
A workload is a dict with keys ``n, src, dst, w (or None), directed, S``
where ``S`` is a list of float64 opinion vectors (already rounded to FP32 and
back when the workload is an FP32 one).
"""
from __future__ import annotations

import numpy as np

from . import OP_ARCSINE, OP_BETA_MIX, OP_EXP, OP_PARETO, OP_SIGN, OP_UNIFORM, ba, loguniform_sizes, opinions, rmat, sbm, uniform_array

BASE_SEED = 20250714


def _f32(s: np.ndarray) -> np.ndarray:
    return s.astype(np.float32).astype(np.float64)


def ba_graph(n: int = 20000, m: int = 5, seed_off: int = 1, nvec: int = 1, kind: int = OP_UNIFORM):
    """Undirected Barabasi-Albert graph, unit weights, U[0,1] opinions (FP64)."""
    seed = BASE_SEED + seed_off
    src, dst = ba(n, m, seed)
    S = [opinions(n, kind, seed + 1000, vec=k) for k in range(nvec)]
    return dict(name=f"ba_n{n}_m{m}", n=n, src=src, dst=dst, w=None, directed=False, S=S,
                fp32=False)


def rmat_directed(scale: int = 22, edge_factor: int = 16, seed_off: int = 2, nvec: int = 1,
                  kind: int = OP_UNIFORM):
    """Directed R-MAT (a=.57, b=c=.19), weights U(0.5,1.5) FP32, s of `kind`
    (default U[0,1]; OP_EXP and OP_PARETO are the paper's exponential and
    power-law opinions, normalised by their maximum) rounded to FP32.

    Arc (src, dst) means src listens to dst: row src of A holds dst.
    """
    seed = BASE_SEED + seed_off
    src, dst, w = rmat(scale, edge_factor, seed=seed, weighted=True)
    n = 1 << scale
    S = [_f32(opinions(n, kind, seed + 1000, vec=k)) for k in range(nvec)]
    return dict(name=f"rmat{scale}_dir_w", n=n, src=src, dst=dst, w=w, directed=True, S=S,
                fp32=True)


def rmat_undirected(scale: int = 24, edge_factor: int = 16, seed_off: int = 3,
                    kinds=(OP_BETA_MIX,), nvec: int = 1):
    """Undirected R-MAT with unit weights; opinion vector k has kind kinds[k % len(kinds)]."""
    seed = BASE_SEED + seed_off
    src, dst, _ = rmat(scale, edge_factor, seed=seed, weighted=False)
    n = 1 << scale
    S = [_f32(opinions(n, kinds[k % len(kinds)], seed + 1000, vec=k)) for k in range(nvec)]
    return dict(name=f"rmat{scale}_und", n=n, src=src, dst=dst, w=None, directed=False, S=S,
                fp32=True)


def rmat_multirhs(scale: int = 22, nvec: int = 64, seed_off: int = 4):
    """Undirected R-MAT with nvec opinion vectors cycling U[0,1] / Beta(1/2,1/2) / +-1."""
    return rmat_undirected(scale, 16, seed_off, kinds=(OP_UNIFORM, OP_ARCSINE, OP_SIGN),
                           nvec=nvec)


def ragged_ba(count: int = 256, lo: int = 1000, hi: int = 200000, m: int = 5, seed_off: int = 4):
    """A batch of BA graphs with log-uniform sizes, one U[0,1] vector each (FP32-rounded)."""
    seed = BASE_SEED + seed_off
    sizes = loguniform_sizes(count, lo, hi, seed)
    graphs = []
    for i, n in enumerate(sizes.tolist()):
        src, dst = ba(int(n), m, seed + 17 * (i + 1))
        s = _f32(opinions(int(n), OP_UNIFORM, seed + 5000 + i))
        graphs.append(dict(n=int(n), src=src, dst=dst, s=s))
    return dict(name=f"ragged{count}_ba", graphs=graphs, directed=False, fp32=True)


def sbm_graph(n: int, nblocks: int = 4, deg_in: float = 12.0, deg_out: float = 3.0,
              seed_off: int = 5, index: int = 0):
    seed = BASE_SEED + seed_off + 7919 * index
    src, dst = sbm(n, nblocks, deg_in, deg_out, seed)
    S = [opinions(n, OP_UNIFORM, seed + 1000)]
    return dict(name=f"sbm_n{n}_b{nblocks}", n=n, src=src, dst=dst, w=None, directed=False,
                S=S, fp32=False)


def symmetrize_arcs(src: np.ndarray, dst: np.ndarray, w=None):
    """Arc list of an undirected edge list: arc 2e = (src_e, dst_e), arc 2e+1 = (dst_e, src_e).

    Both arcs of edge e carry e's weight; the interleaving fixes which arc comes
    first when duplicates are later dropped keep-first.
    """
    m = src.shape[0]
    asrc = np.empty(2 * m, np.int32)
    adst = np.empty(2 * m, np.int32)
    asrc[0::2] = src
    asrc[1::2] = dst
    adst[0::2] = dst
    adst[1::2] = src
    aw = None
    if w is not None:
        aw = np.empty(2 * m, np.float32)
        aw[0::2] = w
        aw[1::2] = w
    return asrc, adst, aw


def warm_training_set(seed_off: int = 7, nvec: int = 3, rmat_scales=(14, 16, 17)):
    """Training graphs of the learned warm start: SBM and BA graphs with n from
    10^4 to 10^6, nvec U[0,1] vectors each.  SBM graphs are undirected with
    unit weights; BA graphs are directed, each edge oriented by a fair coin
    and weighted U(0.5, 1.5) FP32, so the network also sees nodes that listen
    to nobody, nodes nobody listens to, and weights.  Then small weighted
    directed R-MAT graphs (rmat_scales), from seeds of their own: the same
    family as the evaluation graph, held out by seed and scale."""
    sizes = [10_000, 30_000, 100_000, 300_000, 1_000_000, 20_000, 60_000, 200_000]
    out = []
    for i, n in enumerate(sizes):
        seed = BASE_SEED + seed_off + 104729 * (i + 1)
        S = [_f32(opinions(n, OP_UNIFORM, seed + 1000, vec=k)) for k in range(nvec)]
        if i % 2 == 0:
            src, dst = sbm(n, 2 + i % 7, 12.0, 3.0, seed)
            out.append(dict(name=f"sbm_n{n}", n=n, src=src, dst=dst, w=None, directed=False, S=S, fp32=True))
        else:
            a, b = ba(n, 5, seed)
            flip = uniform_array(seed, 7, a.shape[0]) < 0.5
            src = np.where(flip, b, a).astype(np.int32)
            dst = np.where(flip, a, b).astype(np.int32)
            w = (0.5 + uniform_array(seed, 8, a.shape[0])).astype(np.float32)
            out.append(dict(name=f"ba_dir_n{n}", n=n, src=src, dst=dst, w=w, directed=True, S=S, fp32=True))
    for i, sc in enumerate(rmat_scales):
        seed = BASE_SEED + seed_off + 7919 * (i + 1) + 500
        src, dst, w = rmat(sc, 16, seed=seed, weighted=True)
        n = 1 << sc
        S = [_f32(opinions(n, OP_UNIFORM, seed + 1000, vec=k)) for k in range(nvec)]
        out.append(dict(name=f"rmat{sc}_dir_train", n=n, src=src, dst=dst, w=w, directed=True, S=S, fp32=True))
    return out
