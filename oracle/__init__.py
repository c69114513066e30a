"""FP64 CPU oracle for the Friedkin-Johnsen solver (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is independent of the CUDA library:
the sequential loops are in ``fj_oracle.c`` (plain C, FP64), the graph ingest
and the small definitional helpers are plain numpy below.  Every function
names the passage of the paper it follows.

Graph convention: CSR ``row_ptr (int64, n+1)``, ``col (int32)``, optional
``w (float32)``.  Row u lists the nodes u listens to, so a_uj = w[k] and the
Laplacian is L = D - A with D the weighted out-degrees (Section 3.2, Eq. 1).

Parity unpinned: ``push_rounds`` update counts (the paper publishes none).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfjoracle.so")
_lib_handle = None

C_DEFAULT = 1e-5      # the constant c of Alg. 2 (Section 6 settings)
SIGMA_DEFAULT = 1e-5  # the threshold sigma of Alg. 2 (Section 6 settings)


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "fj_oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-shared",
                    "-fPIC", "-pthread", src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    build()
    lib = ctypes.CDLL(_SO)
    I64, D, VP = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    lib.oracle_blisor_fifo.argtypes = [I64, VP, VP, VP, VP, D, D, D, D, ctypes.c_int, I64, VP, VP, VP]
    lib.oracle_blisor_fifo.restype = ctypes.c_int
    lib.oracle_push_rounds.argtypes = [I64, VP, VP, VP, VP, D, D, D, D, I64, VP, VP, VP]
    lib.oracle_push_rounds.restype = ctypes.c_int
    lib.oracle_push_rounds_threads.argtypes = [I64, VP, VP, VP, VP, D, D, D, D, I64, ctypes.c_int, VP, VP, VP]
    lib.oracle_push_rounds_threads.restype = ctypes.c_int
    lib.oracle_sor_truth.argtypes = [I64, VP, VP, VP, VP, D, D, I64, VP, VP]
    lib.oracle_sor_truth.restype = I64
    lib.oracle_gs_sweep_from_zero.argtypes = [I64, VP, VP, VP, VP, VP]
    lib.oracle_gs_sweep_from_zero.restype = None
    lib.oracle_sor_ordered.argtypes = [I64, VP, VP, VP, VP, VP, D, D, D, D, I64, VP, VP, VP]
    lib.oracle_sor_ordered.restype = ctypes.c_int
    lib.oracle_residual.argtypes = [I64, VP, VP, VP, VP, VP, VP]
    lib.oracle_residual.restype = None
    lib.oracle_csr_build.argtypes = [I64, I64, VP, VP, VP, VP, VP, VP]
    lib.oracle_csr_build.restype = I64
    lib.oracle_residual_dot2.argtypes = [I64, VP, VP, VP, VP, VP, VP]
    lib.oracle_residual_dot2.restype = None
    lib.oracle_lu_solve.argtypes = [I64, VP, VP, VP]
    lib.oracle_lu_solve.restype = ctypes.c_int
    lib.oracle_metrics.argtypes = [I64, VP, VP, VP, VP, VP, ctypes.c_int, VP]
    lib.oracle_metrics.restype = None
    lib.oracle_greedy_colour.argtypes = [I64, VP, VP, VP, VP]
    lib.oracle_greedy_colour.restype = I64
    lib.oracle_palette_colour.argtypes = [I64, VP, VP, VP, VP, ctypes.c_int, VP]
    lib.oracle_palette_colour.restype = I64
    _lib_handle = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data


def _graph_args(row_ptr, col, w):
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w64 = None if w is None else np.ascontiguousarray(w, np.float64)
    return row_ptr, col, w64


# --------------------------------------------------------------- graph ingest

def csr_from_arcs(n: int, src, dst, w=None):
    """Simple-graph CSR from an arc list (Section 3.2: simple graphs).

    Drops self-loops, orders arcs by (src, dst) keeping generation order among
    repeats (stable), keeps the first arc of every repeated (src, dst) pair.
    Returns ``(row_ptr int64[n+1], col int32[nnz], w float32[nnz] or None)``.
    Built by the C routine ``oracle_csr_build``; ``csr_from_arcs_np`` is the
    same definition in numpy, and the pins check the two agree.
    """
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    m = int(src.shape[0])
    wf = None if w is None else np.ascontiguousarray(w, np.float32)
    row_ptr = np.empty(n + 1, np.int64)
    col = np.empty(max(m, 1), np.int32)
    wout = None if w is None else np.empty(max(m, 1), np.float32)
    nnz = _lib().oracle_csr_build(n, m, _p(src), _p(dst), _p(wf), _p(row_ptr), _p(col), _p(wout))
    if nnz < 0:
        raise ValueError("arc list names a node outside [0, n)")
    return row_ptr, col[:nnz].copy(), None if wout is None else wout[:nnz].copy()


def csr_from_arcs_np(n: int, src, dst, w=None):
    """csr_from_arcs by a stable lexicographic sort in numpy (the pins' second route)."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    keep = src != dst
    idx = np.flatnonzero(keep)
    order = idx[np.lexsort((idx, dst[idx], src[idx]))]
    s_sorted = src[order]
    d_sorted = dst[order]
    first = np.ones(order.shape[0], bool)
    if order.shape[0] > 1:
        first[1:] = (s_sorted[1:] != s_sorted[:-1]) | (d_sorted[1:] != d_sorted[:-1])
    order = order[first]
    rows = src[order]
    col = dst[order].astype(np.int32)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    wout = None if w is None else np.asarray(w, np.float32)[order]
    return row_ptr, col, wout


def transpose(n: int, row_ptr, col, w=None):
    """In-neighbour CSR: row v lists every u with a_uv > 0 in ascending u (stable by col)."""
    rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(row_ptr))
    order = np.argsort(col, kind="stable")
    tcol = rows[order]
    tptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(col, minlength=n), out=tptr[1:])
    tw = None if w is None else np.asarray(w, np.float32)[order]
    return tptr, tcol, tw


def out_degree(n: int, row_ptr, w=None) -> np.ndarray:
    """d_u = sum_j a_uj in FP64 (Section 3.2)."""
    if w is None:
        return np.diff(row_ptr).astype(np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    return np.bincount(rows, weights=np.asarray(w, np.float64), minlength=n)


def inv_diag32(d64: np.ndarray) -> np.ndarray:
    """1/(1 + d_v) as an FP64 quotient rounded to FP32."""
    return (1.0 / (1.0 + d64)).astype(np.float32)


def shift_params(s, eps: float, c: float = C_DEFAULT, sigma: float = SIGMA_DEFAULT):
    """Alg. 2: c_eff = c + max(0, -min s) and eps' = sigma * eps / (c + sigma)."""
    c_eff = c - min(0.0, float(np.min(s))) if len(s) else c
    return c_eff, sigma * eps / (c + sigma)


def frontier(r, h) -> np.ndarray:
    """F = {v : |r_v| > h_v} in ascending order (strict test of Alg. 1 and Alg. 3)."""
    return np.flatnonzero(np.abs(r) > h).astype(np.int32)


def dense_i_plus_l(n: int, row_ptr, col, w=None) -> np.ndarray:
    """Dense I + L = I + D - A (Section 3.2)."""
    M = np.zeros((n, n), np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    vals = np.ones(len(col)) if w is None else np.asarray(w, np.float64)
    np.add.at(M, (rows, np.asarray(col, np.int64)), -vals)
    M[np.arange(n), np.arange(n)] += 1.0 + out_degree(n, row_ptr, w)
    return M


# --------------------------------------------------------------- solvers

def lu_solve(n: int, row_ptr, col, w, s) -> np.ndarray:
    """z = (I + L)^{-1} s by dense LU with partial pivoting (Lemma 1); n <= 2000."""
    if n > 4000:
        raise ValueError("dense oracle is for small graphs")
    M = np.ascontiguousarray(dense_i_plus_l(n, row_ptr, col, w))
    b = np.ascontiguousarray(s, np.float64)
    x = np.empty(n, np.float64)
    if _lib().oracle_lu_solve(n, _p(M), _p(b), _p(x)) != 0:
        raise RuntimeError("singular I + L")
    return x


def neumann_series(n: int, row_ptr, col, w, s, terms: int = 4000) -> np.ndarray:
    """Lemma 2: z = (I + D)^{-1} sum_i (A (I + D)^{-1})^i s, truncated (tiny graphs only)."""
    M = dense_i_plus_l(n, row_ptr, col, w)
    d = np.diag(M) - 1.0
    A = -(M - np.diag(np.diag(M)))
    inv = 1.0 / (1.0 + d)
    term = np.asarray(s, np.float64).copy()
    acc = np.zeros(n)
    for _ in range(terms):
        acc += term
        term = A @ (inv * term)
        if np.max(np.abs(term)) < 1e-18:
            break
    return inv * acc


def blisor_fifo(n, row_ptr, col, w, s, eps, omega=1.0, c=C_DEFAULT, sigma=SIGMA_DEFAULT,
                single_pass=False, max_pops=None):
    """ImprovedBLI / ImprovedBLISOR with a FIFO queue (Alg. 1-3), FP64.

    Returns ``(z, r, pushes, updates, finished)``; r is the residual of the
    shifted system s' = s + c_eff.
    """
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    z = np.empty(n)
    r = np.empty(n)
    stats = np.zeros(4, np.int64)
    if max_pops is None:
        max_pops = np.iinfo(np.int64).max
    rc = _lib().oracle_blisor_fifo(n, _p(row_ptr), _p(col), _p(w64), _p(s), eps, omega, c, sigma,
                                   1 if single_pass else 0, max_pops, _p(z), _p(r), _p(stats))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    return z, r, int(stats[0]), int(stats[1]), rc == 0


def push_rounds(n, row_ptr, col, w, s, eps, omega=1.0, c=C_DEFAULT, sigma=SIGMA_DEFAULT,
                max_rounds=1 << 40):
    """Synchronous frontier rounds (all nodes above threshold push together), FP64.

    Returns ``(z, r, pushes, updates, rounds, finished)``.
    """
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    z = np.empty(n)
    r = np.empty(n)
    stats = np.zeros(4, np.int64)
    rc = _lib().oracle_push_rounds(n, _p(row_ptr), _p(col), _p(w64), _p(s), eps, omega, c, sigma,
                                   max_rounds, _p(z), _p(r), _p(stats))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    return z, r, int(stats[0]), int(stats[1]), int(stats[2]), rc == 0


def push_rounds_threads(n, row_ptr, col, w, s, eps, omega=1.0, threads=None, c=C_DEFAULT,
                        sigma=SIGMA_DEFAULT, max_rounds=1 << 40):
    """push_rounds on `threads` host threads (default: every core), for the
    all-core CPU baseline; bit for bit push_rounds' result.

    Returns ``(z, r, pushes, updates, rounds, finished, threads_used)``.
    """
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    threads = int(threads or os.cpu_count() or 1)
    z = np.empty(n)
    r = np.empty(n)
    stats = np.zeros(4, np.int64)
    rc = _lib().oracle_push_rounds_threads(n, _p(row_ptr), _p(col), _p(w64), _p(s), eps, omega, c, sigma,
                                           max_rounds, threads, _p(z), _p(r), _p(stats))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    return z, r, int(stats[0]), int(stats[1]), int(stats[2]), rc == 0, int(stats[3])


def sor_ordered(n, row_ptr, col, w, s, order, eps, omega, c=C_DEFAULT, sigma=SIGMA_DEFAULT,
                max_sweeps=1 << 40):
    """Residual-push SOR (Section 5.2) sweeping nodes in a fixed order, FP64.

    Returns ``(z, r, pushes, updates, sweeps, finished)``.
    """
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    order = np.ascontiguousarray(order, np.int32)
    z = np.empty(n)
    r = np.empty(n)
    stats = np.zeros(4, np.int64)
    rc = _lib().oracle_sor_ordered(n, _p(row_ptr), _p(col), _p(w64), _p(s), _p(order), eps, omega,
                                   c, sigma, max_sweeps, _p(z), _p(r), _p(stats))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    return z, r, int(stats[0]), int(stats[1]), int(stats[2]), rc == 0


def truth(n, row_ptr, col, w, s, tol=None, omega=1.0, max_sweeps=200000, force_sor=False):
    """Certified FP64 equilibrium: LU for n <= 2000, else SOR sweeps to a tiny residual.

    The bound max_v |z_v - z*_v| <= max_v |r_v| holds because (I + L)^{-1} is
    nonnegative and row-stochastic (Section 3.3).  Returns ``(z, resid_inf)``.
    ``force_sor`` takes the sweep branch at any n (its pins compare the two
    branches on small graphs).
    """
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    if n <= 2000 and not force_sor:
        z = lu_solve(n, row_ptr, col, w, s)
        return z, float(np.max(np.abs(residual(n, row_ptr, col, w, s, z)))) if n else 0.0
    if tol is None:
        # the FP64 residual itself carries rounding of order (1 + d_max) ulp, so the
        # reachable floor grows with the largest weighted degree
        dmax = float(np.max(out_degree(n, row_ptr, w))) if n else 0.0
        tol = max(1e-13, 4e-15 * (1.0 + dmax)) * max(1.0, float(np.max(np.abs(s))))
    z = np.zeros(n)
    res = ctypes.c_double()
    sweeps = _lib().oracle_sor_truth(n, _p(row_ptr), _p(col), _p(w64), _p(s), omega, tol,
                                     max_sweeps, _p(z), ctypes.addressof(res))
    if sweeps <= 0:
        raise RuntimeError(f"truth solve did not reach {tol} (residual {res.value})")
    return z, res.value


def gs_sweep_from_zero(n, row_ptr, col, w, s) -> np.ndarray:
    """One Gauss-Seidel sweep in node order from zero (Eq. gauss, Theorem 2)."""
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    z = np.empty(n)
    _lib().oracle_gs_sweep_from_zero(n, _p(row_ptr), _p(col), _p(w64), _p(s), _p(z))
    return z


def residual(n, row_ptr, col, w, s, z) -> np.ndarray:
    """r = s - (I + L) z in FP64, row by row (Lemma 3's residual)."""
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    r = np.empty(n)
    _lib().oracle_residual(n, _p(row_ptr), _p(col), _p(w64), _p(s), _p(z), _p(r))
    return r


def residual_accurate(n, row_ptr, col, w, s, z) -> np.ndarray:
    """r = s - (I + L) z accumulated with Dot2 (compensated), then rounded once.

    Agrees with the exact rational value of the residual of the given FP64
    inputs to within a few units in its last place whatever the cancellation.
    """
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    r = np.empty(n)
    _lib().oracle_residual_dot2(n, _p(row_ptr), _p(col), _p(w64), _p(s), _p(z), _p(r))
    return r


def metrics(n, row_ptr, col, w, s, z, directed: bool) -> dict:
    """Table 1: mean, C, P, I, D (undirected D counts each edge once)."""
    row_ptr, col, w64 = _graph_args(row_ptr, col, w)
    s = np.ascontiguousarray(s, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    out = np.empty(5)
    _lib().oracle_metrics(n, _p(row_ptr), _p(col), _p(w64), _p(s), _p(z),
                          0 if directed else 1, _p(out))
    return dict(mean_z=out[0], C=out[1], P=out[2], I=out[3], D=out[4])


# --------------------------------------------------------------- colouring

_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(x) -> np.ndarray:
    """SplitMix64 output for state x (Steele, Lea & Flood 2014): mix(x + gamma)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def symmetric_pattern(n, row_ptr, col):
    """Adjacency of the symmetrised graph (u ~ v when a_uv > 0 or a_vu > 0), sorted, unique."""
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    c = np.asarray(col, np.int64)
    a = np.concatenate([rows, c])
    b = np.concatenate([c, rows])
    key = np.unique(a * n + b)
    sa = key // n
    sb = (key % n).astype(np.int32)
    ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(sa, minlength=n), out=ptr[1:])
    return ptr, sb


def colour_priority_order(n, sym_ptr) -> np.ndarray:
    """Largest-degree-first order: symmetric degree descending, then the high 32 bits
    of splitmix64(v) descending, then v ascending."""
    deg = np.diff(sym_ptr).astype(np.int64)
    h = (splitmix64(np.arange(n, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)
    return np.lexsort((np.arange(n), -h, -deg)).astype(np.int32)


def greedy_colour(n, row_ptr, col):
    """Greedy colouring of the symmetrised graph in largest-degree-first order.

    Returns ``(colour int32[n], ncolours)``; each class is an independent set,
    so a class-by-class sweep is a valid Gauss-Seidel order (Theorem 2).
    """
    sym_ptr, sym_col = symmetric_pattern(n, row_ptr, col)
    order = colour_priority_order(n, sym_ptr)
    colour = np.empty(n, np.int32)
    sym_ptr = np.ascontiguousarray(sym_ptr, np.int64)
    sym_col = np.ascontiguousarray(sym_col, np.int32)
    k = _lib().oracle_greedy_colour(n, _p(sym_ptr), _p(sym_col), _p(order), _p(colour))
    if k < 0:
        raise MemoryError("oracle allocation failed")
    return colour, int(k)


def fixed_point_weight(w):
    """Arc weight in 32.32 fixed point (round to nearest), the unit in which
    colouring conflicts are summed."""
    return np.rint(np.asarray(w, np.float64) * 4294967296.0).astype(np.int64)


def symmetric_weights(n, row_ptr, col, w, directed: bool):
    """Symmetric adjacency for the colouring conflicts, with per-pair weights
    as (float a_uv + a_vu, fixed-point q(a_uv) + q(a_vu)) for a directed graph
    and (a_uv, q(a_uv)) for an undirected one.  Sorted rows, unique columns."""
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    c = np.asarray(col, np.int64)
    wv = np.ones(len(c)) if w is None else np.asarray(w, np.float64)
    qv = fixed_point_weight(wv)
    if directed:
        a = np.concatenate([rows, c])
        b = np.concatenate([c, rows])
        ww = np.concatenate([wv, wv])
        qq = np.concatenate([qv, qv])
    else:
        a, b, ww, qq = rows, c, wv, qv
    key = a * n + b
    order = np.argsort(key, kind="stable")
    key, ww, qq = key[order], ww[order], qq[order]
    first = np.ones(len(key), bool)
    first[1:] = key[1:] != key[:-1]
    starts = np.flatnonzero(first)
    uk = key[starts]
    sw = np.add.reduceat(ww, starts) if len(ww) else ww
    sq = np.add.reduceat(qq, starts) if len(qq) else qq
    sa = uk // n
    ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(sa, minlength=n), out=ptr[1:])
    return ptr, (uk % n).astype(np.int32), sw, sq


def palette_colour(n, row_ptr, col, w, directed: bool, K: int):
    """Greedy colouring with a palette of K colours in largest-degree-first order
    (least-conflict colour when the palette is exhausted).  Returns
    (colour int32[n], colours used, in-class weight per node float64[n])."""
    sp_, sc_, sw_, sq_ = symmetric_weights(n, row_ptr, col, w, directed)
    order = colour_priority_order(n, sp_)
    colour = np.empty(n, np.int32)
    k = _lib().oracle_palette_colour(n, _p(np.ascontiguousarray(sp_)), _p(np.ascontiguousarray(sc_)),
                                     _p(np.ascontiguousarray(sq_)), _p(order), int(K), _p(colour))
    if k < 0:
        raise MemoryError("oracle allocation failed")
    rows = np.repeat(np.arange(n), np.diff(sp_))
    same = colour[rows] == colour[sc_]
    din = np.bincount(rows[same], weights=sw_[same], minlength=n)
    return colour, int(k), din


# Largest hub prefix of the multicolour row order (a layout parameter of the
# sweep, not of the method: the size of its shared-memory increment table).
HUB_CAPACITY = 49152


def sweep_order(n, row_ptr, col, colour, hubs: bool):
    """Row order of the multicolour schedule: any order is a Gauss-Seidel order
    (Theorem 2), so the one chosen only has to be reproducible.  With hubs (one
    graph, a bounded palette), the nodes of largest in-degree come first,
    ordered by class: in-degree >= the smallest threshold that admits at most
    HUB_CAPACITY of them (every node when n <= HUB_CAPACITY).  Then every
    class's other nodes.  Inside each range: in-degree descending (clamped to
    2^22 - 1), then id.  Without hubs: colour, then id.

    Returns (perm int32[n]: id of row i, nhub, hub_row[K+1], class_row[K+1]);
    class c is rows [hub_row[c], hub_row[c+1]) and [class_row[c], class_row[c+1]).
    """
    colour = np.asarray(colour, np.int64)
    col = np.asarray(col, np.int64)
    K = int(colour.max()) + 1 if n else 0
    indeg = np.bincount(col, minlength=n).astype(np.int64)  # rows that list the node
    ids = np.arange(n)
    if hubs:
        if n <= HUB_CAPACITY:
            hub = np.ones(n, bool)
        else:
            v = int(np.sort(indeg)[::-1][HUB_CAPACITY - 1])
            thr = v if int(np.count_nonzero(indeg >= v)) <= HUB_CAPACITY else v + 1
            hub = indeg >= thr
        d = np.minimum(indeg, (1 << 22) - 1)
        perm = np.lexsort((ids, -d, colour, ~hub))
    else:
        hub = np.zeros(n, bool)
        perm = np.lexsort((ids, colour))
    nhub = int(np.count_nonzero(hub))
    pc = colour[perm]
    hub_row = np.array([int(np.searchsorted(pc[:nhub], c, side="left")) for c in range(K + 1)], np.int64)
    class_row = np.array([nhub + int(np.searchsorted(pc[nhub:], c, side="left")) for c in range(K + 1)], np.int64)
    hub_row[K], class_row[K] = nhub, n
    return perm.astype(np.int32), nhub, hub_row, class_row


def safe_omega(omega, d64, din):
    """Per-node relaxation for a colouring with in-class conflicts: the largest
    omega_v <= omega with (2 / omega_v - 1)(1 + d_v) >= din_v / 0.98, which keeps
    M + M^T - (I + L) diagonally dominant (Gershgorin) on undirected graphs."""
    bound = 0.98 * 2.0 * (1.0 + d64) / (1.0 + d64 + din)
    return np.where(din > 0, np.minimum(omega, bound), omega)


def jacobi_radius_power(n, row_ptr, col, w, iters: int) -> float:
    """mu = rho((I + D)^{-1} A), the spectral radius of the Jacobi iteration
    matrix M of (I + L) z = s (Section 5.2, the quantity of Eq. 17), by `iters`
    steps of power iteration on B = (I + M) / 2 from the all-ones vector.
    B's dominant eigenvalue is (1 + mu) / 2, strictly largest in modulus even
    when M has -mu in its spectrum (bipartite graphs), so the estimate
    2 nu - 1, nu = sum(B x) / sum(x), converges to mu.  x is rescaled to sum n
    after every step.  Plain FP64."""
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    a = np.ones(col.shape[0]) if w is None else np.asarray(w, np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    d = np.bincount(rows, weights=a, minlength=n)
    inv = 1.0 / (1.0 + d)
    x = np.ones(n)
    nu = 0.0
    for _ in range(iters):
        ax = np.bincount(rows, weights=a * x[col], minlength=n)
        y = 0.5 * (x + inv * ax)
        nu = y.sum() / x.sum()
        x = y * (n / y.sum())
    return 2.0 * nu - 1.0


def omega_opt(mu: float) -> float:
    """The optimal SOR factor of Eq. 17: 1 + (mu / (1 + sqrt(1 - mu^2)))^2."""
    return 1.0 + (mu / (1.0 + np.sqrt(1.0 - mu * mu))) ** 2
