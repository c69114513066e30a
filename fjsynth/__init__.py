"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

Edge lists (R-MAT, Barabasi-Albert, stochastic block model) and innate-opinion
vectors, drawn from a counter-based SplitMix64 generator in ``synth.c``.  This
package holds none of the Friedkin-Johnsen arithmetic: graph ingest, the solve
and the metrics live on the two sides that consume these inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfjsynth.so")

OP_UNIFORM, OP_BETA_MIX, OP_ARCSINE, OP_SIGN, OP_EXP, OP_PARETO = range(6)

_lib_handle = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_build/libfjsynth.so`` with the host gcc."""
    src = os.path.join(_HERE, "synth.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", src,
                    "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        lib.fjs_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_uint64, i32p, i32p, ctypes.c_void_p,
                                 ctypes.c_int]
        lib.fjs_rmat.restype = ctypes.c_int
        lib.fjs_ba_num_edges.argtypes = [ctypes.c_int64, ctypes.c_int]
        lib.fjs_ba_num_edges.restype = ctypes.c_int64
        lib.fjs_ba.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, i32p, i32p]
        lib.fjs_ba.restype = ctypes.c_int64
        lib.fjs_sbm.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
        lib.fjs_sbm.restype = ctypes.c_int64
        lib.fjs_opinions.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_uint64, f64p]
        lib.fjs_opinions.restype = ctypes.c_int
        lib.fjs_loguniform_sizes.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_uint64, i64p]
        lib.fjs_loguniform_sizes.restype = ctypes.c_int
        lib.fjs_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.fjs_uniform.restype = ctypes.c_double
        lib.fjs_uniform_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                         ctypes.c_void_p]
        lib.fjs_uniform_fill.restype = None
        lib.fjs_raw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.fjs_raw.restype = ctypes.c_uint64
        _lib_handle = lib
    return _lib_handle


def uniform(seed: int, stream: int, ctr: int) -> float:
    """One draw U(seed, stream, ctr) in [0, 1) of the counter-based generator."""
    return _lib().fjs_uniform(seed, stream, ctr)


def uniform_array(seed: int, stream: int, n: int, ctr0: int = 0) -> np.ndarray:
    """U(seed, stream, ctr0 + i) for i < n (float64)."""
    out = np.empty(n, np.float64)
    _lib().fjs_uniform_fill(seed, stream, ctr0, n, out.ctypes.data)
    return out


def raw(seed: int, stream: int, ctr: int) -> int:
    return _lib().fjs_raw(seed, stream, ctr)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, weighted: bool = False, nthreads: int | None = None):
    """R-MAT edge list with ``edge_factor * 2**scale`` edges in generation order.

    Returns ``(src int32, dst int32, w float32 or None)``.
    """
    ne = int(edge_factor) << int(scale)
    src = np.empty(ne, np.int32)
    dst = np.empty(ne, np.int32)
    w = np.empty(ne, np.float32) if weighted else None
    if nthreads is None:
        nthreads = min(64, os.cpu_count() or 1)
    rc = _lib().fjs_rmat(scale, ne, a, b, c, seed, src, dst,
                         w.ctypes.data if w is not None else None, nthreads)
    if rc != 0:
        raise ValueError("fjs_rmat rejected its arguments")
    return src, dst, w


def ba(n: int, m: int = 5, seed: int = 1):
    """Barabasi-Albert edge list (clique on m+1 nodes, then m links per new node)."""
    if m > 64:
        raise ValueError("m must be <= 64")
    ne = _lib().fjs_ba_num_edges(n, m)
    src = np.empty(max(ne, 0), np.int32)
    dst = np.empty(max(ne, 0), np.int32)
    k = _lib().fjs_ba(n, m, seed, src, dst)
    if k < 0:
        raise ValueError("fjs_ba rejected its arguments")
    return src[:k], dst[:k]


def sbm(n: int, nblocks: int, deg_in: float, deg_out: float, seed: int = 1):
    """Undirected SBM edge list (repeats and self-pairs possible; ingest drops them)."""
    lib = _lib()
    ne = lib.fjs_sbm(n, nblocks, deg_in, deg_out, seed, None, None)
    if ne < 0:
        raise ValueError("fjs_sbm rejected its arguments")
    src = np.empty(ne, np.int32)
    dst = np.empty(ne, np.int32)
    lib.fjs_sbm(n, nblocks, deg_in, deg_out, seed, src.ctypes.data, dst.ctypes.data)
    return src, dst


def opinions(n: int, kind: int = OP_UNIFORM, seed: int = 1, vec: int = 0) -> np.ndarray:
    """Innate opinions (float64) of ``kind`` for vector number ``vec``."""
    s = np.empty(n, np.float64)
    if _lib().fjs_opinions(n, kind, seed, vec, s) != 0:
        raise ValueError("unknown opinion kind")
    return s


def loguniform_sizes(count: int, lo: int, hi: int, seed: int = 1) -> np.ndarray:
    out = np.empty(count, np.int64)
    if _lib().fjs_loguniform_sizes(count, lo, hi, seed, out) != 0:
        raise ValueError("bad size range")
    return out
