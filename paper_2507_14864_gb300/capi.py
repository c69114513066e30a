"""Thin Python binding of the C ABI in ``include/fj.h`` (argument marshalling only).

Every computation runs in ``libfj.so``'s CUDA kernels.  Arrays may be numpy
arrays (host memory) or CUDA torch tensors (device memory); the library is
told which through the ``mem`` argument of each call.  There is no fallback:
if ``libfj.so`` has not been built, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfj.so")

FJ_OK, FJ_ERR_INVALID_ARG, FJ_ERR_CUDA, FJ_ERR_OOM, FJ_ERR_NOT_CONVERGED, FJ_ERR_DIVERGED, \
    FJ_ERR_UNSUPPORTED, FJ_ERR_TIMEOUT = range(8)
FJ_MEM_HOST, FJ_MEM_DEVICE = 0, 1
FJ_PREC_FP64, FJ_PREC_FP32 = 0, 1
FJ_SCHED_AUTO, FJ_SCHED_JACOBI, FJ_SCHED_MULTICOLOUR = 0, 1, 2

EXPORTED = [
    "fj_solve_opts_default", "fj_status_string", "fj_last_error", "fj_graph_create",
    "fj_graph_create_from_arcs", "fj_graph_create_ragged", "fj_graph_destroy", "fj_graph_info",
    "fj_graph_export", "fj_graph_colour", "fj_solve", "fj_solve_warm", "fj_solve_batch",
    "fj_metrics", "fj_metrics_batch", "fj_frontier", "fj_frontier_static", "fj_residual", "fj_solve_batch_warm", "fj_graph_order",
    "fj_wait_selftest", "fj_debug_fail_allocation",
    "fj_graph_tune", "fj_graph_tune_batch", "fj_graph_omega_opt", "fj_solve_trace", "fj_mpnn_param_count", "fj_mpnn_create", "fj_mpnn_destroy", "fj_mpnn_get_params", "fj_mpnn_set_params",
    "fj_mpnn_predict", "fj_mpnn_grad", "fj_mpnn_adam_step",
]


class fj_solve_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("omega", ctypes.c_double), ("c", ctypes.c_double),
                ("sigma", ctypes.c_double), ("precision", ctypes.c_int), ("schedule", ctypes.c_int),
                ("max_sweeps", ctypes.c_int64), ("max_refine", ctypes.c_int),
                ("palette", ctypes.c_int), ("check_every", ctypes.c_int), ("profile", ctypes.c_int), ("stream", ctypes.c_void_p)]


class fj_solve_info(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("pushes", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("refine_passes", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("c_eff", ctypes.c_double), ("eps_prime", ctypes.c_double), ("resid_inf", ctypes.c_double),
                ("resid_rel_max", ctypes.c_double), ("z_inf", ctypes.c_double), ("err_bound", ctypes.c_double),
                ("launches", ctypes.c_int64), ("push_launches", ctypes.c_int64), ("push_ms", ctypes.c_double),
                ("push_bytes", ctypes.c_double), ("frontier_rounds", ctypes.c_int64),
                ("frontier_pushes", ctypes.c_int64), ("omega_used", ctypes.c_double),
                ("frontier_edges", ctypes.c_int64), ("method_bytes", ctypes.c_double),
                ("seconds", ctypes.c_double), ("cert_rel_err", ctypes.c_double),
                ("warm_start", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fj_metrics_out(ctypes.Structure):
    _fields_ = [("P", ctypes.c_double), ("D", ctypes.c_double), ("I", ctypes.c_double),
                ("C", ctypes.c_double), ("mean_z", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded ``libfj.so`` with argument types declared; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the CUDA extension is required; there is no CPU path)")
    L = ctypes.CDLL(LIB_PATH)
    VP, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    st = ctypes.c_int
    L.fj_solve_opts_default.argtypes = [ctypes.POINTER(fj_solve_opts)]
    L.fj_solve_opts_default.restype = None
    L.fj_status_string.argtypes = [st]
    L.fj_status_string.restype = ctypes.c_char_p
    L.fj_last_error.argtypes = []
    L.fj_last_error.restype = ctypes.c_char_p
    L.fj_graph_create.argtypes = [I64, VP, VP, VP, I32, I32, VP, ctypes.POINTER(VP)]
    L.fj_graph_create_from_arcs.argtypes = [I64, I64, VP, VP, VP, I32, I32, VP, ctypes.POINTER(VP)]
    L.fj_graph_create_ragged.argtypes = [I32, VP, VP, VP, VP, I32, I32, VP, ctypes.POINTER(VP)]
    L.fj_graph_destroy.argtypes = [VP]
    L.fj_graph_destroy.restype = None
    L.fj_graph_info.argtypes = [VP, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32),
                                ctypes.POINTER(I32)]
    L.fj_graph_export.argtypes = [VP, I32, VP, VP, VP, VP, I32, VP]
    L.fj_graph_colour.argtypes = [VP, I32, VP, ctypes.POINTER(I32), I32, VP]
    L.fj_graph_order.argtypes = [VP, I32, VP, ctypes.POINTER(I64), VP, VP, I32, VP]
    L.fj_wait_selftest.argtypes = [I64, VP]
    L.fj_debug_fail_allocation.argtypes = [I64]
    L.fj_debug_fail_allocation.restype = None
    L.fj_solve.argtypes = [VP, VP, ctypes.POINTER(fj_solve_opts), VP, VP, I32]
    L.fj_solve_warm.argtypes = [VP, VP, VP, ctypes.POINTER(fj_solve_opts), VP, VP, I32]
    L.fj_solve_batch.argtypes = [VP, VP, I32, ctypes.POINTER(fj_solve_opts), VP, VP, I32]
    L.fj_solve_batch_warm.argtypes = [VP, VP, VP, I32, ctypes.POINTER(fj_solve_opts), VP, VP, I32]
    L.fj_metrics.argtypes = [VP, VP, VP, VP, I32, VP]
    L.fj_graph_tune.argtypes = [VP, VP, ctypes.POINTER(fj_solve_opts), I32, ctypes.POINTER(fj_solve_opts),
                                ctypes.POINTER(D), I32]
    L.fj_graph_tune_batch.argtypes = [VP, VP, I32, ctypes.POINTER(fj_solve_opts), I32,
                                      ctypes.POINTER(fj_solve_opts), ctypes.POINTER(D), I32]
    L.fj_metrics_batch.argtypes = [VP, VP, VP, I32, VP, I32, VP]
    L.fj_graph_omega_opt.argtypes = [VP, I32, ctypes.POINTER(D), ctypes.POINTER(D), VP]
    L.fj_solve_trace.argtypes = [VP, VP, ctypes.POINTER(fj_solve_opts), VP, VP, I32, VP, I32,
                                 ctypes.POINTER(I32)]
    L.fj_frontier.argtypes = [I64, VP, VP, I32, VP, VP, VP]
    L.fj_frontier_static.argtypes = [I64, VP, VP, I32, VP, VP, VP]
    L.fj_residual.argtypes = [VP, VP, VP, D, VP, I32, VP]
    L.fj_mpnn_param_count.argtypes = []
    L.fj_mpnn_param_count.restype = I64
    L.fj_mpnn_create.argtypes = [VP, ctypes.POINTER(VP)]
    L.fj_mpnn_destroy.argtypes = [VP]
    L.fj_mpnn_destroy.restype = None
    L.fj_mpnn_get_params.argtypes = [VP, VP]
    L.fj_mpnn_set_params.argtypes = [VP, VP]
    L.fj_mpnn_predict.argtypes = [VP, VP, VP, VP, I32, VP]
    L.fj_mpnn_grad.argtypes = [VP, VP, VP, VP, ctypes.POINTER(D), VP, I32, VP]
    L.fj_mpnn_adam_step.argtypes = [VP, D, VP]
    for name in EXPORTED:
        if name not in ("fj_solve_opts_default", "fj_graph_destroy", "fj_status_string", "fj_last_error",
                        "fj_debug_fail_allocation",
                        "fj_graph_tune", "fj_graph_tune_batch", "fj_mpnn_param_count", "fj_mpnn_destroy"):
            getattr(L, name).restype = st
    _lib = L
    return L


class FJError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().fj_last_error().decode(errors="replace")
        name = lib().fj_status_string(status).decode()
        super().__init__(f"{where}: {name} ({msg})")
        self.status = status


def _check(status: int, where: str, allow=()):
    if status != FJ_OK and status not in allow:
        raise FJError(status, where)
    return status


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _mem_of(*arrays):
    kinds = set()
    for a in arrays:
        if a is None:
            continue
        if _is_torch(a):
            if not a.is_cuda:
                raise ValueError("torch tensors passed to libfj must live on the GPU")
            if not a.is_contiguous():
                raise ValueError("tensors must be contiguous")
            kinds.add(FJ_MEM_DEVICE)
        else:
            kinds.add(FJ_MEM_HOST)
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return kinds.pop() if kinds else FJ_MEM_HOST


def _ptr(a, dtype=None):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    if dtype is not None and a.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {a.dtype}")
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return a.ctypes.data


def current_stream():
    """The current torch CUDA stream handle (or None when CUDA is unavailable)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def default_opts(**kw) -> fj_solve_opts:
    o = fj_solve_opts()
    lib().fj_solve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    if "stream" not in kw:
        o.stream = current_stream()
    return o


class Graph:
    """Owns an ``fj_graph`` handle (device CSR, derived arrays and solve scratch)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)

    # ------------------------------------------------------------ creation
    @classmethod
    def from_csr(cls, n, row_ptr, col, w=None, directed=False, stream=None):
        mem = _mem_of(row_ptr, col, w)
        h = ctypes.c_void_p()
        _check(lib().fj_graph_create(int(n), _ptr(row_ptr, np.int64), _ptr(col, np.int32),
                                     _ptr(w, np.float32), 1 if directed else 0, mem,
                                     stream if stream is not None else current_stream(), ctypes.byref(h)),
               "fj_graph_create")
        return cls(h.value)

    @classmethod
    def from_arcs(cls, n, src, dst, w=None, directed=False, stream=None):
        mem = _mem_of(src, dst, w)
        h = ctypes.c_void_p()
        m = int(src.shape[0])
        _check(lib().fj_graph_create_from_arcs(int(n), m, _ptr(src, np.int32), _ptr(dst, np.int32),
                                               _ptr(w, np.float32), 1 if directed else 0, mem,
                                               stream if stream is not None else current_stream(),
                                               ctypes.byref(h)), "fj_graph_create_from_arcs")
        return cls(h.value)

    @classmethod
    def ragged_from_arcs(cls, graphs, directed=False):
        """A ragged handle from per-graph arc lists [(n, src, dst, w or None), ...] (host
        arrays): each graph goes through the library's own ingest (keep-first dedup,
        self-loops dropped) and export, then the CSRs are laid out block-diagonally."""
        rps, cols, ws, offs = [], [], [], [0]
        nnz_at = 0
        weighted = any(g[3] is not None for g in graphs)
        for n, src, dst, w in graphs:
            one = cls.from_arcs(n, np.ascontiguousarray(src, np.int32), np.ascontiguousarray(dst, np.int32),
                                None if w is None else np.ascontiguousarray(w, np.float32), directed=directed)
            rp, col, wc, _ = one.export(weights=weighted)
            one.close()
            rps.append(rp[1:] + nnz_at)
            cols.append(col + offs[-1])
            if weighted:
                ws.append(wc)
            nnz_at += int(rp[-1])
            offs.append(offs[-1] + int(n))
        row_ptr = np.concatenate([np.zeros(1, np.int64)] + rps).astype(np.int64)
        col = np.concatenate(cols).astype(np.int32)
        w = np.concatenate(ws).astype(np.float32) if weighted else None
        return cls.ragged(np.array(offs, np.int64), row_ptr, col, w, directed=directed)

    @classmethod
    def ragged(cls, node_offsets, row_ptr, col, w=None, directed=False, stream=None):
        mem = _mem_of(node_offsets, row_ptr, col, w)
        h = ctypes.c_void_p()
        ng = int(node_offsets.shape[0]) - 1
        _check(lib().fj_graph_create_ragged(ng, _ptr(node_offsets, np.int64), _ptr(row_ptr, np.int64),
                                            _ptr(col, np.int32), _ptr(w, np.float32), 1 if directed else 0,
                                            mem, stream if stream is not None else current_stream(),
                                            ctypes.byref(h)), "fj_graph_create_ragged")
        return cls(h.value)

    def close(self):
        if self._h and self._h.value:
            lib().fj_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ------------------------------------------------------------ queries
    def info(self):
        n, nnz = ctypes.c_int64(), ctypes.c_int64()
        ng, nc = ctypes.c_int(), ctypes.c_int()
        _check(lib().fj_graph_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(ng),
                                   ctypes.byref(nc)), "fj_graph_info")
        return dict(n=n.value, nnz=nnz.value, ngraphs=ng.value, ncolours=nc.value)

    def export(self, transposed=False, weights=True):
        inf = self.info()
        n, nnz = inf["n"], inf["nnz"]
        rp = np.empty(n + 1, np.int64)
        col = np.empty(nnz, np.int32)
        w = np.empty(nnz, np.float32) if weights else None
        deg = np.empty(n, np.float64)
        _check(lib().fj_graph_export(self._h, 1 if transposed else 0, _ptr(rp), _ptr(col), _ptr(w), _ptr(deg),
                                     FJ_MEM_HOST, current_stream()), "fj_graph_export")
        return rp, col, w, deg

    def colour(self, palette=0):
        n = self.info()["n"]
        out = np.empty(n, np.int32)
        k = ctypes.c_int()
        _check(lib().fj_graph_colour(self._h, int(palette), _ptr(out), ctypes.byref(k), FJ_MEM_HOST,
                                     current_stream()), "fj_graph_colour")
        return out, k.value

    def order(self, palette=16):
        """fj_graph_order: (perm, nhub, hub_row, class_row) of the multicolour row order."""
        _, k = self.colour(palette)
        n = self.info()["n"]
        perm = np.empty(n, np.int32)
        nhub = ctypes.c_int64()
        hub_row = np.empty(k + 1, np.int64)
        class_row = np.empty(k + 1, np.int64)
        _check(lib().fj_graph_order(self._h, int(palette), _ptr(perm), ctypes.byref(nhub), _ptr(hub_row),
                                    _ptr(class_row), FJ_MEM_HOST, current_stream()), "fj_graph_order")
        return perm, nhub.value, hub_row, class_row

    # ------------------------------------------------------------ compute
    def solve(self, s, out=None, z0=None, allow_unconverged=False, **opts):
        """fj_solve / fj_solve_warm.  Returns (z, [fj_solve_info per graph], status)."""
        o = default_opts(**opts)
        ng = self.info()["ngraphs"]
        infos = (fj_solve_info * ng)()
        mem = _mem_of(s, out, z0)
        if out is None:
            if mem == FJ_MEM_DEVICE:
                import torch
                out = torch.empty_like(s)
            else:
                out = np.empty_like(np.asarray(s, np.float64))
        if z0 is None:
            st = lib().fj_solve(self._h, _ptr(s, np.float64), ctypes.byref(o), _ptr(out, np.float64), infos, mem)
            where = "fj_solve"
        else:
            st = lib().fj_solve_warm(self._h, _ptr(s, np.float64), _ptr(z0, np.float64), ctypes.byref(o),
                                     _ptr(out, np.float64), infos, mem)
            where = "fj_solve_warm"
        allow = (FJ_ERR_NOT_CONVERGED, FJ_ERR_DIVERGED) if allow_unconverged else ()
        _check(st, where, allow)
        return out, [i.as_dict() for i in infos], st

    def solve_trace(self, s, out=None, cap=4096, **opts):
        """fj_solve_trace.  Returns (z, [info per graph], status, trace) with trace an
        array of rows [ms, sweeps, max |r| / s', kind (0 push residual, 1 certificate)]."""
        o = default_opts(**opts)
        ng = self.info()["ngraphs"]
        infos = (fj_solve_info * ng)()
        mem = _mem_of(s, out)
        if out is None:
            if mem == FJ_MEM_DEVICE:
                import torch
                out = torch.empty_like(s)
            else:
                out = np.empty_like(np.asarray(s, np.float64))
        rows = np.zeros((int(cap), 4), np.float64)
        count = ctypes.c_int()
        st = lib().fj_solve_trace(self._h, _ptr(s, np.float64), ctypes.byref(o), _ptr(out, np.float64), infos, mem,
                                  rows.ctypes.data_as(ctypes.c_void_p), int(cap), ctypes.byref(count))
        _check(st, "fj_solve_trace")
        return out, [i.as_dict() for i in infos], st, rows[:count.value].copy()

    def solve_batch(self, S, out=None, Z0=None, allow_unconverged=False, **opts):
        """fj_solve_batch (fj_solve_batch_warm with Z0) on node-major S[n, k].
        Returns (Z, [info per vector], status)."""
        o = default_opts(**opts)
        k = int(S.shape[1])
        infos = (fj_solve_info * k)()
        mem = _mem_of(S, out, Z0)
        if out is None:
            if mem == FJ_MEM_DEVICE:
                import torch
                out = torch.empty_like(S)
            else:
                out = np.empty_like(S)
        if Z0 is None:
            st = lib().fj_solve_batch(self._h, _ptr(S, np.float64), k, ctypes.byref(o), _ptr(out, np.float64),
                                      infos, mem)
            where = "fj_solve_batch"
        else:
            st = lib().fj_solve_batch_warm(self._h, _ptr(S, np.float64), _ptr(Z0, np.float64), k, ctypes.byref(o),
                                           _ptr(out, np.float64), infos, mem)
            where = "fj_solve_batch_warm"
        allow = (FJ_ERR_NOT_CONVERGED, FJ_ERR_DIVERGED) if allow_unconverged else ()
        _check(st, where, allow)
        return out, [i.as_dict() for i in infos], st

    def metrics(self, s, z):
        ng = self.info()["ngraphs"]
        outs = (fj_metrics_out * ng)()
        mem = _mem_of(s, z)
        _check(lib().fj_metrics(self._h, _ptr(s, np.float64), _ptr(z, np.float64), outs, mem, current_stream()),
               "fj_metrics")
        res = [m.as_dict() for m in outs]
        return res[0] if ng == 1 else res

    def tune(self, s, reps=2, **opts):
        """fj_graph_tune: the fastest certified (schedule, palette, omega) for s.
        Returns (dict of solve options to pass to solve(), mean ms)."""
        base = default_opts(**opts)
        best = fj_solve_opts()
        ms = ctypes.c_double()
        _check(lib().fj_graph_tune(self._h, _ptr(s, np.float64), ctypes.byref(base), int(reps), ctypes.byref(best),
                                   ctypes.byref(ms), _mem_of(s)), "fj_graph_tune")
        return {"schedule": best.schedule, "palette": best.palette, "omega": best.omega}, ms.value

    def omega_opt(self, iters=200):
        """fj_graph_omega_opt: (mu, omega_opt) of Eq. 17, mu by `iters` power-iteration steps."""
        mu = ctypes.c_double()
        om = ctypes.c_double()
        _check(lib().fj_graph_omega_opt(self._h, int(iters), ctypes.byref(mu), ctypes.byref(om), None),
               "fj_graph_omega_opt")
        return mu.value, om.value

    def tune_batch(self, S, reps=1, **opts):
        """fj_graph_tune_batch; the chosen gather depth stays on the handle."""
        base = default_opts(**opts)
        best = fj_solve_opts()
        ms = ctypes.c_double()
        _check(lib().fj_graph_tune_batch(self._h, _ptr(S, np.float64), int(S.shape[1]), ctypes.byref(base),
                                         int(reps), ctypes.byref(best), ctypes.byref(ms), _mem_of(S)),
               "fj_graph_tune_batch")
        return {"schedule": best.schedule, "palette": best.palette, "omega": best.omega}, ms.value

    def metrics_batch(self, S, Z):
        """fj_metrics_batch on node-major S, Z [n, k]: one dict per vector."""
        k = int(S.shape[1])
        outs = (fj_metrics_out * k)()
        mem = _mem_of(S, Z)
        _check(lib().fj_metrics_batch(self._h, _ptr(S, np.float64), _ptr(Z, np.float64), k, outs, mem,
                                      current_stream()), "fj_metrics_batch")
        return [m.as_dict() for m in outs]

    def residual(self, s, z, c_eff):
        mem = _mem_of(s, z)
        if mem == FJ_MEM_DEVICE:
            import torch
            r = torch.empty_like(s)
        else:
            r = np.empty(np.asarray(s).shape[0], np.float64)
        _check(lib().fj_residual(self._h, _ptr(s, np.float64), _ptr(z, np.float64), float(c_eff), _ptr(r), mem,
                                 current_stream()), "fj_residual")
        return r


def frontier(r, h):
    """fj_frontier on CUDA tensors r, h (float32 or float64).  Returns (list tensor, count)."""
    import torch
    n = int(r.shape[0])
    prec = FJ_PREC_FP32 if r.dtype == torch.float32 else FJ_PREC_FP64
    if h.dtype != r.dtype:
        raise TypeError("r and h must share a dtype")
    lst = torch.empty(max(n, 1), dtype=torch.int32, device=r.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=r.device)
    _check(lib().fj_frontier(n, r.data_ptr(), h.data_ptr(), prec, lst.data_ptr(), cnt.data_ptr(),
                             current_stream()), "fj_frontier")
    c = int(cnt.item())
    return lst[:c], c


class MPNN:
    """Owns an ``fj_mpnn`` handle: the learned warm-start network (parameters,
    Adam state, activations) on the current device."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, np.float32)
        if p.shape != (self.param_count(),):
            raise ValueError(f"expected {self.param_count()} parameters, got {p.shape}")
        h = ctypes.c_void_p()
        _check(lib().fj_mpnn_create(p.ctypes.data, ctypes.byref(h)), "fj_mpnn_create")
        self._h = h

    @staticmethod
    def param_count() -> int:
        return int(lib().fj_mpnn_param_count())

    @classmethod
    def initial_params(cls, seed: int = 0) -> np.ndarray:
        """A start for training: each weight matrix uniform in +-1/sqrt(2 F_in)
        (F_in = 4, 64, 64), zero biases, head weights uniform in +-1/8."""
        rng = np.random.default_rng(seed)
        parts = []
        for fin in (4, 64, 64):
            lim = 1.0 / np.sqrt(2 * fin)
            parts += [rng.uniform(-lim, lim, fin * 64), rng.uniform(-lim, lim, fin * 64), np.zeros(64)]
        parts += [rng.uniform(-0.125, 0.125, 64), np.zeros(1)]
        p = np.concatenate(parts).astype(np.float32)
        assert p.shape[0] == cls.param_count()
        return p

    def close(self):
        if self._h and self._h.value:
            lib().fj_mpnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.param_count(), np.float32)
        _check(lib().fj_mpnn_get_params(self._h, out.ctypes.data), "fj_mpnn_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        _check(lib().fj_mpnn_set_params(self._h, p.ctypes.data), "fj_mpnn_set_params")

    def predict(self, graph: "Graph", s, out=None):
        mem = _mem_of(s, out)
        if out is None:
            if mem == FJ_MEM_DEVICE:
                import torch
                out = torch.empty_like(s)
            else:
                out = np.empty(np.asarray(s).shape[0], np.float64)
        _check(lib().fj_mpnn_predict(self._h, graph.handle, _ptr(s, np.float64), _ptr(out, np.float64), mem,
                                     current_stream()), "fj_mpnn_predict")
        return out

    def grad(self, graph: "Graph", s, z, want_grad=True):
        """Loss and (optionally) the gradient (host FP32) on one triple; keeps it for adam_step."""
        mem = _mem_of(s, z)
        loss = ctypes.c_double()
        g = np.empty(self.param_count(), np.float32) if want_grad else None
        _check(lib().fj_mpnn_grad(self._h, graph.handle, _ptr(s, np.float64), _ptr(z, np.float64),
                                  ctypes.byref(loss), None if g is None else g.ctypes.data, mem,
                                  current_stream()), "fj_mpnn_grad")
        return loss.value, g

    def adam_step(self, lr: float):
        _check(lib().fj_mpnn_adam_step(self._h, float(lr), current_stream()), "fj_mpnn_adam_step")

    def train_step(self, graph: "Graph", s, z, lr: float) -> float:
        loss, _ = self.grad(graph, s, z, want_grad=False)
        self.adam_step(lr)
        return loss
