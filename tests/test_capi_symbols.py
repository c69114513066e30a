"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/fj.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    text = open(os.path.join(ROOT, "include", "fj.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fj_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi
    return capi.lib()


def test_header_declares_entry_points():
    names = declared()
    assert "fj_solve" in names and "fj_graph_create" in names and "fj_metrics" in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert missing == []


def test_binding_names_match_header(lib):
    from paper_2507_14864_gb300 import capi
    assert sorted(capi.EXPORTED) == declared()


def test_status_strings_and_defaults(lib):
    from paper_2507_14864_gb300 import capi
    assert lib.fj_status_string(capi.FJ_ERR_DIVERGED) == b"diverged"
    o = capi.fj_solve_opts()
    lib.fj_solve_opts_default(ctypes.byref(o))
    assert o.eps == 1e-6 and o.omega == 1.0 and o.c == 1e-5 and o.sigma == 1e-5
    assert o.max_refine == 8 and o.precision == capi.FJ_PREC_FP64


def test_argument_checks_need_no_gpu(lib):
    from paper_2507_14864_gb300 import capi
    h = ctypes.c_void_p()
    st = lib.fj_graph_create(0, None, None, None, 0, 0, None, ctypes.byref(h))
    assert st == capi.FJ_ERR_INVALID_ARG
    assert b"n must be" in lib.fj_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2507_14864_gb300 import capi
    monkeypatch.setattr(capi, "_lib", None)
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU path"):
        capi.lib()


def test_new_entry_points_check_arguments_without_gpu(lib):
    from paper_2507_14864_gb300 import capi
    mu, om = ctypes.c_double(), ctypes.c_double()
    assert lib.fj_graph_omega_opt(None, 10, ctypes.byref(mu), ctypes.byref(om), None) == capi.FJ_ERR_INVALID_ARG
    o = capi.fj_solve_opts()
    lib.fj_solve_opts_default(ctypes.byref(o))
    cnt = ctypes.c_int()
    st = lib.fj_solve_trace(None, None, ctypes.byref(o), None, None, capi.FJ_MEM_HOST, None, 4, ctypes.byref(cnt))
    assert st == capi.FJ_ERR_INVALID_ARG
    assert b"graph is NULL" in lib.fj_last_error()
