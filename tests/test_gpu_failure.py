"""Failure paths in the forms that fault no GPU.

- Bounded device waits: the library's two kinds of wait (a scan look-back on
  a tile status word, the bulk-copy ring on an mbarrier), run on something
  that nothing completes, give up after their poll limit and report
  FJ_ERR_TIMEOUT; the context stays usable: a solve afterwards certifies.
- A device allocation that fails (made to fail on the host by the library's
  allocation hook, as a full device would): the call returns FJ_ERR_OOM, and
  the same handle solves correctly once memory is available again.
"""
import numpy as np
import pytest

import oracle
from fjsynth import workloads as W
from gpu_common import FP32_TOL, csr_of, rel_inf, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi as c
    return c


def _small(capi):
    g = W.ba_graph(2500, 4, seed_off=91)
    rp, col, w = csr_of(g)
    s = g["S"][0]
    z_star, _ = oracle.truth(g["n"], rp, col, w, s)
    return g["n"], rp, col, w, s, z_star


def test_bounded_waits_give_up_and_context_survives(capi):
    lib = capi.lib()
    for polls in (1, 1000):
        st = lib.fj_wait_selftest(polls, capi.current_stream())
        assert st == capi.FJ_ERR_TIMEOUT, lib.fj_last_error()
        assert b"gave up" in lib.fj_last_error()
    n, rp, col, w, s, z_star = _small(capi)
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    z, info, st = G.solve(to_dev(s)[0], eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    assert rel_inf(z.cpu().numpy(), z_star) <= FP32_TOL


@pytest.mark.parametrize("after", [0, 1, 3])
def test_failed_allocation_reports_oom_and_handle_recovers(capi, after):
    lib = capi.lib()
    n, rp, col, w, s, z_star = _small(capi)
    G = capi.Graph.from_csr(n, *to_dev(rp, col, w), directed=False)
    (s_d,) = to_dev(s)
    opts = dict(eps=1e-6, omega=1.5, precision=capi.FJ_PREC_FP32)
    lib.fj_debug_fail_allocation(after)
    try:
        with pytest.raises(capi.FJError) as ei:
            G.solve(s_d, **opts)
        assert ei.value.status == capi.FJ_ERR_OOM
    finally:
        lib.fj_debug_fail_allocation(-1)
    z, info, st = G.solve(s_d, **opts)
    assert st == capi.FJ_OK and info[0]["converged"] == 1
    assert rel_inf(z.cpu().numpy(), z_star) <= FP32_TOL
    G.close()
