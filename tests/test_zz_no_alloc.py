"""fj_frontier_static against fj_frontier, through the C ABI.

fj_frontier_static serves callers that cannot allocate device memory (a
process whose device memory is all handed out up front by its own pool or
arena, where a cudaMalloc would fail or take memory promised elsewhere): its
scratch is a fixed array inside the library.  Its output must equal the
allocating entry point's, bit for bit, on consecutive calls that reuse that
array, from the empty input up to the largest n the array serves.  This file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _frontier(capi, fn, r, h):
    import torch
    n = int(r.shape[0])
    prec = capi.FJ_PREC_FP32 if r.dtype == torch.float32 else capi.FJ_PREC_FP64
    lst = torch.full((max(n, 1),), -7, dtype=torch.int32, device=r.device)
    cnt = torch.full((1,), -1, dtype=torch.int64, device=r.device)
    st = fn(n, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(h.data_ptr()), prec,
            ctypes.c_void_p(lst.data_ptr()), ctypes.c_void_p(cnt.data_ptr()), capi.current_stream())
    assert st == capi.FJ_OK, capi.lib().fj_last_error()
    c = int(cnt.item())
    return lst[:c].cpu().numpy(), c


def _frontier_n(capi, fn, n, r, h):
    """_frontier on the first n entries of r and h (n may be 0)."""
    import torch
    prec = capi.FJ_PREC_FP32 if r.dtype == torch.float32 else capi.FJ_PREC_FP64
    lst = torch.full((max(n, 1),), -7, dtype=torch.int32, device=r.device)
    cnt = torch.full((1,), -1, dtype=torch.int64, device=r.device)
    st = fn(n, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(h.data_ptr()), prec,
            ctypes.c_void_p(lst.data_ptr()), ctypes.c_void_p(cnt.data_ptr()), capi.current_stream())
    assert st == capi.FJ_OK, capi.lib().fj_last_error()
    c = int(cnt.item())
    return lst[:c].cpu().numpy(), c


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_static_scratch_frontier_matches_allocating_one(dtype):
    import torch
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi
    lib = capi.lib()
    rng = np.random.default_rng(2026)
    for n in (300001, 4099):  # two calls in a row, the second on a smaller case
        h = rng.random(n).astype(dtype)
        r = ((rng.random(n) * 2 - 1) * 1.5).astype(dtype)
        r[::11] = h[::11]  # |r| == h is not in the frontier
        rd, hd = torch.from_numpy(r).cuda(), torch.from_numpy(h).cuda()
        want, cw = _frontier(capi, lib.fj_frontier, rd, hd)
        got, cg = _frontier(capi, lib.fj_frontier_static, rd, hd)
        assert cg == cw and np.array_equal(got, want)


def test_static_scratch_empty_and_largest_inputs():
    import torch
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi
    lib = capi.lib()
    # n = 0: nothing selected, the count is still written
    e = torch.zeros(1, dtype=torch.float32, device="cuda")
    want, cw = _frontier_n(capi, lib.fj_frontier, 0, e, e)
    got, cg = _frontier_n(capi, lib.fj_frontier_static, 0, e, e)
    assert cw == 0 and cg == 0
    # n = 2^26 (the last status word of the array) and 2^26 - 1, a sparse frontier
    big = 1 << 26
    gen = torch.Generator(device="cuda").manual_seed(7)
    h = torch.full((big,), 0.5, dtype=torch.float32, device="cuda")
    r = torch.zeros(big, dtype=torch.float32, device="cuda")
    hit = torch.randint(0, big, (4096,), device="cuda", generator=gen)
    r[hit] = 0.75
    r[big - 1] = -0.9  # the last node is in the frontier
    for n in (big, big - 1):
        want, cw = _frontier_n(capi, lib.fj_frontier, n, r, h)
        got, cg = _frontier_n(capi, lib.fj_frontier_static, n, r, h)
        assert cg == cw and cw > 0 and np.array_equal(got, want)
    del r, h
    torch.cuda.empty_cache()


def test_static_scratch_rejects_oversized_input():
    import torch
    import __graft_entry__

    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi
    lib = capi.lib()
    x = torch.zeros(1, dtype=torch.float32, device="cuda")
    lst = torch.zeros(1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = lib.fj_frontier_static((1 << 26) + 1, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                capi.FJ_PREC_FP32, ctypes.c_void_p(lst.data_ptr()),
                                ctypes.c_void_p(cnt.data_ptr()), capi.current_stream())
    assert st == capi.FJ_ERR_INVALID_ARG
    assert b"static scratch limit" in lib.fj_last_error()
