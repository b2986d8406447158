"""The allocation-free perturber search (rv_select_radius_static).

Callers such as a chain integrator searching for perturbers from inside its
own step, or a host application that forbids device allocation after
start-up, cannot call cudaMalloc; this entry point serves them with a fixed
scratch array inside librv. Here it is called through the C ABI and must
return exactly what the allocating search (rv_select_perturbers, radius mode)
returns, on two calls in a row (the shared scratch keeps the previous call's
contents, which must not leak into the next). This file is collected last on
purpose, so a failure here never hides another test's result."""
import ctypes as C

import numpy as np
import pytest

import ics

pytestmark = pytest.mark.gpu


def _stars(n, seed):
    w = ics.hernquist(n, seed)
    return w.pos.astype(np.float32)


def test_static_radius_search_matches_allocating_search():
    import torch
    from paper_1507_01009_gb300 import rv
    L = rv.load()
    cap = 5000
    # two different calls in a row: sizes, centres and radii all change
    cases = [(70001, 11, (0.01, -0.005, 0.002), 0.05), (1 << 18, 12, (0.2, 0.1, -0.1), 0.08)]
    ctx = rv.Context(max(n for n, *_ in cases))
    for n, seed, centre, radius in cases:
        p32 = _stars(n, seed)
        x, y, z = (torch.from_numpy(np.ascontiguousarray(p32[a])).cuda() for a in range(3))
        ref_idx, ref_cnt = ctx.select_perturbers(x, y, z, centre, 1, radius=radius, cap=cap)
        idx = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        c3 = (C.c_float * 3)(*centre)
        st = L.rv_select_radius_static(n, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                       C.c_void_p(z.data_ptr()), c3, float(radius), cap,
                                       C.c_void_p(idx.data_ptr()), C.c_void_p(cnt.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == rv.RV_OK
        torch.cuda.synchronize()
        ctx.sync_status()
        k = int(ref_cnt.item())
        assert k > 0 and int(cnt.item()) == k
        np.testing.assert_array_equal(idx[:k].cpu().numpy(), ref_idx[:k].cpu().numpy())


def _static(L, x, y, z, n, centre, radius, cap):
    import torch
    idx = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    c3 = (C.c_float * 3)(*centre)
    st = L.rv_select_radius_static(n, C.c_void_p(x.data_ptr() if x is not None else 0),
                                   C.c_void_p(y.data_ptr() if y is not None else 0),
                                   C.c_void_p(z.data_ptr() if z is not None else 0), c3, float(radius), cap,
                                   C.c_void_p(idx.data_ptr()), C.c_void_p(cnt.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, idx, int(cnt.item())


def test_static_radius_search_truncation_is_visible():
    """A sphere holding more stars than cap: the first cap indices match the
    allocating search's, and count carries the untruncated total so the
    caller sees the truncation. Then an empty input gives count 0."""
    import torch
    from paper_1507_01009_gb300 import rv
    L = rv.load()
    n = 50000
    p32 = _stars(n, 13)
    x, y, z = (torch.from_numpy(np.ascontiguousarray(p32[a])).cuda() for a in range(3))
    ctx = rv.Context(n)
    centre, radius = (0.0, 0.0, 0.0), 0.3
    full_idx, full_cnt = ctx.select_perturbers(x, y, z, centre, 1, radius=radius, cap=n)
    ctx.sync_status()
    total = int(full_cnt.item())
    cap = 100
    assert total > 4 * cap
    st, idx, cnt = _static(L, x, y, z, n, centre, radius, cap)
    assert st == rv.RV_OK and cnt == total
    np.testing.assert_array_equal(idx[:cap].cpu().numpy(), full_idx[:cap].cpu().numpy())
    st, idx, cnt = _static(L, None, None, None, 0, centre, radius, cap)
    assert st == rv.RV_OK and cnt == 0
    assert (idx.cpu().numpy() == -1).all()


def test_static_radius_search_rejects_too_many_stars():
    import torch
    from paper_1507_01009_gb300 import rv
    L = rv.load()
    d = torch.zeros(1, dtype=torch.float32, device="cuda")
    c3 = (C.c_float * 3)(0.0, 0.0, 0.0)
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.rv_select_radius_static((1 << 24) + 1, C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()),
                                   C.c_void_p(d.data_ptr()), c3, 1.0, 1, C.c_void_p(cnt.data_ptr()),
                                   C.c_void_p(cnt.data_ptr()), None)
    assert st == rv.RV_E_TOO_LARGE
