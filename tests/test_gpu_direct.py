"""The GPU FP64 direct sum (the reference of the accuracy measurements)
against the oracle's direct sum: softened and unsoftened bodies, coincident
unsoftened bodies, many source chunks, and the edge cases."""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rvmod():
    from paper_1507_01009_gb300 import rv
    rv.load()
    return rv


def _bodies(n, seed, n_hard=3):
    """A Plummer sphere (eps 0.01) plus n_hard unsoftened bodies, two of which
    coincide."""
    w = ics.plummer(n, seed)
    pos = np.concatenate([w.pos, np.array([[0.1, 0.1, 0.3], [0.1, 0.1, 0.3], [-0.5, 0.2, 0.0]])[:n_hard].T], 1)
    m = np.concatenate([w.mass, np.full(n_hard, 0.01)])
    eps = np.concatenate([np.full(n, 0.01), np.zeros(n_hard)])
    return pos, m, eps


def _rel(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def test_direct_matches_oracle(rvmod):
    pos, m, eps = _bodies(4096, 3)
    n = pos.shape[1]
    tg = np.concatenate([np.arange(0, n, 37), [n - 3, n - 2, n - 1]])
    a, p = rvmod.direct_fp64(pos, m, eps, tg)
    ao, po = oracle.direct(pos, m, eps, targets=tg)
    assert _rel(a, ao).max() <= 1e-12
    assert np.abs(p - po).max() <= 1e-12 * np.abs(po).max()


def test_direct_many_chunks_matches_oracle(rvmod):
    """2^18 bodies: the sources are split over many chunks whose partial sums
    are added in order; the result equals the oracle's and repeats bit for bit."""
    pos, m, eps = _bodies(1 << 18, 4, n_hard=1)
    tg = ics.subsample(pos.shape[1], 1000, seed=5)
    a, p = rvmod.direct_fp64(pos, m, eps, tg)
    ao, po = oracle.direct(pos, m, eps, targets=tg)
    assert _rel(a, ao).max() <= 1e-11
    assert np.abs(p - po).max() <= 1e-11 * np.abs(po).max()
    a2, p2 = rvmod.direct_fp64(pos, m, eps, tg)
    assert np.array_equal(a, a2) and np.array_equal(p, p2)


def test_direct_edge_cases(rvmod):
    import torch
    pos, m, eps = _bodies(100, 6)
    # one body: no pairs
    a, p = rvmod.direct_fp64(pos[:, :1], m[:1], eps[:1], [0])
    assert np.all(a == 0) and np.all(p == 0)
    # no targets
    a, p = rvmod.direct_fp64(pos, m, eps, np.zeros(0, np.int64))
    assert a.shape == (3, 0) and p.shape == (0,)
    # a target index outside the bodies: NaN for it, the others unaffected
    a, p = rvmod.direct_fp64(pos, m, eps, [5, 10_000, -1, 7])
    ao, po = oracle.direct(pos, m, eps, targets=[5, 7])
    assert np.all(np.isnan(a[:, 1:3])) and np.all(np.isnan(p[1:3]))
    assert _rel(a[:, [0, 3]], ao).max() <= 1e-12
    # scratch too small
    L = rvmod.load()
    d = dict(dtype=torch.float64, device="cuda")
    x = torch.zeros(4, **d)
    t = torch.zeros(2, dtype=torch.int64, device="cuda")
    o = [torch.empty(2, **d) for _ in range(4)]
    need = int(L.rv_direct_fp64_scratch_bytes(2))
    s = torch.empty(need, dtype=torch.uint8, device="cuda")
    ptr = [rvmod._ptr(u) for u in (x, x, x, x, x)]
    assert L.rv_direct_fp64(4, *ptr, 2, rvmod._ptr(t), *[rvmod._ptr(u) for u in o], rvmod._ptr(s), need - 1,
                            None) == rvmod.RV_E_WORKSPACE
    assert L.rv_direct_fp64(0, *ptr, 2, rvmod._ptr(t), *[rvmod._ptr(u) for u in o], rvmod._ptr(s), need,
                            None) == rvmod.RV_E_INVAL
