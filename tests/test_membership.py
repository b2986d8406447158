"""The chain-membership routines (Sect. 2, Eqs. 4 and 5) against the oracle.

rv_chain_escape is a host routine of librv: it is checked here without a
GPU, bit for bit against the oracle on random chains and on the cases the
rules single out. rv_chain_absorb runs on the GPU and is marked so."""
import numpy as np
import pytest

import ics
import oracle


def _rv():
    from paper_1507_01009_gb300 import build_lib, rv
    build_lib.build()
    return rv


def _same(a, b):
    assert list(a["escape"]) == list(b["escape"])
    assert a["terminate"] == b["terminate"] and a["designated"] == b["designated"]
    assert a["r_chain"] == b["r_chain"] and a["r_escape"] == b["r_escape"]


def test_escape_matches_oracle_on_random_chains():
    """300 random chains (2 to 40 members, one to three SMBHs, members spread
    around the escape radius, random velocities, with and without absorptions
    under way): every flag, the termination and the designated member agree
    with the oracle exactly, and so do r_chain and r_escape (FP64, same
    operation order)."""
    rv = _rv()
    g = ics.rng(61)
    seen = {"escape": 0, "terminate": 0, "handover": 0, "delayed": 0}
    for trial in range(300):
        k = int(g.integers(2, 41))
        nbh = int(g.integers(1, min(3, k) + 1))
        m = np.concatenate([g.uniform(0.002, 0.006, nbh), g.uniform(1e-7, 1e-5, k - nbh)])
        x = g.normal(0, 1, (k, 3)) * g.uniform(0.2, 2.0, (k, 1)) * 0.01
        x[:nbh] *= g.uniform(0, 2.5)
        v = g.normal(0, 1, (k, 3))
        massive = np.r_[np.ones(nbh, np.int32), np.zeros(k - nbh, np.int32)]
        des = int(g.integers(0, nbh))
        r0, gam = 0.008, 1.5
        nab = int(g.integers(0, 3)) if trial % 3 else 0
        a = rv.chain_escape(m, x, v, massive, des, r0, gam, nab)
        b = oracle.chain_escape(m, x, v, massive, des, r0, gam, nab)
        _same(a, b)
        assert a["escape_count"] == int(b["escape"].sum())
        seen["escape"] += int(b["escape"].any())
        seen["terminate"] += b["terminate"]
        seen["handover"] += int(b["designated"] != des)
        seen["delayed"] += int(nab > 0 and not b["escape"].any() and b["r_chain"] > b["r_escape"])
    assert all(v > 0 for v in seen.values()), seen


def test_escape_rejects_bad_arguments():
    rv = _rv()
    with pytest.raises(rv.RvError):
        rv.chain_escape([1.0], [[0, 0, 0]], [[0, 0, 0]], [1], 1, 1.0, 1.5, 0)     # designated out of range
    with pytest.raises(rv.RvError):
        rv.chain_escape([1.0], [[0, 0, 0]], [[0, 0, 0]], [1], 0, -1.0, 1.5, 0)    # negative r_chain0


@pytest.mark.gpu
@pytest.mark.parametrize("n,seed,members", [(1 << 16, 71, 12), (100003, 72, 2), (50000, 73, 40)])
def test_absorb_matches_oracle(n, seed, members):
    """Eq. 4 on the GPU: the stars inside the chain radius of a chain at a
    Hernquist galaxy's centre (an SMBH pair plus stars taken from the galaxy
    as members), bit for bit against the oracle; the same with a cap smaller
    than the count (first cap indices, untruncated count)."""
    import torch
    rv = _rv()
    w = ics.hernquist(n, seed)
    p32 = w.pos.astype(np.float32)
    r = np.linalg.norm(p32.astype(np.float64), axis=0)
    # members: stars drawn from the inner region (not the nearest ones), so that
    # stars inside the chain radius remain in the tree
    inner = np.flatnonzero(r < 0.04)
    near = np.sort(ics.rng(seed).choice(inner, members - 2, replace=False))
    cm = np.concatenate([[0.005, 0.005], np.full(members - 2, 1.0 / n)])
    cx = np.concatenate([[[0.0055, 0.0, 0.0], [-0.0055, 0.0, 0.0]], p32[:, near].T.astype(np.float64)])
    keep = np.setdiff1d(np.arange(n), near)                    # members are no longer tree particles
    ps = np.ascontiguousarray(p32[:, keep])
    ctx = rv.Context(len(keep))
    xs = [torch.from_numpy(np.ascontiguousarray(ps[a])).cuda() for a in range(3)]
    ref, rch = oracle.absorb(ps, cm, cx)
    assert len(ref) > 0
    idx, cnt, rc = ctx.chain_absorb(*xs, cm, cx, cap=len(keep))
    ctx.sync_status()
    assert int(cnt.item()) == len(ref) and float(rc.item()) == rch
    np.testing.assert_array_equal(idx[:len(ref)].cpu().numpy(), ref)
    cap = max(1, len(ref) // 3)
    idx2, cnt2, _ = ctx.chain_absorb(*xs, cm, cx, cap=cap)
    ctx.sync_status()
    assert int(cnt2.item()) == len(ref)
    np.testing.assert_array_equal(idx2[:cap].cpu().numpy(), ref[:cap])
