"""GPU parity of the walk under the relative opening criterion (Sect. 3's
"Gadget" criterion with an error tolerance) against the CPU oracle: the same
FP32 decision on both sides, so with equal-mass stars of mass 2^-k (cell
masses exact in FP32) the interaction counts match exactly; forces match the
oracle tree to a median relative error <= 1e-5 and a maximum <= 1e-4, and the
FP64 direct sum to p99 below the tolerance. Reference accelerations come from
the oracle (direct sum or its tree), never from the CUDA path."""
import numpy as np
import pytest

import ics
import oracle
from gpu_helpers import err_stats, gpu_tree, hernquist32, stars32, to_dev

pytestmark = pytest.mark.gpu

MED_TOL, MAX_TOL = 1e-5, 1e-4


@pytest.fixture(scope="module")
def rvmod():
    from paper_1507_01009_gb300 import rv
    rv.load()
    return rv


def _case(kind, n):
    if kind == "plummer":
        w = ics.plummer(n, 1)
        return stars32(w.pos, w.mass)
    if kind == "two_clusters":
        g = ics.rng(17)
        a = g.normal(0, 1e-3, (3, n // 2))
        b = g.normal(0, 1e-3, (3, n - n // 2)) + 50.0
        return stars32(np.concatenate([a, b], 1), np.full(n, 1.0 / n))
    return hernquist32(n, 5 + n)


def _aref_direct(p32, m32, eps):
    """Reference accelerations (FP32, (3, n)) from the oracle's direct sum."""
    ad, _ = oracle.direct(p32.astype(np.float64), m32.astype(np.float64), eps)
    return ad.astype(np.float32), ad


def _dev3(a):
    return tuple(to_dev(np.ascontiguousarray(a[k])) for k in range(3))


RELMAC_CASES = [("plummer", 4096, 1e-3, 0.01, 16, 32, 64, True), ("hernquist", 65536, 1e-3, 0.005, 32, 64, 128, True),
                ("hernquist", 65536, 1e-2, 0.005, 16, 32, 64, True), ("plummer", 4096, 3e-3, 0.01, 8, 47, 32, False),
                ("two_clusters", 4096, 1e-3, 0.001, 16, 64, 64, True), ("hernquist", 16384, 1e-3, 0.0, 16, 32, 64, True)]


@pytest.mark.parametrize("kind,n,alpha,eps,n_leaf,G,tile,quad", RELMAC_CASES)
def test_relmac_forces_vs_oracle_tree(rvmod, kind, n, alpha, eps, n_leaf, G, tile, quad):
    p32, m32 = _case(kind, n)
    eps = float(np.float32(eps))
    aref, ad = _aref_direct(p32, m32, eps)
    ctx = rvmod.Context(n, theta=0.5, eps_star=eps, n_leaf=n_leaf, group=G, tile=tile, quadrupole=quad)
    gpu_tree(ctx, p32, m32)
    ax, ay, az, pot = ctx.tree_forces_rel(alpha, _dev3(aref), eps_star=eps)
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    p = pot.cpu().numpy().astype(np.float64)
    T = oracle.Tree(p32, m32, n_leaf, G)
    ao, po, cnt = T.forces_rel(alpha, eps, aref, quad, counts=True)
    med, p99, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL, (med, p99, mx)
    ep = np.abs(p - po) / np.abs(po)
    assert np.median(ep) <= MED_TOL and ep.max() <= MAX_TOL
    # the same FP32 decisions: identical interaction counts (the GPU counts each star's own pair)
    n_p2p, n_m2p = ctx.walk_stats()
    assert n_p2p == int(cnt[:, 0].sum()) + n
    assert n_m2p == int(cnt[:, 1].sum())
    if quad:
        _, p99d, _ = err_stats(a, ad)
        assert p99d < alpha, p99d


def test_relmac_zero_tolerance_is_direct_sum(rvmod):
    p32, m32 = _case("hernquist", 3000)
    eps = float(np.float32(0.005))
    aref, ad = _aref_direct(p32, m32, eps)
    ctx = rvmod.Context(3000, eps_star=eps)
    gpu_tree(ctx, p32, m32)
    ax, ay, az, _ = ctx.tree_forces_rel(0.0, _dev3(aref))
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    assert err_stats(a, ad)[2] <= 1e-5
    assert ctx.walk_stats()[1] == 0


def test_relmac_rejects_bad_arguments(rvmod):
    p32, m32 = _case("plummer", 256)
    ctx = rvmod.Context(256)
    gpu_tree(ctx, p32, m32)
    with pytest.raises(rvmod.RvError):
        ctx.tree_forces_rel(-1.0, _dev3(np.ones((3, 256), np.float32)))


@pytest.mark.slow
@pytest.mark.parametrize("G,n_leaf,tile", [(64, 32, 128), (64, 24, 128)])
def test_relmac_full_size_sampled(rvmod, G, n_leaf, tile):
    """2^20 Hernquist stars at the paper's tolerance 1e-3, reference |a| from
    the oracle tree at theta = 0.5: sampled stars against the oracle under the
    same criterion and against the FP64 direct sum."""
    n = 1 << 20
    w = ics.hernquist_bh_workload(n, seed=2)
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(w.eps_star))
    T = oracle.Tree(p32, m32, n_leaf, G)
    a0, _, _, _ = T.forces(0.5, eps, True)
    aref = a0.astype(np.float32)
    ctx = rvmod.Context(n, eps_star=eps, n_leaf=n_leaf, group=G, tile=tile)
    gpu_tree(ctx, p32, m32)
    ax, ay, az, _ = ctx.tree_forces_rel(1e-3, _dev3(aref))
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    tg = ics.subsample(n, 512, seed=19)
    ao, _ = T.forces_rel(1e-3, eps, aref, targets=tg)
    med, _, mx = err_stats(a[:, tg], ao[:, tg])
    assert med <= MED_TOL and mx <= MAX_TOL
    ad, _ = oracle.direct(p32.astype(np.float64), m32.astype(np.float64), eps, targets=tg)
    _, p99, _ = err_stats(a[:, tg], ad)
    assert p99 <= 1e-3


def test_relmac_system_forces_and_kdk(rvmod):
    """cfg.mac = 1 in the full force pass (stars + one SMBH, perturbers within
    r = 0.02): the stars' groups use the relative criterion with the system's
    accelerations as references, the SMBH's centre-of-mass walk uses theta.
    References are written into the system by the test (from the oracle's
    direct sum); the result is compared with the oracle following the same
    steps. Zero references (before any pass) give the theta walk exactly, and
    a KDK step with cfg.mac = 1 runs."""
    import torch
    from test_gpu_parity import _oracle_system_forces, _system
    w = ics.hernquist_bh_workload(1 << 16, seed=12)
    w.chain.pos[0] = [0.02, 0.0, 0.0]
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(w.eps_star))
    n = p32.shape[1]
    ctx = rvmod.Context(n, theta=0.5, eps_star=eps, mac=1, alpha=1e-3)
    ctx0 = rvmod.Context(n, theta=0.5, eps_star=eps)
    S = _system(rvmod, w, n, pert_mode=1, pert_radius=0.02)
    S0 = _system(rvmod, w, n, pert_mode=1, pert_radius=0.02)
    ctx.system_forces(S)                       # zero references: theta everywhere
    ctx0.system_forces(S0)
    ctx.sync_status()
    for u, v in ((S.ax, S0.ax), (S.ay, S0.ay), (S.az, S0.az), (S.pot, S0.pot)):
        assert torch.equal(u, v)
    # references from the oracle's direct sum (stars and SMBH)
    allp = np.concatenate([p32.astype(np.float64), w.chain.pos.T], 1)
    allm = np.concatenate([m32.astype(np.float64), w.chain.mass])
    epsv = np.concatenate([np.full(n, eps), [0.0]])
    ad, _ = oracle.direct(allp, allm, epsv, targets=np.arange(n))
    aref = ad.astype(np.float32)
    for k, t in enumerate((S.ax, S.ay, S.az)):
        t.copy_(torch.from_numpy(np.ascontiguousarray(aref[k])))
    ctx.system_forces(S)
    ctx.sync_status()
    com32 = w.chain.com.astype(np.float32)
    pert = oracle.radius(p32, com32, np.float32(np.float32(0.02) * np.float32(0.02)))
    T = oracle.Tree(p32, m32, 16, 32)
    xp = w.chain.com.astype(np.float32).reshape(3, 1)
    xm = np.array([np.float32(w.chain.total_mass)], dtype=np.float64)
    ao, _, xa, _ = T.forces(0.5, eps, True, xp, xm, [0.0], rel=(1e-3, aref))
    o = oracle.perturber(w.chain.mass, w.chain.pos, m32[pert].astype(np.float64), p32[:, pert].T.astype(np.float64))
    ao[:, pert] += o["a_pert"].T
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    med, _, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL, (med, mx)
    _, p99, _ = err_stats(a, ad)
    assert p99 <= 1e-3
    a_bh = xa[:, 0] - o["sub"] + o["a_chain"][0]
    got = S.chain_a.cpu().numpy()[:3]
    assert np.linalg.norm(got - a_bh) / np.linalg.norm(a_bh) <= MAX_TOL
    ctx.kdk_step(S, 1e-3, 2)
    ctx.sync_status()
    assert torch.isfinite(S.ax).all()


def test_relmac_in_place_references(rvmod):
    """The reference arrays may be the output arrays: each group reads its own
    stars' references before writing their forces, so the result equals the
    call with separate arrays bit for bit."""
    import torch
    p32, m32 = _case("hernquist", 65536)
    eps = float(np.float32(0.005))
    aref, _ = _aref_direct(p32, m32, eps)
    ctx = rvmod.Context(65536, eps_star=eps, group=64, n_leaf=32, tile=128)
    gpu_tree(ctx, p32, m32)
    sep = ctx.tree_forces_rel(1e-3, _dev3(aref))
    out = list(_dev3(aref)) + [torch.empty(65536, device="cuda")]
    ctx.tree_forces_rel(1e-3, tuple(out[:3]), out=out)
    ctx.sync_status()
    for u, v in zip(sep, out):
        assert torch.equal(u, v)
