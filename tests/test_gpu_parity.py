"""GPU parity: librv (through its C ABI) against the CPU oracle on the same
seeded inputs. Integer work (keys, permutation, topology, groups, perturber
selection) must match bit for bit; forces must match the oracle tree at the
same opening angle to a median relative error <= 1e-5 and a maximum <= 1e-4,
and the FP64 direct sum at p99 <= 1e-3 (theta = 0.5, quadrupole)."""
import math

import numpy as np
import pytest

import ics
import oracle
from gpu_helpers import (err_stats, gpu_cells_as_oracle, gpu_com, gpu_tree, hernquist32, sorted_groups, stars32,
                         to_dev)

pytestmark = pytest.mark.gpu

MED_TOL, MAX_TOL, P99_DIRECT = 1e-5, 1e-4, 1e-3


@pytest.fixture(scope="module")
def rvmod():
    from paper_1507_01009_gb300 import rv
    rv.load()
    return rv


def _ctx(rv, n, **kw):
    return rv.Context(max(n, 1), **kw)


def _inputs(kind, n, seed=0):
    if kind == "hernquist":
        return hernquist32(n, seed + n)
    if kind == "plummer":
        w = ics.plummer(n, seed + 1)
        return stars32(w.pos, w.mass)
    if kind == "coincident":
        return np.full((3, n), 0.3, dtype=np.float32), np.full(n, 1.0 / n, dtype=np.float32)
    if kind == "two_clusters":
        g = ics.rng(seed + 7)
        a = g.normal(0, 1e-3, (3, n // 2))
        b = g.normal(0, 1e-3, (3, n - n // 2)) + 50.0
        return stars32(np.concatenate([a, b], 1), np.full(n, 1.0 / n))
    if kind == "ghosts":                                      # near-massless chain ghosts (Sect. 2)
        p, m = hernquist32(n, seed + 3)
        m = m.copy()
        m[::5] = 1e-30
        return p, m
    if kind == "lattice":                                     # stars exactly on cell boundaries
        k = round(n ** (1 / 3))
        g = np.arange(k, dtype=np.float64) / (k - 1)          # 0 .. 1: the bounding cube's corners
        q = np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1)
        return q.astype(np.float32), np.full(q.shape[1], 1.0 / q.shape[1], dtype=np.float32)
    raise ValueError(kind)


TREE_CASES = [("hernquist", 1, 16, 32), ("hernquist", 2, 16, 32), ("hernquist", 3, 1, 1), ("hernquist", 7, 2, 4),
              ("hernquist", 33, 16, 32), ("hernquist", 1000, 8, 32), ("hernquist", 4097, 16, 32),
              ("hernquist", 65659, 16, 32), ("plummer", 4096, 16, 32), ("coincident", 100, 16, 32),
              ("two_clusters", 3000, 16, 32), ("ghosts", 5000, 16, 32), ("hernquist", 20000, 32, 32),
              ("hernquist", 20000, 4, 8), ("hernquist", 20000, 16, 64), ("hernquist", 4097, 8, 48),
              ("coincident", 100, 16, 64), ("lattice", 4913, 8, 32), ("lattice", 4096, 1, 1)]


@pytest.mark.parametrize("kind,n,n_leaf,G", TREE_CASES)
def test_tree_bit_exact(rvmod, kind, n, n_leaf, G):
    p32, m32 = _inputs(kind, n)
    ctx = _ctx(rvmod, n, n_leaf=n_leaf, group=G)
    gpu_tree(ctx, p32, m32)
    v = ctx.tree_view()
    ctx.sync_status()
    T = oracle.Tree(p32, m32, n_leaf, G)
    np.testing.assert_array_equal(v["bounds"].cpu().numpy(), np.array([*T.lo, T.L, T.scale]))
    np.testing.assert_array_equal(v["keys"].cpu().numpy().view(np.uint64), T.key)
    np.testing.assert_array_equal(v["perm"].cpu().numpy(), T.perm)
    pos = v["pos"].cpu().numpy()
    np.testing.assert_array_equal(pos[:, 0], p32[0][T.perm])
    np.testing.assert_array_equal(pos[:, 3], m32[T.perm])
    assert v["ncell"] == T.ncell
    np.testing.assert_array_equal(gpu_cells_as_oracle(v), T.cells)
    assert v["ngroup"] == T.ngroup
    np.testing.assert_array_equal(sorted_groups(v["groups"].cpu().numpy()), sorted_groups(T.groups))


def _adversarial_coords(seed, lo, hi):
    """FP32 coordinates (3, n) that sit on, and one or two FP32 steps either
    side of, the quantisation grid's cell boundaries (exactly on them when the
    extent hi - lo is a power of two), with tiny magnitudes and a negative
    minimum: the cases in which the key's floor is decided next to an
    integer."""
    g = ics.rng(seed)
    lo = np.float32(lo)
    hi = np.float32(hi)
    L = float(hi) - float(lo)
    k = g.integers(0, 1 << 21, 30000)
    on = (float(lo) + k * (L / 2.0 ** 21)).astype(np.float32)
    near = np.concatenate([on, np.nextafter(on, np.float32(np.inf)), np.nextafter(on, np.float32(-np.inf)),
                           np.nextafter(np.nextafter(on, np.float32(np.inf)), np.float32(np.inf))])
    extra = np.array([lo, hi, 0.0, 1e-30, -1e-30, 1e-38, np.float32(2.0 ** -149), 1.0, -1.0, 3.3333333],
                     dtype=np.float32)
    v = np.concatenate([near, extra, g.uniform(float(lo), float(hi), 20000).astype(np.float32)])
    v = np.clip(v, lo, hi).astype(np.float32)
    pos = np.stack([v, g.permutation(v), g.permutation(v)]).astype(np.float32)
    pos[1, 0], pos[2, 0] = lo, lo       # every axis reaches the same minimum and extent
    pos[1, 1], pos[2, 1] = hi, hi
    return pos


@pytest.mark.parametrize("seed,lo,hi", [(1, -4.0, 12.0), (2, -3.7, 11.3), (3, 0.0, 1.0)])
def test_keys_exact_next_to_grid_boundaries(rvmod, seed, lo, hi):
    """Morton keys bit-exact against the oracle's FP64 quantisation on
    coordinates placed on and next to the grid's cell boundaries."""
    p32 = _adversarial_coords(seed, lo, hi)
    n = p32.shape[1]
    m32 = np.full(n, 1.0 / n, dtype=np.float32)
    ctx = _ctx(rvmod, n)
    gpu_tree(ctx, p32, m32)
    v = ctx.tree_view()
    ctx.sync_status()
    k = np.zeros(n, dtype=np.uint64)
    k[v["perm"].cpu().numpy()] = v["keys"].cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(k, oracle.keys(p32))


def test_tiny_golden_tree_on_gpu(rvmod):
    """The hand-derived five-point tree (tests/golden/tiny_tree.txt)."""
    from test_oracle import _read_sections
    g = _read_sections("tiny_tree.txt")
    p32 = np.array(g["points"], dtype=np.float32).T
    ctx = _ctx(rvmod, 5, n_leaf=2, group=2)
    gpu_tree(ctx, p32, np.ones(5, np.float32))
    v = ctx.tree_view()
    np.testing.assert_array_equal(v["perm"].cpu().numpy(), np.array(g["perm"][0]))
    np.testing.assert_array_equal(gpu_cells_as_oracle(v), np.array(g["cells"]))
    np.testing.assert_array_equal(sorted_groups(v["groups"].cpu().numpy()), sorted_groups(g["groups"]))


@pytest.mark.parametrize("kind,n", [("hernquist", 65659), ("plummer", 4096), ("ghosts", 5000), ("coincident", 100),
                                    ("two_clusters", 3000)])
def test_moments(rvmod, kind, n):
    """FP32 multipoles vs FP64 brute force per cell: mass to 1e-6 relative,
    centre of mass to 1e-6 of the cell side, quadrupole to 1e-5 of M s^2."""
    p32, m32 = _inputs(kind, n)
    ctx = _ctx(rvmod, n)
    gpu_tree(ctx, p32, m32)
    v = ctx.tree_view()
    T = oracle.Tree(p32, m32, 16, 32)
    g = v["cmom"].cpu().numpy().astype(np.float64)
    o = T.moments
    side = T.L / 2 ** 21 * 2.0 ** (21 - T.cells[:, 0])
    M = o[:, 0]
    np.testing.assert_allclose(g[:, 0], M, rtol=1e-6, atol=1e-37)
    scale = np.maximum(side, 1e-30)
    com = gpu_com(v)
    assert np.all(np.abs(com - o[:, 1:4]).max(1) <= 1e-6 * scale)
    gq = g[:, [4, 5, 6, 7, 8, 9]]
    oq = o[:, 4:10]
    qs = np.maximum(M * side * side, 1e-37)
    assert np.all(np.abs(gq - oq).max(1) <= 1e-5 * qs)


FORCE_CASES = [("plummer", 4096, 0.5, 0.01, 16, 32, 64, True), ("hernquist", 65659, 0.5, 0.005, 16, 32, 64, True),
               ("hernquist", 65659, 0.7, 0.005, 8, 16, 32, True), ("hernquist", 30000, 0.5, 0.005, 16, 32, 128, False),
               ("ghosts", 5000, 0.5, 0.005, 16, 32, 64, True), ("two_clusters", 3000, 0.6, 0.001, 4, 8, 64, True),
               ("hernquist", 1000, 0.5, 0.0, 16, 32, 64, True), ("hernquist", 65659, 0.5, 0.005, 32, 64, 128, True),
               ("plummer", 4096, 0.6, 0.01, 16, 64, 64, True), ("two_clusters", 3000, 0.5, 0.001, 8, 47, 32, True),
               ("ghosts", 5000, 0.5, 0.005, 16, 64, 64, False),
               # the configuration limits: largest leaf, group and tile; one star per leaf and group
               ("hernquist", 65659, 0.5, 0.005, 64, 64, 256, True), ("plummer", 4096, 0.5, 0.01, 1, 1, 32, True)]


@pytest.mark.parametrize("kind,n,theta,eps,n_leaf,G,tile,quad", FORCE_CASES)
def test_forces_vs_oracle_tree(rvmod, kind, n, theta, eps, n_leaf, G, tile, quad):
    p32, m32 = _inputs(kind, n)
    eps = float(np.float32(eps))
    ctx = _ctx(rvmod, n, theta=theta, eps_star=eps, n_leaf=n_leaf, group=G, tile=tile, quadrupole=quad)
    gpu_tree(ctx, p32, m32)
    ax, ay, az, pot = ctx.tree_forces()
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    p = pot.cpu().numpy().astype(np.float64)
    T = oracle.Tree(p32, m32, n_leaf, G)
    ao, po, _, _, cnt = T.forces(theta, eps, quad, counts=True)
    med, p99, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL, (med, p99, mx)
    ep = np.abs(p - po) / np.abs(po)
    assert np.median(ep) <= MED_TOL and ep.max() <= MAX_TOL
    # identical opening decisions: same interaction counts (the GPU also counts each star's own pair)
    n_p2p, n_m2p = ctx.walk_stats()
    assert n_p2p == int(cnt[:, 0].sum()) + n
    assert n_m2p == int(cnt[:, 1].sum())


def test_forces_vs_direct_plummer(rvmod):
    p32, m32 = _inputs("plummer", 4096)
    ctx = _ctx(rvmod, 4096, theta=0.5, eps_star=0.01)
    gpu_tree(ctx, p32, m32)
    ax, ay, az, _ = ctx.tree_forces()
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    ad, _ = oracle.direct(p32.astype(np.float64), m32.astype(np.float64), float(np.float32(0.01)))
    _, p99, _ = err_stats(a, ad)
    assert p99 <= P99_DIRECT


def test_small_theta_is_direct_sum(rvmod):
    """At theta = 1e-7 no cell can pass the opening test (theta^2 d^2 < 1 for
    every grid distance d < 2^21 sqrt 3), so the walk is the direct sum."""
    p32, m32 = _inputs("hernquist", 3000)
    ctx = _ctx(rvmod, 3000, theta=1e-7, eps_star=0.005)
    gpu_tree(ctx, p32, m32)
    ax, ay, az, pot = ctx.tree_forces()
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    ad, pd = oracle.direct(p32.astype(np.float64), m32.astype(np.float64), float(np.float32(0.005)))
    _, _, mx = err_stats(a, ad)
    assert mx <= 1e-5
    np.testing.assert_allclose(pot.cpu().numpy(), pd, rtol=1e-5)
    assert ctx.walk_stats()[1] == 0


def test_coincident_unsoftened_is_finite(rvmod):
    p32, m32 = _inputs("coincident", 100)
    ctx = _ctx(rvmod, 100, eps_star=0.0)
    gpu_tree(ctx, p32, m32)
    out = ctx.tree_forces()
    ctx.sync_status()
    for t in out:
        assert np.all(np.isfinite(t.cpu().numpy())) and np.all(t.cpu().numpy() == 0)


def test_empty_input(rvmod):
    import torch
    ctx = _ctx(rvmod, 16)
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    ctx.build_tree(e, e, e, e)
    out = ctx.tree_forces()
    ctx.sync_status()
    assert all(t.numel() == 0 for t in out)


def test_forces_before_build_rejected(rvmod):
    ctx = _ctx(rvmod, 16)
    with pytest.raises(rvmod.RvError) as ei:
        ctx.tree_forces()
    assert ei.value.status == rvmod.RV_E_NOTBUILT


def test_deterministic(rvmod):
    p32, m32 = _inputs("hernquist", 65659)
    ctx = _ctx(rvmod, 65659)
    gpu_tree(ctx, p32, m32)
    a1 = [t.cpu().numpy().copy() for t in ctx.tree_forces()]
    gpu_tree(ctx, p32, m32)
    a2 = [t.cpu().numpy().copy() for t in ctx.tree_forces()]
    for u, w in zip(a1, a2):
        np.testing.assert_array_equal(u, w)


def test_every_star_written_in_every_queue_order(rvmod):
    """The walk takes its groups in an order estimated from costs: box volume
    on the first walk of a context or after the star count changed, the
    recorded list costs on later walks, build order below 2^17 stars. Every
    star is written under each order, and the results do not depend on it."""
    import torch
    n = 1 << 18
    p32, m32 = hernquist32(n, 31)
    ctx = rvmod.Context(n, theta=0.5, eps_star=0.005, n_leaf=32, group=64, tile=128)

    def walk(k):
        gpu_tree(ctx, p32[:, :k].copy(), m32[:k].copy())
        out = [torch.full((k,), float("nan"), dtype=torch.float32, device="cuda") for _ in range(4)]
        ctx.tree_forces(out=out)
        ctx.sync_status()
        a = np.stack([o.cpu().numpy() for o in out])
        assert np.all(np.isfinite(a)), k
        return a

    runs = [walk(n) for _ in range(3)]        # volume order, then recorded costs twice
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[1], runs[2])
    k = n - 1000                                # another star count: volume order again
    a1, a2 = walk(k), walk(k)
    assert np.array_equal(a1, a2)
    walk(5000)                                  # build order


def test_extra_particle_vs_oracle(rvmod):
    """An unsoftened centre-of-mass particle outside the tree (Sect. 2/3)."""
    p32, m32 = _inputs("hernquist", 65659)
    xp = np.array([[0.05], [-0.02], [0.01]], dtype=np.float32)
    xm = np.array([0.01])
    ctx = _ctx(rvmod, 65659, eps_star=0.005)
    gpu_tree(ctx, p32, m32)
    xyzm = to_dev(np.array([[xp[0, 0], xp[1, 0], xp[2, 0], xm[0]]], dtype=np.float32))
    xeps = to_dev(np.zeros(1, np.float32))
    ax, ay, az, pot, xo = ctx.tree_forces(extra_xyzm=xyzm, extra_eps=xeps)
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    T = oracle.Tree(p32, m32, 16, 32)
    ao, po, xa, xpot = T.forces(0.5, float(np.float32(0.005)), True, xp, np.float32(xm).astype(np.float64), [0.0])
    med, _, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL
    xo = xo.cpu().numpy().astype(np.float64)
    assert oracle.rel_err(xo[:, :3].T, xa).max() <= MAX_TOL
    assert abs(xo[0, 3] / xpot[0] - 1) <= MAX_TOL


def test_perturber_forces_vs_oracle(rvmod):
    import torch
    b = ics.central_binary()
    g = ics.rng(31)
    px = g.normal(0, 0.01, (256, 3))
    pm = np.full(256, 1.0 / (1 << 20))
    ctx = _ctx(rvmod, 16)
    d = ctx.perturber_forces(to_dev(b.mass), to_dev(b.pos), to_dev(pm), to_dev(px))
    torch.cuda.synchronize()
    o = oracle.perturber(b.mass, b.pos, pm, px)
    np.testing.assert_allclose(d["a_pert"].cpu().numpy(), o["a_pert"], rtol=1e-11, atol=1e-11 * np.abs(o["a_pert"]).max())
    np.testing.assert_allclose(d["pot_pert"].cpu().numpy(), o["pot_pert"], rtol=1e-11, atol=1e-11 * np.abs(o["pot_pert"]).max())
    np.testing.assert_allclose(d["a_chain"].cpu().numpy(), o["a_chain"], rtol=1e-12)
    np.testing.assert_allclose(d["pot_chain"].cpu().numpy(), o["pot_chain"], rtol=1e-12)
    out8 = d["out8"].cpu().numpy()
    np.testing.assert_allclose(out8[0:3], o["corr"], rtol=1e-12)
    np.testing.assert_allclose(out8[3:6], o["sub"], rtol=1e-12)
    np.testing.assert_allclose(out8[6:8], [o["corr_pot"], o["sub_pot"]], rtol=1e-12)
    np.testing.assert_allclose(out8[8:12], [*o["com"], o["M"]], rtol=1e-15, atol=1e-18)


@pytest.mark.parametrize("mode", [1, 2])
def test_perturber_selection_exact(rvmod, mode):
    p32, m32 = _inputs("hernquist", 65659)
    c = np.array([0.01, -0.005, 0.002], dtype=np.float32)
    ctx = _ctx(rvmod, 65659)
    x, y, z = (to_dev(p32[a]) for a in range(3))
    if mode == 1:
        r = np.float32(0.05)
        idx, cnt = ctx.select_perturbers(x, y, z, c, 1, radius=r)
        ref = oracle.radius(p32, c, np.float32(r * r))
    else:
        idx, cnt = ctx.select_perturbers(x, y, z, c, 2, k=256)
        ref = oracle.knn(p32, c, 256)
    ctx.sync_status()
    k = int(cnt.item())
    assert k == len(ref) and k > 0
    np.testing.assert_array_equal(idx[:k].cpu().numpy(), ref)


def _system(rvmod, w, ctx_n, **kw):
    ch = w.chain
    kwargs = {}
    if ch is not None:
        kwargs = dict(chain_m=ch.mass, chain_x=ch.pos, chain_v=ch.vel)
    return rvmod.System(w.stars.pos, w.stars.vel, w.stars.mass, **kwargs, **kw)


def _oracle_system_forces(w, p32, m32, theta, eps, sub=None, pert=None, n_leaf=16, G=32, quad=True):
    """Oracle forces of a star + chain system, following the same steps:
    tree over stars with the chain centre of mass as an unsoftened extra
    particle (plus the chain's quadrupole when it has several members and
    quad is set, as rv_system.chain_quad = 1 does), then the resolved-chain
    corrections of the perturbers (Sect. 2)."""
    ch = w.chain
    T = oracle.Tree(p32, m32, n_leaf, G)
    com = ch.com
    M = ch.total_mass
    xp = com.astype(np.float32).reshape(3, 1)
    xm = np.array([np.float32(M)], dtype=np.float64)
    quad = quad and len(ch.mass) > 1
    xq = [oracle.chain_moments(ch.mass, ch.pos)["Q"]] if quad else None
    ao, po, xa, xpot = T.forces(theta, eps, True, xp, xm, [0.0], targets=sub, extra_quad=xq,
                                quad_skip=pert if quad else None)
    o = oracle.perturber(ch.mass, ch.pos, m32[pert].astype(np.float64), p32[:, pert].T.astype(np.float64))
    return ao, po, xa, xpot, o


def test_system_forces_hernquist_bh(rvmod):
    """Stars + one SMBH (a chain of one member), perturbers within r = 0.02."""
    import torch
    w = ics.hernquist_bh_workload(1 << 16, seed=12)
    w.chain.pos[0] = [0.02, 0.0, 0.0]                       # put it in the dense core: several perturbers
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(w.eps_star))
    ctx = _ctx(rvmod, p32.shape[1], theta=0.5, eps_star=eps)
    S = _system(rvmod, w, p32.shape[1], pert_mode=1, pert_radius=0.02)
    ctx.system_forces(S)
    ctx.sync_status()
    com32 = w.chain.com.astype(np.float32)
    pert = oracle.radius(p32, com32, np.float32(np.float32(0.02) * np.float32(0.02)))
    assert len(pert) > 3
    ao, po, xa, xpot, o = _oracle_system_forces(w, p32, m32, 0.5, eps, pert=pert)
    ao[:, pert] += o["a_pert"].T
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    med, _, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL
    # chain member: tree force on the CoM - perturbers' direct terms + per-member perturber pull
    a_bh = xa[:, 0] - o["sub"] + o["a_chain"][0]
    got = S.chain_a.cpu().numpy()[:3]
    assert np.linalg.norm(got - a_bh) / np.linalg.norm(a_bh) <= MAX_TOL
    # vs the FP64 direct sum over everything (stars softened, SMBH pairs unsoftened)
    allp = np.concatenate([p32.astype(np.float64), w.chain.pos.T], 1)
    allm = np.concatenate([m32.astype(np.float64), w.chain.mass])
    epsv = np.concatenate([np.full(p32.shape[1], eps), [0.0]])
    tg = ics.subsample(p32.shape[1], 2048, seed=5)
    ad, _ = oracle.direct(allp, allm, epsv, targets=tg)
    _, p99, _ = err_stats(a[:, tg], ad)
    assert p99 <= P99_DIRECT


def test_energy_reduction_vs_oracle(rvmod):
    import torch
    w = ics.hernquist_binary_workload(1 << 14, seed=8)
    ctx = _ctx(rvmod, w.stars.n, eps_star=0.005)
    S = _system(rvmod, w, w.stars.n, pert_mode=2, pert_k=64)
    ctx.system_forces(S)
    E = ctx.energy(S).cpu().numpy()
    ctx.sync_status()
    pos = np.concatenate([np.stack([t.cpu().numpy() for t in (S.x, S.y, S.z)]).astype(np.float64),
                          S.chain_x.cpu().numpy().reshape(-1, 3).T], 1)
    vel = np.concatenate([np.stack([t.cpu().numpy() for t in (S.vx, S.vy, S.vz)]).astype(np.float64),
                          S.chain_v.cpu().numpy().reshape(-1, 3).T], 1)
    m = np.concatenate([S.m.cpu().numpy().astype(np.float64), S.chain_m.cpu().numpy()])
    pot = np.concatenate([S.pot.cpu().numpy().astype(np.float64), S.chain_pot.cpu().numpy()])
    ref = oracle.energy(pos, vel, m, pot)
    np.testing.assert_allclose(E[0], ref["ekin"], rtol=1e-12)
    np.testing.assert_allclose(E[1], ref["epot"], rtol=1e-12)
    np.testing.assert_allclose(E[3:6], ref["P"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(E[6:9], ref["L"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(E[9], m.sum(), rtol=1e-12)


@pytest.mark.slow
def test_kdk_plummer_100_steps(rvmod):
    """Plummer N=4096, eps=0.01, theta=0.5, 100 KDK steps of 1e-3: GPU and
    oracle (FP64 tree forces) both conserve energy to 1e-5 and their final
    positions agree to 1e-4 relative."""
    import torch
    w = ics.plummer_workload()
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(0.01))
    ctx = _ctx(rvmod, 4096, theta=0.5, eps_star=eps)
    S = rvmod.System(p32, w.stars.vel.astype(np.float32), m32)
    ctx.system_forces(S)
    E0 = ctx.energy(S).cpu().numpy()[2]
    ctx.kdk_step(S, 1e-3, 100)
    E1 = ctx.energy(S).cpu().numpy()[2]
    ctx.sync_status()
    assert abs(E1 / E0 - 1) <= 1e-5

    def f(x):
        x32 = x.astype(np.float32)
        return oracle.Tree(x32, m32, 16, 32).forces(0.5, eps)[0]

    x0 = p32.astype(np.float64)
    v0 = w.stars.vel.astype(np.float32).astype(np.float64)
    xo, vo, _ = oracle.kdk(x0, v0, f(x0), 1e-3, f, 100)
    xg = np.stack([t.cpu().numpy() for t in (S.x, S.y, S.z)]).astype(np.float64)
    rel = np.linalg.norm(xg - xo, axis=0) / np.linalg.norm(xo, axis=0)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-4


@pytest.mark.slow
@pytest.mark.parametrize("G,n_leaf,tile", [(32, 16, 64), (64, 32, 128), (64, 16, 128), (64, 24, 128)])
def test_full_size_hernquist_bh_sampled(rvmod, G, n_leaf, tile):
    """The 2^20-star Hernquist + SMBH workload in the launch configurations the
    benchmark's autotuner picks from: sampled stars against the oracle tree
    (same theta and groups) and the FP64 direct sum over all 2^20 + 1 bodies."""
    w = ics.hernquist_bh_workload(1 << 20, seed=2)
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(w.eps_star))
    ctx = _ctx(rvmod, p32.shape[1], theta=0.5, eps_star=eps, group=G, n_leaf=n_leaf, tile=tile)
    S = _system(rvmod, w, p32.shape[1], pert_mode=1, pert_radius=0.02)
    ctx.system_forces(S)
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    tg = ics.subsample(p32.shape[1], 512, seed=9)
    com32 = w.chain.com.astype(np.float32)
    pert = oracle.radius(p32, com32, np.float32(np.float32(0.02) * np.float32(0.02)))
    ao, _, _, _, o = _oracle_system_forces(w, p32, m32, 0.5, eps, sub=tg, pert=pert, n_leaf=n_leaf, G=G)
    ao[:, pert] += o["a_pert"].T
    med, _, mx = err_stats(a[:, tg], ao[:, tg])
    assert med <= MED_TOL and mx <= MAX_TOL
    allp = np.concatenate([p32.astype(np.float64), w.chain.pos.T], 1)
    allm = np.concatenate([m32.astype(np.float64), w.chain.mass])
    epsv = np.concatenate([np.full(p32.shape[1], eps), [0.0]])
    ad, _ = oracle.direct(allp, allm, epsv, targets=tg)
    _, p99, _ = err_stats(a[:, tg], ad)
    assert p99 <= P99_DIRECT


@pytest.mark.slow
def test_energy_conserved_over_1000_steps(rvmod):
    """The 2^20-star Hernquist galaxy (the benchmark's stars, without the SMBH)
    through 1000 KDK steps of 1e-3, replayed from the captured step: the total
    energy drifts by less than 1e-5 (measured: 1.5e-6 at most)."""
    import torch
    w = ics.hernquist_bh_workload(1 << 20, seed=2)
    eps = float(np.float32(0.005))
    ctx = _ctx(rvmod, 1 << 20, theta=0.5, eps_star=eps, n_leaf=24, group=64, tile=128)
    S = rvmod.System(w.stars.pos, w.stars.vel, w.stars.mass)
    stream = torch.cuda.Stream()
    e = torch.zeros(10, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        ctx.system_forces(S, stream=stream)
        ctx.energy(S, out=e, stream=stream)
    torch.cuda.synchronize()
    E0 = e[2].item()
    drift = []
    for _ in range(10):
        with torch.cuda.stream(stream):
            ctx.kdk_step_graph(S, 1e-3, 100, energy_out=e, stream=stream)
        torch.cuda.synchronize()
        drift.append(abs(e[2].item() / E0 - 1))
    ctx.sync_status(stream=stream)
    assert max(drift) <= 1e-5, drift


@pytest.mark.slow
def test_full_size_hernquist_binary_sampled(rvmod):
    """The 2^22-star Hernquist + SMBH-binary workload in the benchmark's launch
    configuration (group 64, n_leaf 24, tile 128; the 256 nearest stars as
    perturbers): sampled stars, some of them perturbers, against the oracle
    running the same method (tree with the binary's centre of mass as one
    unsoftened particle, resolved corrections on the perturbers, Eq. 3)."""
    w = ics.hernquist_binary_workload(1 << 22, seed=3)
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(w.eps_star))
    n = p32.shape[1]
    ctx = _ctx(rvmod, n, theta=0.5, eps_star=eps, group=64, n_leaf=24, tile=128)
    S = _system(rvmod, w, n, pert_mode=2, pert_k=256)
    ctx.system_forces(S)
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    pert = oracle.knn(p32, w.chain.com.astype(np.float32), 256)
    tg = np.union1d(ics.subsample(n, 512, seed=21), pert[::8])
    ao, _, _, _, o = _oracle_system_forces(w, p32, m32, 0.5, eps, sub=tg, pert=pert, n_leaf=24, G=64)
    ao[:, pert] += o["a_pert"].T
    med, _, mx = err_stats(a[:, tg], ao[:, tg])
    assert med <= MED_TOL and mx <= MAX_TOL, (med, mx)


@pytest.mark.slow
@pytest.mark.parametrize("chain_quad", [True, False])
def test_hernquist_binary_p99_vs_resolved_direct(rvmod, chain_quad):
    """The 2^22-star Hernquist + SMBH-pair workload against the fully resolved
    FP64 direct sum (every star softened, both SMBHs unsoftened, no chain
    model): with the chain's quadrupole acting beyond the 256 nearest
    perturbers the sampled p99 meets 1e-3 (and the stars within r < 0.15,
    where the pair's quadrupole matters, are oversampled and still meet it at
    the 90th percentile); with the centre of mass alone the stars near the pair
    miss it. Sample: 2048 random stars plus 512 of those inside r < 0.15."""
    w = ics.hernquist_binary_workload(1 << 22, seed=3)
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(w.eps_star))
    n = p32.shape[1]
    ctx = _ctx(rvmod, n, theta=0.5, eps_star=eps, group=64, n_leaf=24, tile=128)
    S = _system(rvmod, w, n, pert_mode=2, pert_k=256, chain_quad=chain_quad)
    ctx.system_forces(S)
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    r = np.linalg.norm(p32.astype(np.float64), axis=0)
    inner = np.flatnonzero(r < 0.15)
    g = ics.rng(41)
    tg_in = np.sort(g.choice(inner, 512, replace=False))
    tg = ics.subsample(n, 2048, seed=40)
    allp = np.concatenate([p32.astype(np.float64), w.chain.pos.T], 1)
    allm = np.concatenate([m32.astype(np.float64), w.chain.mass])
    epsv = np.concatenate([np.full(n, eps), [0.0, 0.0]])
    ad, _ = oracle.direct(allp, allm, epsv, targets=np.concatenate([tg, tg_in]))
    e = np.linalg.norm(a[:, np.concatenate([tg, tg_in])] - ad, axis=0) / np.linalg.norm(ad, axis=0)
    p99 = oracle.percentile(e[:len(tg)], 0.99)
    p90_inner = oracle.percentile(e[len(tg):], 0.90)
    if chain_quad:
        assert p99 <= 1e-3 and p90_inner <= 1e-3, (p99, p90_inner)
    else:
        assert p90_inner > 1e-3, p90_inner


@pytest.mark.slow
def test_full_size_ensemble_sampled(rvmod):
    """The 64-member ensemble (7.67 M stars of log-uniform member sizes, a
    central SMBH pair each) in one system, benchmark configuration: for the
    smallest, a middle and the largest member, sampled stars against the
    oracle running that member alone with the same method."""
    e = ics.ensemble_workload(64, seed=4)
    off = e["offsets"]
    p32, m32 = stars32(e["pos"], e["mass"])
    eps = float(np.float32(0.005))
    n = p32.shape[1]
    ctx = _ctx(rvmod, n, theta=0.5, eps_star=eps, group=64, n_leaf=24, tile=128)
    S = rvmod.System(e["pos"], e["vel"], e["mass"], chain_m=e["chain_m"], chain_x=e["chain_x"],
                     chain_v=e["chain_v"], pert_mode=2, pert_k=256, member_offsets=off)
    ctx.system_forces(S)
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    sizes = np.diff(off)
    for k in (int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))):
        s0, s1 = int(off[k]), int(off[k + 1])
        mw = ics.Workload(name="member", stars=ics.Particles(pos=e["pos"][:, s0:s1], vel=e["vel"][:, s0:s1],
                                                             mass=e["mass"][s0:s1]),
                          chain=ics.Chain(mass=e["chain_m"][2 * k:2 * k + 2], pos=e["chain_x"][2 * k:2 * k + 2],
                                          vel=e["chain_v"][2 * k:2 * k + 2]), eps_star=0.005, theta=0.5)
        mp, mm = p32[:, s0:s1], m32[s0:s1]
        pert = oracle.knn(mp, mw.chain.com.astype(np.float32), 256)
        tg = np.union1d(ics.subsample(s1 - s0, 128, seed=30 + k), pert[::16])
        ao, _, _, _, o = _oracle_system_forces(mw, mp, mm, 0.5, eps, sub=tg, pert=pert, n_leaf=24, G=64)
        ao[:, pert] += o["a_pert"].T
        med, _, mx = err_stats(a[:, s0 + tg], ao[:, tg])
        assert med <= MED_TOL and mx <= MAX_TOL, (k, med, mx)


def test_walk_stack_stays_within_its_bound(rvmod):
    """The worst case for the walk's range stack: every cell opened (theta ->
    0) in a tree of one star per leaf. The depth-first traversal, 64 cells a
    pass, keeps at most 64 pending ranges per level, so the deepest stack stays
    at or below 21 x 64 = 1344 of its 1408 entries (those beyond the first 256
    in the warp's spill area), and the walk completes (the direct sum)."""
    n = 1 << 17
    p32, m32 = _inputs("hernquist", n)
    ctx = _ctx(rvmod, n, theta=0.5, eps_star=0.005, n_leaf=1, group=64, tile=128)
    gpu_tree(ctx, p32, m32)
    a = [t.cpu().numpy() for t in ctx.tree_forces(theta=1e-7)]
    ctx.sync_status()
    p2p, m2p, hwm = ctx.walk_stats3()
    assert m2p == 0 and p2p == n * n
    assert 0 < hwm <= 21 * 64
    assert all(np.all(np.isfinite(u)) for u in a)


def test_radius_overflow_reported(rvmod):
    """More stars inside the radius than the output holds: the first `cap`
    ascending indices are written and rv_sync_status reports RV_E_WORKSPACE."""
    p32, m32 = _inputs("hernquist", 20000)
    ctx = _ctx(rvmod, 20000)
    x, y, z = (to_dev(p32[a]) for a in range(3))
    idx, cnt = ctx.select_perturbers(x, y, z, (0.0, 0.0, 0.0), 1, radius=1.0, cap=100)
    with pytest.raises(rvmod.RvError) as ei:
        ctx.sync_status()
    assert ei.value.status == rvmod.RV_E_WORKSPACE
    ref = oracle.radius(p32, np.zeros(3, np.float32), np.float32(1.0))
    assert int(cnt.item()) == 100
    np.testing.assert_array_equal(idx[:100].cpu().numpy(), ref[:100])
    ctx.sync_status()                      # the latched error was cleared


def test_pair_record_overflow_reported(rvmod):
    p32, m32 = _inputs("hernquist", 20000)
    eps = float(np.float32(0.005))
    ctx = _ctx(rvmod, 20000, theta=0.9, eps_star=eps)
    gpu_tree(ctx, p32, m32)
    mlp = rvmod.Mlp(seed=1)
    rvmod.tree_forces_mlp(ctx, mlp, 0.9, 0.5, eps, pair_cap=16)
    with pytest.raises(rvmod.RvError) as ei:
        ctx.sync_status()
    assert ei.value.status == rvmod.RV_E_WORKSPACE


def test_tidal_selection_matches_oracle(rvmod):
    """Eq. 2 on the GPU and in the oracle: the same FP64 decision without a
    cube root, so the index sets are identical; unequal masses (heavier stars
    reach farther) and a tiny cap (truncation reported)."""
    g = ics.rng(43)
    n = 200000
    p32, _ = hernquist32(n, 44)
    m32 = (g.uniform(0.5, 8.0, n) / n).astype(np.float32)
    centre = np.array([0.01, -0.02, 0.0], np.float32)
    ctx = _ctx(rvmod, n)
    x, y, z = (to_dev(p32[a]) for a in range(3))
    m = to_dev(m32)
    for gam, rc in ((1e-3, 0.05), (1e-2, 0.2)):
        idx, cnt = ctx.select_perturbers_tidal(x, y, z, m, centre, 0.01, gam, rc, cap=20000)
        ctx.sync_status()
        ref = oracle.tidal(p32, m32, centre, np.float32(0.01), np.float32(gam), np.float32(rc))
        assert len(ref) > 20
        k = int(cnt.item())
        np.testing.assert_array_equal(idx[:k].cpu().numpy(), ref)
    idx, cnt = ctx.select_perturbers_tidal(x, y, z, m, centre, 0.01, 1e-2, 0.2, cap=10)
    with pytest.raises(rvmod.RvError):
        ctx.sync_status()
    np.testing.assert_array_equal(idx[:10].cpu().numpy(), ref[:10])
    ctx.sync_status()


def test_system_forces_with_tidal_perturbers(rvmod):
    """pert_mode 3 in the full force pass: the perturbers are the Eq. 2 set and
    the forces match the oracle following the same steps."""
    w = ics.hernquist_bh_workload(1 << 16, seed=12)
    w.chain.pos[0] = [0.02, 0.0, 0.0]
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(w.eps_star))
    ctx = _ctx(rvmod, p32.shape[1], theta=0.5, eps_star=eps)
    S = _system(rvmod, w, p32.shape[1], pert_mode=3, pert_radius=0.03, pert_gamma=1e-4)
    ctx.system_forces(S)
    ctx.sync_status()
    com32 = w.chain.com.astype(np.float32)
    pert = oracle.tidal(p32, m32, com32, np.float32(w.chain.total_mass), np.float32(1e-4), np.float32(0.03))
    assert len(pert) > 3
    ao, po, xa, xpot, o = _oracle_system_forces(w, p32, m32, 0.5, eps, pert=pert)
    ao[:, pert] += o["a_pert"].T
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    med, _, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL
    a_bh = xa[:, 0] - o["sub"] + o["a_chain"][0]
    got = S.chain_a.cpu().numpy()[:3]
    assert np.linalg.norm(got - a_bh) / np.linalg.norm(a_bh) <= MAX_TOL


def test_chain_perturber_forces_predicted(rvmod):
    """The chain integrator's perturber pull: the last force pass's perturbers
    predicted to first order, x + v dt, acting on chain members at positions
    the caller gives, against the oracle's FP64 perturber sum on the same
    predicted positions (only the summation order differs)."""
    import torch
    w = ics.hernquist_binary_workload(1 << 16, seed=13)
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    v32 = np.ascontiguousarray(w.stars.vel, dtype=np.float32)
    eps = float(np.float32(w.eps_star))
    ctx = _ctx(rvmod, p32.shape[1], theta=0.5, eps_star=eps)
    S = _system(rvmod, w, p32.shape[1], pert_mode=2, pert_k=256)
    with pytest.raises(rvmod.RvError):                      # no force pass yet: no perturber set
        ctx.chain_perturber_forces(S, 0.0, S.chain_x)
    ctx.system_forces(S)
    ctx.sync_status()
    com32 = w.chain.com.astype(np.float32)
    pert = oracle.knn(p32, com32, 256)
    for dt in (0.0, 3e-4, -2e-4):
        cx = w.chain.pos + np.array([[1e-4, -2e-4, 5e-5], [-1e-4, 2e-4, -5e-5]]) * (dt * 1e3)
        a, pot = ctx.chain_perturber_forces(S, dt, torch.from_numpy(cx.reshape(-1)).cuda())
        xp = p32[:, pert].astype(np.float64) + v32[:, pert].astype(np.float64) * dt
        o = oracle.perturber(w.chain.mass, cx, m32[pert].astype(np.float64), xp.T)
        got = a.cpu().numpy().reshape(-1, 3)
        assert np.abs(got - o["a_chain"]).max() <= 1e-12 * np.abs(o["a_chain"]).max()
        np.testing.assert_allclose(pot.cpu().numpy(), o["pot_chain"], rtol=1e-12)


@pytest.mark.parametrize("kind,n,theta,n_leaf,G,tile,quad,rel", [("plummer", 4096, 0.5, 16, 32, 64, True, False),
                                                                  ("hernquist", 65536, 0.5, 16, 64, 128, True, False),
                                                                  ("two_clusters", 3000, 0.6, 8, 47, 32, False, False),
                                                                  ("hernquist", 65536, 1e-3, 32, 64, 128, True, True)])
def test_spline_softening_vs_oracle(rvmod, kind, n, theta, n_leaf, G, tile, quad, rel):
    """Spline softening (h = 2.8 eps) on the GPU against the oracle tree with the
    same softening (same opening decisions: identical interaction counts), and
    against the spline direct sum."""
    p32, m32 = _inputs(kind, n)
    eps = float(np.float32(0.005 if kind != "plummer" else 0.01))
    ctx = _ctx(rvmod, n, theta=theta if not rel else 0.5, eps_star=eps, n_leaf=n_leaf, group=G, tile=tile,
               quadrupole=quad, softening=1)
    gpu_tree(ctx, p32, m32)
    ad, pd = oracle.direct(p32.astype(np.float64), m32.astype(np.float64), eps, kind=1)
    T = oracle.Tree(p32, m32, n_leaf, G)
    if rel:
        aref = ad.astype(np.float32)
        ax, ay, az, pot = ctx.tree_forces_rel(theta, tuple(to_dev(np.ascontiguousarray(aref[k])) for k in range(3)))
        ao, po, _, _, cnt = T.forces(0.5, eps, quad, counts=True, rel=(theta, aref), kind=1)
    else:
        ax, ay, az, pot = ctx.tree_forces(theta=theta, eps_star=eps)
        ao, po, _, _, cnt = T.forces(theta, eps, quad, counts=True, kind=1)
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    p = pot.cpu().numpy().astype(np.float64)
    med, p99, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL, (med, p99, mx)
    ep = np.abs(p - po) / np.abs(po)
    assert np.median(ep) <= MED_TOL and ep.max() <= MAX_TOL
    n_p2p, n_m2p = ctx.walk_stats()
    assert n_p2p == int(cnt[:, 0].sum()) + n and n_m2p == int(cnt[:, 1].sum())
    if quad:
        assert err_stats(a, ad)[1] <= P99_DIRECT


def test_chain_start_radius_matches_oracle(rvmod):
    """Eq. 1 on the GPU and in the oracle: the same distance order (FP32 d2,
    ties by index) and the same FP64 sums in that order, so r(<2 M_bh), sigma
    and the derived radii agree to the last bit; and around an off-centre
    SMBH of a Hernquist galaxy r_infl is the smaller of the two proxies."""
    w = ics.hernquist_bh_workload(1 << 16, seed=14)
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    v32 = np.ascontiguousarray(w.stars.vel, dtype=np.float32)
    ctx = _ctx(rvmod, p32.shape[1])
    pos = tuple(to_dev(p32[a]) for a in range(3))
    vel = tuple(to_dev(v32[a]) for a in range(3))
    for centre in (np.zeros(3, np.float32), w.chain.pos[0].astype(np.float32)):
        got = ctx.chain_start_radius(pos, vel, to_dev(m32), centre, 0.005, 1.2, 1.5, 0.005)
        ref = oracle.chain_start_radius(p32, v32, m32, centre, 0.005, 1.2, 1.5, 0.005)
        for k in ("r2m", "sigma", "r_sigma", "r_infl", "r_chain0"):
            assert got[k] == ref[k], (k, got[k], ref[k])
        assert got["r_infl"] == min(got["r2m"], got["r_sigma"]) and np.isfinite(got["r2m"])


def test_system_forces_two_chains(rvmod):
    """Two SMBHs far apart in one galaxy, each its own chain with its own
    perturbers (several distant SMBHs: the paper's outlook, Sect. 7): both
    centres of mass are unsoftened particles of the tree, each chain's
    perturbers get its resolved-minus-centre correction, each chain member
    feels the tree (with the other chain as a point mass) and its perturbers.
    Against the oracle following the same steps."""
    w = ics.hernquist_bh_workload(1 << 16, seed=15)
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    eps = float(np.float32(w.eps_star))
    cm = np.array([0.005, 0.003])
    cx = np.array([[0.02, 0.0, 0.0], [-0.3, 0.1, 0.0]])
    cv = np.array([[0.0, 0.4, 0.0], [0.0, -0.3, 0.1]])
    ctx = _ctx(rvmod, p32.shape[1], theta=0.5, eps_star=eps)
    S = rvmod.System(w.stars.pos, w.stars.vel, w.stars.mass, chain_m=cm, chain_x=cx, chain_v=cv, pert_mode=1,
                     pert_radius=0.06, chains_per_member=2)
    assert S.n_chain == 1
    ctx.system_forces(S)
    ctx.sync_status()
    T = oracle.Tree(p32, m32, 16, 32)
    xp = cx.astype(np.float32).T
    xm = np.array([np.float32(v) for v in cm], dtype=np.float64)
    ao, _, xa, _ = T.forces(0.5, eps, True, xp, xm, [0.0, 0.0])
    a_bh = []
    for j in range(2):
        pert = oracle.radius(p32, cx[j].astype(np.float32), np.float32(np.float32(0.06) * np.float32(0.06)))
        assert len(pert) > 3
        o = oracle.perturber(cm[j:j + 1], cx[j:j + 1], m32[pert].astype(np.float64), p32[:, pert].T.astype(np.float64))
        ao[:, pert] += o["a_pert"].T
        a_bh.append(xa[:, j] - o["sub"] + o["a_chain"][0])
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    med, _, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL, (med, mx)
    got = S.chain_a.cpu().numpy().reshape(2, 3)
    for j in range(2):
        assert np.linalg.norm(got[j] - a_bh[j]) / np.linalg.norm(a_bh[j]) <= MAX_TOL
    # a step runs with both chains and the energy totals include both members
    ctx.kdk_step(S, 1e-3, 2)
    e = ctx.energy(S).cpu().numpy()
    ctx.sync_status()
    assert abs(e[9] - (m32.astype(np.float64).sum() + cm.sum())) < 1e-6


def test_new_paths_on_empty_and_tiny_inputs(rvmod):
    """Degenerate inputs on the relative criterion, tidal search, block steps
    and chain start radius: no stars, one star, all stars at one point."""
    import torch
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    ctx = _ctx(rvmod, 16)
    ctx.build_tree(e, e, e, e)
    ctx.tree_forces_rel(1e-3, (e, e, e), out=(e, e, e, e))
    idx, cnt = ctx.select_perturbers_tidal(e, e, e, e, (0, 0, 0), 0.01, 1e-3, 0.1)
    ctx.sync_status()
    assert int(cnt.item()) == 0
    with pytest.raises(rvmod.RvError):
        ctx.chain_start_radius((e, e, e), (e, e, e), e, (0, 0, 0), 0.005, 1, 1, 0.01)
    S0 = rvmod.System(np.zeros((3, 0)), np.zeros((3, 0)), np.zeros(0))
    B0 = rvmod.Blocks(0, 1e-2, 2)
    ctx.block_start(S0, B0)
    ctx.block_steps(S0, B0, 4)
    ctx.sync_status()
    # one star: no force; at one point (softened): finite, zero force, phi = -(n-1) m / eps
    for n in (1, 100):
        p32 = np.full((3, n), 0.25, np.float32)
        m32 = np.full(n, 1.0 / n, np.float32)
        c = _ctx(rvmod, n, eps_star=0.01)
        gpu_tree(c, p32, m32)
        z = tuple(to_dev(np.zeros(n, np.float32)) for _ in range(3))
        ax, ay, az, pot = c.tree_forces_rel(1e-3, z)
        c.sync_status()
        assert np.all(ax.cpu().numpy() == 0) and np.all(np.isfinite(pot.cpu().numpy()))
        np.testing.assert_allclose(pot.cpu().numpy(), -(n - 1) / n / float(np.float32(0.01)), rtol=1e-5)


def test_relmac_mixed_references_vs_oracle(rvmod):
    """References that are zero for some stars: their groups fall back to theta,
    the others use the relative criterion -- the same split on both sides."""
    p32, m32 = _inputs("hernquist", 65536)
    eps = float(np.float32(0.005))
    ad, _ = oracle.direct(p32.astype(np.float64), m32.astype(np.float64), eps)
    aref = ad.astype(np.float32)
    r = np.linalg.norm(p32.astype(np.float64), axis=0)
    aref[:, r > 1.0] = 0.0                             # outer stars: no reference yet
    ctx = _ctx(rvmod, 65536, theta=0.6, eps_star=eps, group=64, n_leaf=32, tile=128)
    gpu_tree(ctx, p32, m32)
    ax, ay, az, _ = ctx.tree_forces_rel(1e-3, tuple(to_dev(np.ascontiguousarray(aref[k])) for k in range(3)))
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    T = oracle.Tree(p32, m32, 32, 64)
    ao, _, cnt = T.forces_rel(1e-3, eps, aref, counts=True, theta=0.6)
    med, _, mx = err_stats(a, ao)
    assert med <= MED_TOL and mx <= MAX_TOL
    n_p2p, n_m2p = ctx.walk_stats()
    assert n_p2p == int(cnt[:, 0].sum()) + 65536 and n_m2p == int(cnt[:, 1].sum())


def test_max_members_tiny(rvmod):
    """512 members (the maximum) of one to three stars each: every member is its
    own tree; each star feels only its own member (closed-form pairs)."""
    g = ics.rng(71)
    sizes = g.integers(1, 4, 512)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    p32 = g.uniform(-1, 1, (3, n)).astype(np.float32)
    m32 = g.uniform(0.5, 1.5, n).astype(np.float32)
    eps = float(np.float32(0.01))
    ctx = _ctx(rvmod, n, eps_star=eps)
    ctx.build_tree_members(off, *(to_dev(p32[a]) for a in range(3)), to_dev(m32))
    ax, ay, az, pot = ctx.tree_forces_members()
    ctx.sync_status()
    a = np.stack([t.cpu().numpy() for t in (ax, ay, az)]).astype(np.float64)
    for k in range(512):
        s, e = int(off[k]), int(off[k + 1])
        ad, pd = oracle.direct(p32[:, s:e].astype(np.float64), m32[s:e].astype(np.float64), eps)
        np.testing.assert_allclose(a[:, s:e], ad, rtol=2e-5, atol=1e-6)
        np.testing.assert_allclose(pot.cpu().numpy()[s:e], pd, rtol=2e-5, atol=1e-6)
