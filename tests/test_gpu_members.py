"""Independent members (galaxy realisations) built and walked together.

Every member must give bit for bit what it gives when built and walked alone
(its keys, tree and interaction lists are its own), with empty and one-star
members in the mix; a system of members with a central SMBH pair each must
match the same systems run one by one; the graph-captured step must equal
the plain step."""
import numpy as np
import pytest

import ics
from gpu_helpers import stars32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rvmod():
    from paper_1507_01009_gb300 import rv
    rv.load()
    return rv


def _members(sizes, seed):
    pos, vel, mass = [], [], []
    for k, n in enumerate(sizes):
        if n == 0:
            continue
        w = ics.hernquist(n, seed + k)
        pos.append(w.pos + 3.0 * k)          # members overlap nothing in particular; shift for variety
        vel.append(w.vel)
        mass.append(w.mass)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(pos, 1), np.concatenate(vel, 1), np.concatenate(mass), off


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SIZES = [3000, 0, 1, 20011, 517, 64, 9000]


def test_members_match_single_builds(rvmod):
    import torch
    pos, _, mass, off = _members(SIZES, 40)
    p32, m32 = stars32(pos, mass)
    ctx = rvmod.Context(int(off[-1]), theta=0.5, eps_star=float(np.float32(0.005)))
    x, y, z, m = _dev(p32[0]), _dev(p32[1]), _dev(p32[2]), _dev(m32)
    ctx.build_tree_members(off, x, y, z, m)
    v = ctx.tree_view()
    ens = [t.cpu().numpy() for t in ctx.tree_forces_members()]
    ctx.sync_status()
    keys = v["keys"].cpu().numpy()
    perm = v["perm"].cpu().numpy()
    for k in range(len(SIZES)):
        s, e = int(off[k]), int(off[k + 1])
        if e == s:
            continue
        single = rvmod.Context(e - s, theta=0.5, eps_star=float(np.float32(0.005)))
        single.build_tree(x[s:e].contiguous(), y[s:e].contiguous(), z[s:e].contiguous(), m[s:e].contiguous())
        sv = single.tree_view()
        one = [t.cpu().numpy() for t in single.tree_forces()]
        single.sync_status()
        np.testing.assert_array_equal(keys[s:e], sv["keys"].cpu().numpy())
        np.testing.assert_array_equal(perm[s:e] - s, sv["perm"].cpu().numpy())
        for a, b in zip(ens, one):
            np.testing.assert_array_equal(a[s:e], b)


def test_members_with_chains_match_single_systems(rvmod):
    import torch
    sizes = [4096, 10000, 2500]
    pos, vel, mass, off = _members(sizes, 60)
    b = ics.central_binary()
    M = len(sizes)
    cm = np.tile(b.mass, M)
    cx = np.concatenate([b.pos + 3.0 * k for k in range(M)])
    cv = np.tile(b.vel, (M, 1))
    eps = float(np.float32(0.005))
    ctx = rvmod.Context(int(off[-1]), theta=0.5, eps_star=eps)
    S = rvmod.System(pos, vel, mass, chain_m=cm, chain_x=cx, chain_v=cv, pert_mode=2, pert_k=32,
                     member_offsets=off)
    ctx.system_forces(S)
    E = ctx.energy(S).cpu().numpy().reshape(M, 10)
    ctx.sync_status()
    for k in range(M):
        s, e = int(off[k]), int(off[k + 1])
        one = rvmod.Context(e - s, theta=0.5, eps_star=eps)
        S1 = rvmod.System(pos[:, s:e], vel[:, s:e], mass[s:e], chain_m=b.mass, chain_x=cx[2 * k:2 * k + 2],
                          chain_v=b.vel, pert_mode=2, pert_k=32)
        one.system_forces(S1)
        E1 = one.energy(S1).cpu().numpy()
        one.sync_status()
        for f in ("ax", "ay", "az", "pot"):
            np.testing.assert_array_equal(getattr(S, f)[s:e].cpu().numpy(), getattr(S1, f).cpu().numpy())
        np.testing.assert_array_equal(S.chain_a.cpu().numpy()[6 * k:6 * k + 6], S1.chain_a.cpu().numpy())
        np.testing.assert_allclose(E[k], E1, rtol=1e-13, atol=1e-18)


def test_graph_step_equals_plain_step(rvmod):
    import torch
    sizes = [3000, 7000]
    pos, vel, mass, off = _members(sizes, 80)
    b = ics.central_binary()
    cm = np.tile(b.mass, 2)
    cx = np.concatenate([b.pos, b.pos + 3.0])
    cv = np.tile(b.vel, (2, 1))
    eps = float(np.float32(0.005))
    out = []
    for graph in (False, True):
        ctx = rvmod.Context(int(off[-1]), theta=0.5, eps_star=eps)
        S = rvmod.System(pos, vel, mass, chain_m=cm, chain_x=cx, chain_v=cv, pert_mode=2, pert_k=16,
                         member_offsets=off)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx.system_forces(S, stream=st)
            if graph:
                eo = torch.zeros(20, dtype=torch.float64, device="cuda")
                ctx.kdk_step_graph(S, 1e-3, 5, energy_out=eo, stream=st)
            else:
                ctx.kdk_step(S, 1e-3, 5, stream=st)
                eo = ctx.energy(S, stream=st)
        st.synchronize()
        ctx.sync_status(stream=st)
        out.append([getattr(S, f).cpu().numpy().copy() for f in ("x", "vx", "ax", "pot", "chain_x")] +
                   [eo.cpu().numpy().copy()])
    for a, g in zip(*out):
        np.testing.assert_array_equal(a, g)


@pytest.mark.parametrize("mode", [1, 2])
def test_graph_step_equals_plain_step_one_member(rvmod, mode):
    """A single system with an SMBH (radius or k-nearest perturbers): the
    replayed graph step equals the plain step bit for bit."""
    import torch
    w = ics.hernquist_bh_workload(1 << 14, seed=16)
    eps = float(np.float32(w.eps_star))
    out = []
    for graph in (False, True):
        ctx = rvmod.Context(1 << 14, theta=0.5, eps_star=eps, group=64, n_leaf=32, tile=128)
        S = rvmod.System(w.stars.pos, w.stars.vel, w.stars.mass, chain_m=w.chain.mass, chain_x=w.chain.pos,
                         chain_v=w.chain.vel, pert_mode=mode, pert_radius=0.05, pert_k=64)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx.system_forces(S, stream=st)
            if graph:
                eo = torch.zeros(10, dtype=torch.float64, device="cuda")
                ctx.kdk_step_graph(S, 1e-3, 4, energy_out=eo, stream=st)
            else:
                ctx.kdk_step(S, 1e-3, 4, stream=st)
                eo = ctx.energy(S, stream=st)
        st.synchronize()
        ctx.sync_status(stream=st)
        out.append([getattr(S, f).cpu().numpy().copy() for f in ("x", "vx", "ax", "pot", "chain_x")] +
                   [eo.cpu().numpy().copy()])
    for a, g in zip(*out):
        np.testing.assert_array_equal(a, g)


def test_graph_step_rejects_default_stream(rvmod):
    ctx = rvmod.Context(100)
    w = ics.plummer(100, 3)
    S = rvmod.System(w.pos, w.vel, w.mass)
    import ctypes as C
    st = ctx.L.rv_kdk_step_graph(ctx.h, C.byref(S.c()), 1e-3, 1, None, None)
    assert st == rvmod.RV_E_INVAL


@pytest.mark.parametrize("softening,mac", [(0, 1), (1, 0), (1, 1)])
def test_members_match_single_builds_relmac_and_spline(rvmod, softening, mac):
    """Members under the relative criterion and/or spline softening: each member
    gives bit for bit what it gives alone (references: each star's own |a|
    from a first theta pass of its own member)."""
    pos, _, mass, off = _members(SIZES, 41)
    p32, m32 = stars32(pos, mass)
    eps = float(np.float32(0.005))
    ctx = rvmod.Context(int(off[-1]), theta=0.5, eps_star=eps, softening=softening, group=64, n_leaf=16, tile=128)
    x, y, z, m = _dev(p32[0]), _dev(p32[1]), _dev(p32[2]), _dev(m32)
    ctx.build_tree_members(off, x, y, z, m)
    ref = ctx.tree_forces_members()[:3]
    ens = ctx.tree_forces_rel(1e-3, ref) if mac else ctx.tree_forces_members()
    ens = [t.cpu().numpy() for t in ens[:4]]
    ctx.sync_status()
    for k in range(len(SIZES)):
        s, e = int(off[k]), int(off[k + 1])
        if e == s:
            continue
        single = rvmod.Context(e - s, theta=0.5, eps_star=eps, softening=softening, group=64, n_leaf=16, tile=128)
        single.build_tree(x[s:e].contiguous(), y[s:e].contiguous(), z[s:e].contiguous(), m[s:e].contiguous())
        r1 = single.tree_forces()[:3]
        one = single.tree_forces_rel(1e-3, r1) if mac else single.tree_forces()
        one = [t.cpu().numpy() for t in one[:4]]
        single.sync_status()
        for a, b in zip(ens, one):
            np.testing.assert_array_equal(a[s:e], b)


def test_members_block_steps_match_single_systems(rvmod):
    """Block time steps over members with a chain each: every member evolves
    as it does alone (same levels, positions and velocities bit for bit)."""
    sizes = [4096, 10000]
    pos, vel, mass, off = _members(sizes, 62)
    b = ics.central_binary()
    M = len(sizes)
    cm = np.tile(b.mass, M)
    cx = np.concatenate([b.pos + 3.0 * k for k in range(M)])
    cv = np.tile(b.vel, (M, 1))
    eps = float(np.float32(0.005))
    ctx = rvmod.Context(int(off[-1]), theta=0.5, eps_star=eps)
    S = rvmod.System(pos, vel, mass, chain_m=cm, chain_x=cx, chain_v=cv, pert_mode=2, pert_k=32,
                     member_offsets=off)
    B = rvmod.Blocks(int(off[-1]), 1.0 / 64, 3, tau_acc=0.3, tau_vel=0.3, eps=eps)
    ctx.block_start(S, B)
    ctx.block_steps(S, B, 8)
    ctx.sync_status()
    for k in range(M):
        s, e = int(off[k]), int(off[k + 1])
        one = rvmod.Context(e - s, theta=0.5, eps_star=eps)
        S1 = rvmod.System(pos[:, s:e], vel[:, s:e], mass[s:e], chain_m=b.mass, chain_x=cx[2 * k:2 * k + 2],
                          chain_v=b.vel, pert_mode=2, pert_k=32)
        B1 = rvmod.Blocks(e - s, 1.0 / 64, 3, tau_acc=0.3, tau_vel=0.3, eps=eps)
        one.block_start(S1, B1)
        one.block_steps(S1, B1, 8)
        one.sync_status()
        np.testing.assert_array_equal(B.level[s:e].cpu().numpy(), B1.level.cpu().numpy())
        for f in ("x", "vx", "ax"):
            np.testing.assert_array_equal(getattr(S, f)[s:e].cpu().numpy(), getattr(S1, f).cpu().numpy())
        np.testing.assert_array_equal(S.chain_x.cpu().numpy()[6 * k:6 * k + 6], S1.chain_x.cpu().numpy())


def test_batched_step_beats_members_one_by_one(rvmod):
    """The batched form's claim, measured: 24 members of 8192..131072 stars
    (log-uniform, seeded), each with a central SMBH pair and 256 nearest
    perturbers, stepped together (one context, one captured step) take less
    time per step than the same members stepped one after another (a context
    and a captured step each), at identical forces (the members' bit-for-bit
    equality is tested above)."""
    import torch
    e = ics.ensemble_workload(24, lo=8192, hi=131072, seed=61)
    sizes, off = e["sizes"], e["offsets"]
    pos, vel, mass, cm, cx, cv = e["pos"], e["vel"], e["mass"], e["chain_m"], e["chain_x"], e["chain_v"]
    eps = float(np.float32(0.005))
    kw = dict(theta=0.5, eps_star=eps, n_leaf=24, group=64, tile=96)
    stream = torch.cuda.Stream()

    def timed(pairs, reps=4):
        ev = []
        with torch.cuda.stream(stream):
            for ctx, S, eo in pairs:
                ctx.system_forces(S, stream=stream)
            for r in range(reps + 2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for ctx, S, eo in pairs:
                    ctx.kdk_step_graph(S, 1e-3, 1, energy_out=eo, stream=stream)
                e1.record(stream)
                ev.append((e0, e1))
        torch.cuda.synchronize()
        for ctx, S, eo in pairs:
            ctx.sync_status(stream=stream)
        return float(np.median([a.elapsed_time(b) for a, b in ev[2:]]))

    M = len(sizes)
    batched = [(rvmod.Context(int(off[-1]), **kw),
                rvmod.System(pos, vel, mass, chain_m=cm, chain_x=cx, chain_v=cv, pert_mode=2, pert_k=256,
                             member_offsets=off),
                torch.zeros(10 * M, dtype=torch.float64, device="cuda"))]
    t_batched = timed(batched)
    del batched
    single = []
    for k in range(M):
        a, b = int(off[k]), int(off[k + 1])
        single.append((rvmod.Context(b - a, **kw),
                       rvmod.System(pos[:, a:b], vel[:, a:b], mass[a:b], chain_m=cm[2 * k:2 * k + 2],
                                    chain_x=cx[2 * k:2 * k + 2], chain_v=cv[2 * k:2 * k + 2], pert_mode=2, pert_k=256),
                       torch.zeros(10, dtype=torch.float64, device="cuda")))
    t_single = timed(single)
    print({"stars": int(off[-1]), "batched_ms": t_batched, "one_by_one_ms": t_single})
    assert t_batched < t_single
