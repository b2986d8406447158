"""Block time steps on the GPU (Sect. 2: a hierarchy of step levels; KDK
form) against the oracle's block integrator, and the level rule against the
oracle's on identical FP32 inputs. Walks are restricted to the groups that
hold an active star."""
import numpy as np
import pytest

import ics
import oracle
from gpu_helpers import stars32, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rvmod():
    from paper_1507_01009_gb300 import rv
    rv.load()
    return rv


def _plummer():
    w = ics.plummer_workload()
    p32, m32 = stars32(w.stars.pos, w.stars.mass)
    v32 = np.ascontiguousarray(w.stars.vel, dtype=np.float32)
    return p32, v32, m32


def _state(S):
    x = np.stack([t.cpu().numpy() for t in (S.x, S.y, S.z)]).astype(np.float64)
    v = np.stack([t.cpu().numpy() for t in (S.vx, S.vy, S.vz)]).astype(np.float64)
    return x, v


def test_block_single_level_is_kdk(rvmod):
    """All stars on level 0 with L = 0: the block scheme is rv_kdk_step,
    operation for operation (positions bit for bit)."""
    p32, v32, m32 = _plummer()
    eps = float(np.float32(0.01))
    c1 = rvmod.Context(4096, theta=0.5, eps_star=eps)
    c2 = rvmod.Context(4096, theta=0.5, eps_star=eps)
    S1 = rvmod.System(p32, v32, m32)
    S2 = rvmod.System(p32, v32, m32)
    c1.system_forces(S1)
    c1.kdk_step(S1, 1e-3, 6)
    B = rvmod.Blocks(4096, 1e-3, 0, adapt=False)
    c2.block_start(S2, B)
    c2.block_steps(S2, B, 6)
    c1.sync_status(); c2.sync_status()
    x1, v1 = _state(S1)
    x2, v2 = _state(S2)
    np.testing.assert_array_equal(x2, x1)
    a1 = np.stack([t.cpu().numpy() for t in (S1.ax, S1.ay, S1.az)]).astype(np.float64)
    np.testing.assert_allclose(v2, v1 + 0.5e-3 * a1, rtol=1e-6, atol=1e-9)   # plus the next opening kick
    assert c2.block_count() == 6 * 4096 and B.substep == 6


def test_block_fixed_levels_vs_oracle(rvmod):
    """Levels by radius (inner stars finer), L = 3, 24 substeps: the GPU block
    integrator against the oracle's (tree forces at theta 0.5 on the FP32
    positions of each substep), and the same number of active updates."""
    p32, v32, m32 = _plummer()
    eps = float(np.float32(0.01))
    r = np.linalg.norm(p32.astype(np.float64), axis=0)
    lv = np.select([r < 0.4, r < 0.8, r < 1.6], [3, 2, 1], 0).astype(np.int8)
    ctx = rvmod.Context(4096, theta=0.5, eps_star=eps)
    S = rvmod.System(p32, v32, m32)
    B = rvmod.Blocks(4096, 8e-3, 3, adapt=False, level=lv)
    ctx.block_start(S, B)
    ctx.block_steps(S, B, 24)
    ctx.sync_status()
    xg, vg = _state(S)

    def f(x, active):
        T = oracle.Tree(x.astype(np.float32), m32, 16, 32)
        return T.forces(0.5, eps, targets=np.nonzero(active)[0])[0]

    xo, vo, _, _, upd = oracle.block_kdk(p32.astype(np.float64), v32.astype(np.float64), f, lv.astype(int), 3, 8e-3,
                                         24)
    rel = np.linalg.norm(xg - xo, axis=0) / np.linalg.norm(xo, axis=0)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-4, (np.median(rel), rel.max())
    relv = np.linalg.norm(vg - vo, axis=0) / np.linalg.norm(vo, axis=0)
    assert np.median(relv) <= 1e-4
    assert ctx.block_count() == upd
    assert upd < 24 * 4096


def test_masked_walk_equals_full_walk_for_active_stars(rvmod):
    """2^18 Hernquist stars (large enough for the cost-ordered walk queue),
    levels by radius, L = 2: after one substep the active stars' new
    accelerations equal, bit for bit, those of a full force pass at the same
    positions (the masked walk skips whole groups and changes no list)."""
    import torch
    n = 1 << 18
    w = ics.hernquist(n, 41)
    p32, m32 = stars32(w.pos, w.mass)
    v32 = np.ascontiguousarray(w.vel, dtype=np.float32)
    eps = float(np.float32(0.005))
    r = np.linalg.norm(p32.astype(np.float64), axis=0)
    lv = np.select([r < 0.3, r < 1.0], [2, 1], 0).astype(np.int8)
    ctx = rvmod.Context(n, theta=0.5, eps_star=eps, n_leaf=24, group=64, tile=128)
    S = rvmod.System(p32, v32, m32)
    B = rvmod.Blocks(n, 4e-3, 2, adapt=False, level=lv)
    ctx.block_start(S, B)
    ctx.block_steps(S, B, 1)                                    # substep 1: level-2 stars active
    ctx.sync_status()
    active = lv == 2
    assert 0 < active.sum() < n and ctx.block_count() == int(active.sum())
    xs = np.stack([t.cpu().numpy() for t in (S.x, S.y, S.z)])
    a_blk = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)])
    full = rvmod.Context(n, theta=0.5, eps_star=eps, n_leaf=24, group=64, tile=128)
    S2 = rvmod.System(xs, v32, m32)
    full.system_forces(S2)
    full.sync_status()
    a_full = np.stack([t.cpu().numpy() for t in (S2.ax, S2.ay, S2.az)])
    np.testing.assert_array_equal(a_blk[:, active], a_full[:, active])


def test_block_levels_match_oracle(rvmod):
    """The level rule on identical FP32 inputs: bit-identical levels, at the
    start and at substeps with and without step boundaries."""
    g = ics.rng(51)
    n = 100000
    a = (10.0 ** g.uniform(-4, 2, n) * g.normal(size=(3, n)) / np.sqrt(3)).astype(np.float32)
    v = (10.0 ** g.uniform(-3, 0.5, n) * g.normal(size=(3, n)) / np.sqrt(3)).astype(np.float32)
    a[:, :10] = 0.0
    v[:, 5:15] = 0.0
    L = 8
    ctx = rvmod.Context(16)
    acc, vel = tuple(to_dev(a[k]) for k in range(3)), tuple(to_dev(v[k]) for k in range(3))
    for sub, start in ((0, True), (96, False), (97, False), (128, False)):
        lv0 = g.integers(0, L + 1, n).astype(np.int8)
        B = rvmod.Blocks(n, 1.0 / 16, L, tau_acc=0.3, tau_vel=0.25, eps=0.005, level=lv0)
        B.substep = sub
        ctx.block_levels(B, acc, vel, start=start)
        ctx.sync_status()
        ref = oracle.block_levels(a, v, lv0, sub, L, 1.0 / 16, 0.3, 0.25, 0.005, start=start)
        np.testing.assert_array_equal(B.level.cpu().numpy(), ref)


def test_block_adaptive_energy_and_work(rvmod):
    """Adaptive levels on the Plummer sphere: the energy at a synchronisation
    point (velocities taken back by the opening half kick) stays within 2e-5
    of the start after 4 dt_max, and the block scheme needs far fewer force
    evaluations than stepping every star at dt_min."""
    p32, v32, m32 = _plummer()
    eps = float(np.float32(0.01))
    ctx = rvmod.Context(4096, theta=0.5, eps_star=eps)
    S = rvmod.System(p32, v32, m32)
    ctx.system_forces(S)
    E0 = ctx.energy(S).cpu().numpy()[2]
    L, dt_max = 4, 1.0 / 32
    B = rvmod.Blocks(4096, dt_max, L, tau_acc=0.3, tau_vel=0.3, eps=eps)
    ctx.block_start(S, B)
    levels0 = B.level.cpu().numpy().copy()
    assert levels0.max() > levels0.min()
    ctx.block_steps(S, B, 4 * 2 ** L)
    ctx.sync_status()
    lv = B.level.cpu().numpy().astype(np.float64)
    x, v = _state(S)
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    vs = v - a * (0.5 * dt_max * 2.0 ** -lv)
    m = m32.astype(np.float64)
    E1 = 0.5 * np.sum(m * (vs * vs).sum(0)) + 0.5 * np.sum(m * S.pot.cpu().numpy().astype(np.float64))
    assert abs(E1 / E0 - 1) <= 2e-5, (E0, E1)
    assert ctx.block_count() < 0.7 * 4096 * 4 * 2 ** L


def test_block_steps_with_smbh(rvmod):
    """A star + SMBH system on block steps (the chain on the finest level):
    runs, stays finite, and the chain moves."""
    import torch
    w = ics.hernquist_bh_workload(1 << 15, seed=12)
    ctx = rvmod.Context(1 << 15, theta=0.5, eps_star=float(np.float32(w.eps_star)))
    S = rvmod.System(w.stars.pos, w.stars.vel, w.stars.mass, chain_m=w.chain.mass, chain_x=w.chain.pos,
                     chain_v=w.chain.vel, pert_mode=1, pert_radius=0.02)
    B = rvmod.Blocks(1 << 15, 1.0 / 64, 3, tau_acc=0.3, tau_vel=0.3, eps=0.005)
    x0 = S.chain_x.clone()
    ctx.block_start(S, B)
    ctx.block_steps(S, B, 16)
    ctx.sync_status()
    assert torch.isfinite(S.ax).all() and torch.isfinite(S.vx).all()
    assert not torch.equal(S.chain_x, x0)
    assert 0 < ctx.block_count() < 16 * (1 << 15)


def test_block_steps_resume_from_saved_state(rvmod):
    """Checkpoint and resume: the block scheme's whole state is the caller's
    (the star arrays, the levels and the substep counter). Stopped in the
    middle of a dt_max, copied to the host, restored into a fresh context and
    continued, it gives bit for bit what the uninterrupted run gives."""
    import torch
    p32, v32, m32 = _plummer()
    eps = float(np.float32(0.01))
    L, dt_max = 4, 1.0 / 32

    def fresh(pos, vel):
        ctx = rvmod.Context(4096, theta=0.5, eps_star=eps)
        S = rvmod.System(pos, vel, m32)
        B = rvmod.Blocks(4096, dt_max, L, tau_acc=0.3, tau_vel=0.3, eps=eps)
        return ctx, S, B

    ctx, S, B = fresh(p32, v32)
    ctx.system_forces(S)
    ctx.block_start(S, B)
    ctx.block_steps(S, B, 2 ** L + 5)            # stop in the middle of the second dt_max
    ctx.sync_status()
    saved = (S.state.cpu().clone(), B.level.cpu().clone(), B.substep)
    ctx.block_steps(S, B, 2 ** L + 7)
    ctx.sync_status()
    want = S.state.cpu().numpy().copy(), B.level.cpu().numpy().copy(), B.substep

    ctx2, S2, B2 = fresh(p32, v32)
    S2.state.copy_(saved[0].cuda())
    B2.level.copy_(saved[1].cuda())
    B2.substep = saved[2]
    ctx2.block_steps(S2, B2, 2 ** L + 7)
    ctx2.sync_status()
    np.testing.assert_array_equal(S2.state.cpu().numpy(), want[0])
    np.testing.assert_array_equal(B2.level.cpu().numpy(), want[1])
    assert B2.substep == want[2]
