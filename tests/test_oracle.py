"""Pins for the CPU oracle: each check ties it to something other than itself
(closed forms, conservation laws, hand-derived fixtures, library routines,
brute force on tiny inputs). A dropped term, a sign or index slip, or a
transposed operand in the oracle fails at least one of these."""
import math
import os

import numpy as np
import pytest

import ics
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# direct sum
# ---------------------------------------------------------------------------
def test_two_body_closed_form():
    """a = m r/(r^2+e^2)^{3/2} toward the other body, phi = -m/(r^2+e^2)^{1/2}."""
    pos = np.array([[0.0, 3.0], [0.0, 4.0], [0.0, 0.0]])  # separation 5
    m = np.array([2.0, 7.0])
    for e in (0.0, 0.5):
        a, p = oracle.direct(pos, m, e)
        d2 = 25.0 + e * e
        f0 = 7.0 / d2 ** 1.5
        np.testing.assert_allclose(a[:, 0], [f0 * 3, f0 * 4, 0.0], rtol=1e-14)
        f1 = 2.0 / d2 ** 1.5
        np.testing.assert_allclose(a[:, 1], [-f1 * 3, -f1 * 4, 0.0], rtol=1e-14)
        np.testing.assert_allclose(p, [-7.0 / math.sqrt(d2), -2.0 / math.sqrt(d2)], rtol=1e-14)


def test_unsoftened_marker_and_max_rule():
    """Pair softening is max(eps_i, eps_j), zero if either particle is marked 0."""
    pos = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 2.0], [0.0, 0.0, 0.0]])
    m = np.array([1.0, 1.0, 1.0])
    eps = np.array([0.1, 0.3, 0.0])
    a, _ = oracle.direct(pos, m, eps, targets=[0])
    expect_x = 1.0 / (1.0 + 0.09) ** 1.5             # pair (0,1): max(0.1, 0.3)
    expect_y = 1.0 * 2.0 / 2.0 ** 3                  # pair (0,2): unsoftened
    np.testing.assert_allclose(a[:, 0], [expect_x, expect_y, 0.0], rtol=1e-14)


def test_direct_momentum_conservation():
    """Newton's third law: sum_i m_i a_i = 0 to rounding."""
    w = ics.plummer(512, seed=11)
    a, _ = oracle.direct(w.pos, w.mass, 0.01)
    tot = (w.mass * a).sum(1)
    scale = (w.mass * np.linalg.norm(a, axis=0)).sum()
    assert np.abs(tot).max() <= 1e-13 * scale


def test_plummer_potential_energy():
    """W = -3 pi / 32 for a Plummer sphere with G = M = b = 1 (sampling noise ~2%)."""
    w = ics.plummer(4096, seed=1)
    _, p = oracle.direct(w.pos, w.mass, 1e-4)
    W = 0.5 * (w.mass * p).sum()
    assert abs(W / (-3 * math.pi / 32) - 1) < 0.05


def _kepler_rel(t, a, e, M):
    """Relative position of a Kepler orbit started at pericentre on +x, moving +y."""
    n = math.sqrt(M / a ** 3)
    Mean = n * t
    E = Mean
    for _ in range(50):
        E -= (E - e * math.sin(E) - Mean) / (1 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _kepler_run(dt, T):
    a, e, M = 1.0, 0.5, 1.0
    m = np.array([0.5, 0.5])
    rp = a * (1 - e)
    vp = math.sqrt(M * (1 + e) / rp)
    pos = np.array([[0.5 * rp, -0.5 * rp], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [0.5 * vp, -0.5 * vp], [0.0, 0.0]])
    f = lambda x: oracle.direct(x, m, 0.0)[0]
    nst = int(round(T / dt))
    pos, vel, _ = oracle.kdk(pos, vel, f(pos), dt, f, nst)
    rel = pos[:, 0] - pos[:, 1]
    en = 0.5 * (m * (vel * vel).sum(0)).sum() - 0.25 / np.linalg.norm(rel)
    return rel, en, _kepler_rel(nst * dt, a, e, M)


def test_kdk_kepler_second_order():
    """KDK on a Kepler orbit: position error vs Kepler's equation shrinks as dt^2,
    and the energy stays at -G m1 m2 / (2a) = -1/8."""
    r1, e1, x1 = _kepler_run(2e-3, 1.3)
    r2, e2, x2 = _kepler_run(1e-3, 1.3)
    err1, err2 = np.linalg.norm(r1 - x1), np.linalg.norm(r2 - x2)
    assert 3.0 < err1 / err2 < 5.0
    assert err2 < 1e-4
    assert abs(e2 + 0.125) < 1e-5


def test_energy_two_body_closed_form():
    pos = np.array([[0.0, 2.0], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [1.0, -0.5], [0.0, 0.0]])
    m = np.array([1.0, 2.0])
    _, p = oracle.direct(pos, m, 0.0)
    E = oracle.energy(pos, vel, m, p)
    assert E["ekin"] == pytest.approx(0.5 * 1 * 1 + 0.5 * 2 * 0.25, rel=1e-15)
    assert E["epot"] == pytest.approx(-1.0 * 2.0 / 2.0, rel=1e-15)
    np.testing.assert_allclose(E["P"], [0.0, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(E["L"], [0.0, 0.0, 2 * 2 * (-0.5)], atol=1e-15)


@pytest.mark.slow
def test_plummer_leapfrog_energy_drift():
    """100 KDK steps, dt = 1e-3, eps = 0.01 on a Plummer sphere: |dE/E| <= 1e-5."""
    w = ics.plummer(1024, seed=5)
    f = lambda x: oracle.direct(x, w.mass, 0.01)[0]
    a0, p0 = oracle.direct(w.pos, w.mass, 0.01)
    E0 = oracle.energy(w.pos, w.vel, w.mass, p0)["etot"]
    pos, vel, _ = oracle.kdk(w.pos, w.vel, a0, 1e-3, f, 100)
    _, p1 = oracle.direct(pos, w.mass, 0.01)
    E1 = oracle.energy(pos, vel, w.mass, p1)["etot"]
    assert abs(E1 / E0 - 1) < 1e-5


# ---------------------------------------------------------------------------
# keys and sort
# ---------------------------------------------------------------------------
def _read_golden_keys():
    pts, kk = [], []
    for line in open(os.path.join(GOLDEN, "morton_keys.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a = line.split()
        pts.append([float(v) for v in a[:3]])
        kk.append(int(a[3]))
    return np.array(pts, dtype=np.float32).T, np.array(kk, dtype=np.uint64)


def test_keys_golden():
    pos, expect = _read_golden_keys()
    np.testing.assert_array_equal(oracle.keys(pos), expect)


def _deinterleave(k):
    k = int(k)
    q = [0, 0, 0]
    for b in range(21):
        for a in range(3):
            q[a] |= ((k >> (3 * b + a)) & 1) << b
    return q


def test_keys_quantisation_properties():
    """Each axis code lies within one grid unit of (x - min) 2^21 / L, codes
    are in range, and code order follows coordinate order."""
    w = ics.hernquist(2000, seed=3)
    p32 = w.pos.astype(np.float32)
    k = oracle.keys(p32)
    lo, L, s = oracle.bounds(p32)
    assert L == max(float(p32[a].max()) - float(p32[a].min()) for a in range(3))
    q = np.array([_deinterleave(v) for v in k]).T
    assert q.min() >= 0 and q.max() <= 2 ** 21 - 1
    exact = (p32.astype(np.float64) - lo[:, None]) * (2 ** 21 / L)
    assert np.all(q <= exact + 1e-6) and np.all(q >= np.minimum(exact, 2 ** 21 - 1) - 1 - 1e-6)
    for a in range(3):
        o = np.argsort(p32[a], kind="stable")
        assert np.all(np.diff(q[a][o]) >= 0)


def test_sort_matches_library_stable_sort():
    g = ics.rng(7)
    key = g.integers(0, 50, 3000).astype(np.uint64)         # many ties
    sk, perm = oracle.stable_sort(key)
    ref = np.argsort(key, kind="stable")
    np.testing.assert_array_equal(perm, ref)
    np.testing.assert_array_equal(sk, key[ref])


# ---------------------------------------------------------------------------
# tree
# ---------------------------------------------------------------------------
def _read_sections(name):
    sec, out = None, {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            sec = line.strip("[]")
            out[sec] = []
            continue
        out[sec].append([float(v) if sec == "points" else int(v) for v in line.split()])
    return out


def test_tiny_tree_golden():
    g = _read_sections("tiny_tree.txt")
    pos = np.array(g["points"], dtype=np.float32).T
    T = oracle.Tree(pos, np.ones(pos.shape[1], np.float32), n_leaf=2, group=2)
    np.testing.assert_array_equal(T.perm, np.array(g["perm"][0]))
    np.testing.assert_array_equal(T.cells, np.array(g["cells"]))
    np.testing.assert_array_equal(T.groups, np.array(g["groups"]))


def _check_tree_invariants(T, n_leaf, G):
    cells = T.cells
    n = T.n
    lev, first, cnt, child, nch, par = (cells[:, i] for i in range(6))
    # breadth-first order
    order = np.lexsort((first, lev))
    np.testing.assert_array_equal(order, np.arange(T.ncell))
    assert cnt[0] == n and first[0] == 0 and lev[0] == 0
    leaf_cover = np.zeros(n, dtype=np.int64)
    q = np.array([_deinterleave(k) for k in T.key]).T if n <= 5000 else None
    for c in range(T.ncell):
        if nch[c] == 0:
            assert cnt[c] <= n_leaf or lev[c] == 21
            leaf_cover[first[c]:first[c] + cnt[c]] += 1
        else:
            assert cnt[c] > n_leaf and lev[c] < 21
            kids = np.arange(child[c], child[c] + nch[c])
            assert np.all(par[kids] == c) and np.all(lev[kids] == lev[c] + 1)
            assert first[kids[0]] == first[c]
            assert np.all(first[kids][1:] == (first[kids] + cnt[kids])[:-1])
            assert first[kids[-1]] + cnt[kids[-1]] == first[c] + cnt[c]
        if q is not None:
            s = 1 << (21 - lev[c])
            sl = slice(first[c], first[c] + cnt[c])
            for a in range(3):
                o = cells[c, 6 + a]
                assert np.all((q[a][sl] >= o) & (q[a][sl] < o + s))
    assert np.all(leaf_cover == 1)
    # groups: each unit (a maximal cell with <= 16 G particles, or a leaf with
    # more) cut into runs of G, the last one shorter; together they partition
    # the particles; each box is the tightest one holding its particles' cells
    U = 16 * G
    unit = [c for c in range(T.ncell) if (cnt[c] <= U and (par[c] < 0 or cnt[par[c]] > U)) or
            (nch[c] == 0 and cnt[c] > U)]
    want = [(f, min(G, first[c] + cnt[c] - f)) for c in sorted(unit, key=lambda c: first[c])
            for f in range(first[c], first[c] + cnt[c], G)]
    gs = T.groups
    np.testing.assert_array_equal(gs[:, :2], np.array(want).reshape(-1, 2))
    assert gs[:, 1].sum() == n
    if q is not None:
        for f, k, *box in gs:
            for a in range(3):
                assert box[a] == q[a][f:f + k].min() and box[3 + a] == q[a][f:f + k].max() + 1


@pytest.mark.parametrize("n,n_leaf,G", [(1, 16, 32), (2, 1, 1), (33, 16, 32), (1000, 8, 32), (3000, 16, 64),
                                        (4000, 8, 4), (5000, 64, 2)])
def test_tree_invariants(n, n_leaf, G):
    w = ics.hernquist(n, seed=n)
    T = oracle.Tree(w.pos.astype(np.float32), w.mass.astype(np.float32), n_leaf, G)
    _check_tree_invariants(T, n_leaf, G)


def test_tree_coincident_particles():
    """All particles at one point: one chain of single-child cells down to an
    overflow leaf at level 21; groups of G share one grid cell as their box."""
    pos = np.full((3, 100), 0.25, dtype=np.float32)
    T = oracle.Tree(pos, np.ones(100, np.float32), 16, 32)
    assert T.ncell == 22 and T.cells[-1, 0] == 21 and T.cells[-1, 2] == 100
    assert list(T.groups[:, 1]) == [32, 32, 32, 4]
    assert np.all(T.groups[:, 5:] - T.groups[:, 2:5] == 1)


def test_moments_two_point_closed_form():
    """Two masses m at +-d on x about the origin: COM 0, Q_xx = 4 m d^2,
    Q_yy = Q_zz = -2 m d^2, no off-diagonal terms."""
    d = 0.25
    pos = np.array([[-d, d], [0.0, 0.0], [0.0, 0.0]], dtype=np.float32)
    T = oracle.Tree(pos, np.array([3.0, 3.0], np.float32), 16, 32)
    mo = T.moments[0]
    np.testing.assert_allclose(mo[:4], [6.0, 0.0, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(mo[4:], [4 * 3 * d * d, -2 * 3 * d * d, -2 * 3 * d * d, 0, 0, 0], atol=1e-15)


def test_moments_far_field_convergence():
    """Multipole field of a cell vs brute-force direct sum of its particles:
    the monopole error falls as (s/r)^2 relative, the quadrupole one as (s/r)^3,
    and adding the quadrupole term reduces the error."""
    g = ics.rng(9)
    pts = g.uniform(-0.5, 0.5, (3, 40))
    m = g.uniform(0.5, 1.5, 40)
    pos = pts.astype(np.float32)
    T = oracle.Tree(pos, m.astype(np.float32), 64, 64)       # one leaf = the root
    M = T.moments[0]
    errs = {}
    for quad in (False, True):
        for R in (8.0, 16.0):
            tgt = np.array([[R], [0.3 * R], [-0.2 * R]])
            exact, _ = oracle.direct(np.concatenate([pos.astype(np.float64), tgt], 1),
                                     np.concatenate([m.astype(np.float32).astype(np.float64), [0.0]]), 0.0,
                                     targets=[40])
            r = tgt[:, 0] - M[1:4]
            rr = np.linalg.norm(r)
            a = -M[0] * r / rr ** 3
            if quad:
                Q = np.array([[M[4], M[7], M[8]], [M[7], M[5], M[9]], [M[8], M[9], M[6]]])
                Qr = Q @ r
                a = a + Qr / rr ** 5 - 2.5 * (r @ Qr) * r / rr ** 7
            errs[(quad, R)] = np.linalg.norm(a - exact[:, 0]) / np.linalg.norm(exact[:, 0])
    assert errs[(True, 8.0)] < errs[(False, 8.0)]
    assert 2.6 < errs[(False, 8.0)] / errs[(False, 16.0)] < 5.5     # ~ 2^2
    assert 5.0 < errs[(True, 8.0)] / errs[(True, 16.0)] < 11.0      # ~ 2^3
    assert abs(M[4] + M[5] + M[6]) < 1e-12 * abs(M[4:7]).max()       # traceless


# ---------------------------------------------------------------------------
# walk
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def plummer_case():
    w = ics.plummer_workload()
    p32 = w.stars.pos.astype(np.float32)
    m32 = w.stars.mass.astype(np.float32)
    ad, pd = oracle.direct(p32.astype(np.float64), m32.astype(np.float64), 0.01)
    return p32, m32, ad, pd


def test_walk_small_theta_equals_direct(plummer_case):
    p32, m32, ad, pd = plummer_case
    T = oracle.Tree(p32, m32, 16, 32)
    a, p, _, _ = T.forces(1e-6, 0.01)
    assert oracle.rel_err(a, ad).max() < 1e-12
    np.testing.assert_allclose(p, pd, rtol=1e-12)


def test_walk_accuracy_ordering(plummer_case):
    """p99 vs direct <= 1e-3 at theta = 0.5 with quadrupoles; error grows with
    theta and is larger without the quadrupole term."""
    p32, m32, ad, _ = plummer_case
    T = oracle.Tree(p32, m32, 16, 32)
    p99 = {}
    for th in (0.3, 0.5, 0.7):
        for q in (False, True):
            a, _, _, _ = T.forces(th, 0.01, q)
            p99[(th, q)] = oracle.percentile(oracle.rel_err(a, ad), 0.99)
    assert p99[(0.5, True)] <= 1e-3
    assert p99[(0.3, True)] < p99[(0.5, True)] < p99[(0.7, True)]
    for th in (0.3, 0.5, 0.7):
        assert p99[(th, True)] < p99[(th, False)]


def test_relative_mac_zero_tolerance_is_direct(plummer_case):
    """alpha = 0: no massive cell passes M s^2 <= 0, so the walk is the direct sum."""
    p32, m32, ad, pd = plummer_case
    T = oracle.Tree(p32, m32, 16, 32)
    aref = ad.astype(np.float32)
    a, p, cnt = T.forces_rel(0.0, 0.01, aref, counts=True)
    assert cnt[:, 1].sum() == 0
    assert oracle.rel_err(a, ad).max() < 1e-12
    np.testing.assert_allclose(p, pd, rtol=1e-12)


def test_relative_mac_error_follows_tolerance(plummer_case):
    """The error grows with the tolerance alpha and stays below it (the
    criterion bounds the monopole truncation term by alpha |a|; the quadrupole
    term makes the actual error smaller), and fewer interactions are needed."""
    p32, m32, ad, _ = plummer_case
    T = oracle.Tree(p32, m32, 16, 32)
    aref = ad.astype(np.float32)
    p99, work = {}, {}
    for al in (1e-4, 1e-3, 1e-2):
        a, _, cnt = T.forces_rel(al, 0.01, aref, counts=True)
        p99[al] = oracle.percentile(oracle.rel_err(a, ad), 0.99)
        work[al] = cnt.sum()
        assert p99[al] < al
    assert p99[1e-4] < p99[1e-3] < p99[1e-2]
    assert work[1e-4] > work[1e-3] > work[1e-2]


def test_relative_mac_scale_invariance(plummer_case):
    """The criterion is dimensionally consistent: M s^2 <= alpha |a| d^4 is
    unchanged when masses and |a| are scaled by c, and when lengths are doubled
    (|a| / 4, softening x 2): same opening decisions, forces scaled exactly."""
    p32, m32, ad, _ = plummer_case
    aref = ad.astype(np.float32)
    T = oracle.Tree(p32, m32, 16, 32)
    a0, _, c0 = T.forces_rel(1e-3, 0.01, aref, counts=True)
    T2 = oracle.Tree(p32, (m32 * np.float32(8.0)).astype(np.float32), 16, 32)
    a2, _, c2 = T2.forces_rel(1e-3, 0.01, (aref * np.float32(8.0)).astype(np.float32), counts=True)
    np.testing.assert_array_equal(c2, c0)
    np.testing.assert_allclose(a2, 8.0 * a0, rtol=1e-12)
    T3 = oracle.Tree((p32 * np.float32(2.0)).astype(np.float32), m32, 16, 32)
    a3, _, c3 = T3.forces_rel(1e-3, 0.02, (aref / np.float32(4.0)).astype(np.float32), counts=True)
    np.testing.assert_array_equal(c3, c0)
    np.testing.assert_allclose(a3, a0 / 4.0, rtol=1e-12)


def test_relative_mac_without_reference_uses_theta(plummer_case):
    """Groups whose smallest reference |a| is 0 (before any force pass) fall
    back to the opening-angle test: all-zero references reproduce the walk at
    theta exactly."""
    p32, m32, _, _ = plummer_case
    T = oracle.Tree(p32, m32, 16, 32)
    a0, p0, _, _, c0 = T.forces(0.6, 0.01, True, counts=True)
    a1, p1, c1 = T.forces_rel(1e-3, 0.01, np.zeros((3, p32.shape[1]), np.float32), counts=True, theta=0.6)
    np.testing.assert_array_equal(c1, c0)
    np.testing.assert_array_equal(a1, a0)
    np.testing.assert_array_equal(p1, p0)


def test_relative_mac_safeguard():
    """A cluster of 1000 stars inside the cell [0.5, 0.625)^3 (side s = 1/8)
    and a group of 8 stars at distance delta beside its +x face. With a huge
    tolerance every separated cell passes M s^2 <= alpha |a| d^4, so only the
    safeguard decides: within s/10 = 0.0125 the group must open the cluster's
    cell (more, smaller multipoles); beyond it the cell is one multipole, as
    far away; touching the face, leaves are opened down to single stars."""
    g = ics.rng(31)
    A = g.uniform(0.51, 0.615, (3, 1000))
    corners = np.array([[0.0, 1.0], [0.0, 1.0], [0.0, 1.0]])   # bounding cube [0, 1]^3
    cnt = {}
    for delta in (0.0003, 0.011, 0.014, 0.1):
        B = np.array([0.625 + delta, 0.56, 0.56])[:, None] + g.uniform(-1e-4, 1e-4, (3, 8))
        pos = np.concatenate([A, B, corners], 1).astype(np.float32)
        m = np.full(pos.shape[1], 1.0 / pos.shape[1], dtype=np.float32)
        T = oracle.Tree(pos, m, 16, 8)
        assert T.L == 1.0
        _, _, c = T.forces_rel(1e30, 0.001, np.ones((3, pos.shape[1]), np.float32), counts=True)
        cnt[delta] = c[1000:1008]
    far = cnt[0.1]
    np.testing.assert_array_equal(cnt[0.014], far)            # beyond s/10: as far away
    assert np.all(cnt[0.011][:, 1] > far[:, 1] + 6)           # within s/10: the cell is opened
    assert np.all(far[:, 0] == 7)                             # only the group's own stars directly
    assert np.all(cnt[0.0003][:, 0] > 7)                      # touching: leaves of the cluster opened


def test_walk_extra_particles_match_direct(plummer_case):
    """An unsoftened centre-of-mass particle outside the tree: at small theta
    the stars' forces and its own equal the direct sum with eps = 0 pairs."""
    p32, m32, _, _ = plummer_case
    xpos = np.array([[0.3], [-0.1], [0.05]], dtype=np.float32)
    xm = np.array([0.01])
    T = oracle.Tree(p32, m32, 16, 32)
    a, p, xa, xp = T.forces(1e-6, 0.01, True, xpos, xm, [0.0])
    allpos = np.concatenate([p32, xpos], 1).astype(np.float64)
    allm = np.concatenate([m32.astype(np.float64), xm])
    eps = np.concatenate([np.full(p32.shape[1], 0.01), [0.0]])
    ad, pd = oracle.direct(allpos, allm, eps)
    assert oracle.rel_err(a, ad[:, :-1]).max() < 1e-12
    assert oracle.rel_err(xa, ad[:, -1:]).max() < 1e-12
    np.testing.assert_allclose(xp, pd[-1:], rtol=1e-12)


# ---------------------------------------------------------------------------
# chain / perturbers (Sect. 2, Eq. 3)
# ---------------------------------------------------------------------------
def test_perturber_single_member_closed_form():
    cm = np.array([0.005])
    cx = np.array([[0.1, 0.0, 0.0]])
    pm = np.array([1e-3, 2e-3])
    px = np.array([[0.1, 0.02, 0.0], [0.1, 0.0, -0.04]])
    r = oracle.perturber(cm, cx, pm, px)
    np.testing.assert_allclose(r["a_pert"], 0.0, atol=1e-18)       # resolved == CoM for one member
    expect = 1e-3 * np.array([0, 0.02, 0]) / 0.02 ** 3 + 2e-3 * np.array([0, 0, -0.04]) / 0.04 ** 3
    np.testing.assert_allclose(r["a_chain"][0], expect, rtol=1e-14)
    np.testing.assert_allclose(r["corr"], expect, rtol=1e-14)
    np.testing.assert_allclose(r["sub"], expect, rtol=1e-14)


def test_perturber_binary_newton_third_law():
    """sum_k m_k a_chain[k] (perturbers on members) balances the resolved
    members' pull on the perturbers; Eq. 3 gives M_chain corr = sum m_k a_k."""
    b = ics.central_binary()
    g = ics.rng(3)
    px = g.normal(0, 0.02, (50, 3))
    pm = np.full(50, 1e-5)
    r = oracle.perturber(b.mass, b.pos, pm, px)
    resolved_on_p = r["a_pert"].copy()
    M = b.mass.sum()
    com = b.com
    for p in range(50):
        d = com - px[p]
        resolved_on_p[p] += M * d / np.linalg.norm(d) ** 3
    f_members = (b.mass[:, None] * r["a_chain"]).sum(0)
    f_perts = (pm[:, None] * resolved_on_p).sum(0)
    np.testing.assert_allclose(f_members, -f_perts, rtol=1e-12, atol=1e-12 * np.abs(f_members).max())
    np.testing.assert_allclose(M * r["corr"], f_members, rtol=1e-13)


def _probe_tree(points):
    """A tree of massless probe stars (they feel the extra particles only)."""
    pos = np.asarray(points, dtype=np.float32).T.copy()
    return oracle.Tree(pos, np.zeros(pos.shape[1], np.float32), 16, 32), pos


def test_chain_quadrupole_two_point_closed_form():
    """Chain of two masses m at +-s on z: Q_zz = 4 m s^2, Q_xx = Q_yy = -2 m s^2.
    With x = s/r, the exact field on the axis is -(m/r^2)(1/(1-x)^2 + 1/(1+x)^2)
    = -(m/r^2)(2 + 6x^2 + 10x^4 + ...), potential -(m/r)(2 + 2x^2 + 2x^4 ...);
    in the plane -(2m/r^2)(1 - 3/2 x^2 + ...), potential -(2m/r)(1 - x^2/2 + ...).
    Centre of mass plus quadrupole must give exactly the first two terms, on
    stars and on another extra particle."""
    m, s, r = 0.005, 0.0055, 0.05
    x = s / r
    mom = oracle.chain_moments([m, m], [[0, 0, s], [0, 0, -s]])
    assert mom["M"] == 2 * m
    np.testing.assert_allclose(mom["com"], 0.0, atol=1e-18)
    np.testing.assert_allclose(mom["Q"], [-2 * m * s * s, -2 * m * s * s, 4 * m * s * s, 0, 0, 0], rtol=1e-14,
                               atol=1e-20)
    T, pos = _probe_tree([[0.0, 0.0, r], [r, 0.0, 0.0]])
    xpos = np.array([[0.0, 0.0], [0.0, 0.0], [0.0, 3 * r]], np.float32)
    a, p, xa, xp = T.forces(0.5, 0.0, True, xpos, [2 * m, 0.0], [0.0, 0.0],
                            extra_quad=[mom["Q"], np.zeros(6)])
    rz, rx = float(pos[2, 0]), float(pos[0, 1])      # the FP32 probe positions
    xz, xx = s / rz, s / rx
    np.testing.assert_allclose(a[:, 0], [0, 0, -(m / rz ** 2) * (2 + 6 * xz * xz)], rtol=1e-13, atol=1e-18)
    np.testing.assert_allclose(p[0], -(m / rz) * (2 + 2 * xz * xz), rtol=1e-13)
    np.testing.assert_allclose(a[:, 1], [-(m / rx ** 2) * (2 - 3 * xx * xx), 0, 0], rtol=1e-13, atol=1e-18)
    np.testing.assert_allclose(p[1], -(m / rx) * (2 - xx * xx), rtol=1e-13)
    r3 = float(xpos[2, 1])
    x3 = s / r3
    np.testing.assert_allclose(xa[:, 1], [0, 0, -(m / r3 ** 2) * (2 + 6 * x3 * x3)], rtol=1e-13, atol=1e-18)
    # the exact two-body field differs by the next (x^4) term only
    exact_axis = -m / (rz - s) ** 2 - m / (rz + s) ** 2
    assert abs(a[2, 0] - exact_axis) == pytest.approx(10 * m / rz ** 2 * xz ** 4, rel=0.1)
    assert x < 0.2


def test_chain_quadrupole_far_field_order():
    """Three unequal chain members: against the resolved field, the centre of
    mass alone errs by O((s/r)^2) of the monopole and the centre of mass plus
    quadrupole by O((s/r)^3): doubling r divides the errors by ~4 and ~8."""
    g = ics.rng(31)
    cm = np.array([0.004, 0.001, 0.0025])
    cx = g.uniform(-0.01, 0.01, (3, 3))
    mom = oracle.chain_moments(cm, cx)
    direction = np.array([0.6, -0.48, 0.64])
    errs = {}
    for R in (1.0, 2.0):
        probe = mom["com"] + R * direction
        T, pos = _probe_tree([probe])
        xp = mom["com"].astype(np.float32).reshape(3, 1)
        allp = np.concatenate([pos.astype(np.float64), cx.T], 1)
        ad, _ = oracle.direct(allp, np.concatenate([[0.0], cm]), 0.0, targets=[0])
        mono = np.linalg.norm(ad[:, 0])
        for quad in (False, True):
            a = T.forces(0.5, 0.0, True, xp, [mom["M"]], [0.0], extra_quad=[mom["Q"]] if quad else None)[0]
            errs[quad, R] = np.linalg.norm(a[:, 0] - ad[:, 0]) / mono
    assert errs[True, 1.0] < 0.05 * errs[False, 1.0]
    assert 3.5 < errs[False, 1.0] / errs[False, 2.0] < 4.5
    assert 7.0 < errs[True, 1.0] / errs[True, 2.0] < 9.0


def test_chain_quadrupole_skips_perturbers_closed_form():
    """Binary of masses m at +-s on z, two probe stars on the axis: the one
    flagged as a perturber keeps the centre-of-mass point mass (-2m/r^2), and
    with its perturber correction it gets the exact two-body field; the other
    gets the centre of mass plus the quadrupole (-(m/r^2)(2 + 6 x^2))."""
    m, s = 0.005, 0.0055
    cx = np.array([[0, 0, s], [0, 0, -s]])
    mom = oracle.chain_moments([m, m], cx)
    T, pos = _probe_tree([[0.0, 0.0, 0.02], [0.0, 0.0, -0.03]])
    xp = np.zeros((3, 1), np.float32)
    a = T.forces(0.5, 0.0, True, xp, [2 * m], [0.0], extra_quad=[mom["Q"]], quad_skip=[0])[0]
    r0, r1 = float(pos[2, 0]), float(-pos[2, 1])
    np.testing.assert_allclose(a[2, 0], -2 * m / r0 ** 2, rtol=1e-14)
    np.testing.assert_allclose(a[2, 1], (m / r1 ** 2) * (2 + 6 * (s / r1) ** 2), rtol=1e-13)
    o = oracle.perturber([m, m], cx, [0.0], pos[:, :1].T.astype(np.float64))
    exact = -m / (r0 - s) ** 2 - m / (r0 + s) ** 2
    np.testing.assert_allclose(a[2, 0] + o["a_pert"][0, 2], exact, rtol=1e-12)


def test_absorption_closed_form():
    """Eq. 4: a chain of two equal masses at +-0.006 on x (centre 0, chain
    radius 0.006) absorbs exactly the stars closer than 0.006: stars placed at
    radii 0.0059 and 0.0061 in several directions, plus one at the FP32 value
    of 0.006 itself (just above 0.006, so outside: the test is strict)."""
    cm = np.array([0.005, 0.005])
    cx = np.array([[0.006, 0.0, 0.0], [-0.006, 0.0, 0.0]])
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, -1], [0.6, 0.8, 0.0], [0.0, -0.6, 0.8]])
    pts, want = [], []
    for r in (0.0059, 0.0061):
        for d in dirs:
            pts.append(r * d)
            want.append(r < 0.006)
    pts.append([0.006, 0.0, 0.0])
    want.append(False)
    pos = np.array(pts, dtype=np.float32).T.copy()
    idx, rch = oracle.absorb(pos, cm, cx)
    assert rch == 0.006
    np.testing.assert_array_equal(idx, np.flatnonzero(want))
    assert len(idx) == 5


def test_escape_rules_closed_form():
    """Eq. 5 and the membership rules: r_escape = gamma r_chain0 = 1.5; a member
    beyond it escapes only when receding; while perturbers are absorbed,
    escapes wait unless the chain radius exceeds 1.05 r_escape; fewer than two
    members left, or the designated SMBH leaving with no other SMBH, ends the
    chain; with another SMBH left, the heavier remaining one takes over."""
    eps = 1e-9                                                 # stars' masses: the centre stays at the SMBH
    m = [1.0, eps, eps]
    x = [[0, 0, 0], [1.55, 0, 0], [0, 2.0, 0]]
    v = [[0, 0, 0], [1.0, 0, 0], [0, -1.0, 0]]                # star 1 recedes, star 2 approaches
    r = oracle.chain_escape(m, x, v, [1, 0, 0], 0, 1.0, 1.5, 0)
    assert list(r["escape"]) == [False, True, False] and r["terminate"] == 0 and r["designated"] == 0
    assert r["r_escape"] == 1.5 and abs(r["r_chain"] - 2.0) < 1e-8
    # absorbing while the chain radius (2.0) is above 1.05 x 1.5: the escape goes ahead
    assert list(oracle.chain_escape(m, x, v, [1, 0, 0], 0, 1.0, 1.5, 3)["escape"]) == [False, True, False]
    # chain radius 1.55 < 1.575: the escape waits for the absorption
    x2 = [[0, 0, 0], [1.55, 0, 0], [0, 1.2, 0]]
    assert not oracle.chain_escape(m, x2, v, [1, 0, 0], 0, 1.0, 1.5, 1)["escape"].any()
    assert list(oracle.chain_escape(m, x2, v, [1, 0, 0], 0, 1.0, 1.5, 0)["escape"]) == [False, True, False]
    # two members, the star escapes: one left, the chain ends
    r = oracle.chain_escape([1.0, eps], [[0, 0, 0], [2.0, 0, 0]], [[0, 0, 0], [1.0, 0, 0]], [1, 0], 0, 1.0, 1.5, 0)
    assert list(r["escape"]) == [False, True] and r["terminate"] == 1
    # the designated SMBH (index 0) recedes from a chain dominated by two others
    mm = [0.002, 0.005, 0.004, eps]
    xx = [[3.0, 0, 0], [0, 0, 0], [0, 0.1, 0], [0, 0, 0.2]]
    vv = [[1.0, 0, 0], [0, 0, 0], [0, 0, 0], [0, 0, 0]]
    r = oracle.chain_escape(mm, xx, vv, [1, 1, 1, 0], 0, 1.0, 1.5, 0)
    assert list(r["escape"]) == [True, False, False, False] and r["terminate"] == 0 and r["designated"] == 1
    r = oracle.chain_escape(mm, xx, vv, [1, 0, 0, 0], 0, 1.0, 1.5, 0)
    assert r["terminate"] == 1


def test_tidal_selection_closed_form():
    """Eq. 2: with equal masses the criterion is a sphere of radius
    R = (2 m / (gamma M))^(1/3) r_crit; a star 8 times heavier reaches twice as
    far (the cube root of its mass ratio)."""
    g = ics.rng(41)
    n = 20000
    pos = g.uniform(-1, 1, (3, n)).astype(np.float32)
    m = np.full(n, 1e-4, np.float32)
    c = np.zeros(3, np.float32)
    M, gam, rc = np.float32(0.01), np.float32(1e-3), np.float32(0.1)
    R = (2 * 1e-4 / (float(gam) * float(M))) ** (1 / 3) * float(rc)
    r = np.linalg.norm(pos.astype(np.float64), axis=0)
    clear = np.abs(r - R) > 1e-6 * R                      # no star on the boundary within rounding
    sel = oracle.tidal(pos, m, c, M, gam, rc)
    want = np.nonzero(r < R)[0]
    assert len(want) > 50
    np.testing.assert_array_equal(sel[np.isin(sel, np.nonzero(clear)[0])], want[clear[want]])
    # eight times the mass: twice the radius
    m8 = m.copy()
    heavy = np.array([0, 1])
    pos[:, heavy] = np.array([[1.9 * R, 2.1 * R], [0, 0], [0, 0]], np.float32)
    m8[heavy] = np.float32(8e-4)
    sel8 = oracle.tidal(pos, m8, c, M, gam, rc)
    assert 0 in sel8 and 1 not in sel8
    assert np.all(np.diff(sel8) > 0)


def test_chain_start_radius_closed_form():
    """Eq. 1 ingredients on a constructed cluster: stars of mass 0.001 on
    shells at radius 0.01 k (k = 1, 2, ...), so the running mass reaches
    2 M_bh = 0.01 at the 10th star; the 50 nearest stars move with velocities
    +-0.3 along x (mean 0): sigma^2 = 0.09 / 3 = 0.03."""
    n = 200
    g = ics.rng(61)
    dirs = g.normal(size=(3, n))
    dirs /= np.linalg.norm(dirs, axis=0)
    r = 0.01 * np.arange(1, n + 1)
    pos = (dirs * r).astype(np.float32)
    vel = np.zeros((3, n), np.float32)
    vel[0, :50] = np.where(np.arange(50) % 2 == 0, 0.3, -0.3)
    m = np.full(n, 0.001, np.float32)
    out = oracle.chain_start_radius(pos, vel, m, np.zeros(3, np.float32), 0.005, 1.2, 1.5, 0.01)
    assert abs(out["r2m"] - 0.10) < 1e-7
    assert abs(out["sigma"] ** 2 - float(np.float32(0.3)) ** 2 / 3) < 1e-12
    assert abs(out["r_sigma"] - 0.005 / out["sigma"] ** 2) < 1e-12
    assert out["r_infl"] == min(out["r2m"], out["r_sigma"])
    assert abs(out["r_chain0"] - max(1.2 * out["r_infl"], 0.015)) < 1e-15
    # not enough mass: infinite r(<2M)
    assert oracle.chain_start_radius(pos[:, :5], vel[:, :5], m[:5], np.zeros(3, np.float32), 0.005, 1, 1,
                                     0.01)["r2m"] == np.inf


def test_knn_and_radius_selection():
    w = ics.hernquist(3000, seed=21)
    p32 = w.pos.astype(np.float32)
    c = np.array([0.01, -0.02, 0.0], dtype=np.float32)
    d = p32 - c[:, None]
    d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
    assert d2.dtype == np.float32
    sel = oracle.knn(p32, c, 64)
    ref = np.lexsort((np.arange(3000), d2))[:64]
    np.testing.assert_array_equal(sel, ref)
    r2 = np.float32(0.3 * 0.3)
    rs = oracle.radius(p32, c, r2)
    np.testing.assert_array_equal(rs, np.nonzero(d2 < r2)[0])


# ---------------------------------------------------------------------------
# block time steps
# ---------------------------------------------------------------------------
def test_block_steps_single_level_is_kdk(plummer_case):
    """Every star on level 0 with L = 0: the block scheme is the global KDK
    leapfrog, operation for operation (same positions bit for bit)."""
    p32, m32, _, _ = plummer_case
    x0 = p32[:, :512].astype(np.float64)
    v0 = np.zeros_like(x0)
    m = m32[:512].astype(np.float64)

    def f(x, active=None):
        return oracle.direct(x, m, 0.01)[0]

    xk, vk, ak = oracle.kdk(x0, v0, f(x0), 1e-2, f, 5)
    xb, vb, ab, lv, upd = oracle.block_kdk(x0, v0, f, np.zeros(512, int), 0, 1e-2, 5)
    np.testing.assert_array_equal(xb, xk)
    np.testing.assert_array_equal(ab, ak)
    np.testing.assert_allclose(vb, vk + 0.5 * 1e-2 * ak, rtol=1e-15, atol=1e-18)   # plus the next opening kick
    assert upd == 5 * 512


def test_block_steps_constant_field_closed_form():
    """In a uniform field g each star's leapfrog is exact: at the end of each of
    its own steps x = x0 + v0 t + g t^2 / 2 and v (before the next opening
    kick) = v0 + g t. Stars on levels 0..3 over 16 substeps of L = 3; each
    level l takes 2^l forces per dt_max."""
    g = np.array([0.3, -0.2, 0.1])
    n = 8
    lv = np.array([0, 1, 2, 3, 0, 1, 2, 3])
    x0 = np.arange(3 * n, dtype=np.float64).reshape(3, n) * 0.1
    v0 = np.ones((3, n)) * np.array([1.0, -0.5, 0.25])[:, None]

    def f(x, active):
        return np.repeat(g[:, None], x.shape[1], 1)

    dt_max, L, nsub = 0.25, 3, 16
    xb, vb, _, _, upd = oracle.block_kdk(x0, v0, f, lv, L, dt_max, nsub)
    t = nsub * dt_max / 2 ** L
    np.testing.assert_allclose(xb, x0 + v0 * t + 0.5 * g[:, None] * t * t, rtol=1e-14, atol=1e-14)
    vt = v0 + g[:, None] * t + g[:, None] * (0.5 * dt_max * 2.0 ** -lv)      # + the next opening kick
    np.testing.assert_allclose(vb, vt, rtol=1e-14, atol=1e-14)
    assert upd == int(sum(nsub // 2 ** (L - l) for l in lv))


def test_block_level_rule_examples():
    """dt = min(tau_acc sqrt(eps/|a|), tau_vel eps/|v|); level = the smallest l
    with dt_max 2^-l <= dt (capped at L); coarser only on a step boundary."""
    tau, eps, dt_max, L = 0.5, 0.01, 1.0, 4
    # |a| = 1: dt_acc = 0.5 sqrt(0.01) = 0.05 < 1/16 -> level 5, capped at 4
    # |a| = 0.01: dt_acc = 0.5 sqrt(1) = 0.5 -> level 1 (dt_max / 2 <= 0.5)
    # |a| = 1e-4: dt_acc = 5; |v| = 0.02: dt_vel = 0.5 * 0.01 / 0.02 = 0.25 -> level 2
    # a = 0, v = 0: no limit -> level 0
    a = np.array([[1.0, 0.01, 1e-4, 0.0], [0, 0, 0, 0], [0, 0, 0, 0]], np.float32)
    v = np.array([[0.0, 0.0, 0.02, 0.0], [0, 0, 0, 0], [0, 0, 0, 0]], np.float32)
    lv = oracle.block_levels(a, v, np.zeros(4, int), 0, L, dt_max, tau, tau, eps, start=True)
    np.testing.assert_array_equal(lv, [4, 1, 2, 0])
    # star on level 4 wanting level 1 at substep 2 (L = 4): levels 1..3 end every 8, 4, 2 substeps -> level 3
    lv = oracle.block_levels(a[:, 1:2], v[:, 1:2], np.array([4]), 2, L, dt_max, tau, tau, eps)
    np.testing.assert_array_equal(lv, [3])
    lv = oracle.block_levels(a[:, 1:2], v[:, 1:2], np.array([4]), 8, L, dt_max, tau, tau, eps)
    np.testing.assert_array_equal(lv, [1])
    # an inactive star keeps its level
    lv = oracle.block_levels(a[:, 1:2], v[:, 1:2], np.array([2]), 3, L, dt_max, tau, tau, eps)
    np.testing.assert_array_equal(lv, [2])


# ---------------------------------------------------------------------------
# spline softening
# ---------------------------------------------------------------------------
def _pair(r, e, kind=1):
    pos = np.array([[0.0, r], [0.0, 0.0], [0.0, 0.0]])
    a, p = oracle.direct(pos, np.array([1.0, 1.0]), e, targets=[0], kind=kind)
    return a[0, 0], p[0]


def test_spline_newton_beyond_support():
    """At r >= h = 2.8 eps the spline field is Newton's exactly."""
    e = 0.01
    for r in (0.028, 0.03, 0.5, 7.0):
        a, p = _pair(r, e)
        assert abs(a - 1.0 / r ** 2) <= 1e-14 / r ** 2 and abs(p + 1.0 / r) <= 1e-14 / r


def test_spline_centre_and_continuity():
    """phi(0) = -m/eps (the Plummer-equivalent length: -2.8 m / h); a(0) = 0;
    force and potential are continuous at u = 1/2 and u = 1."""
    e = 0.01
    h = 2.8 * e
    a0, p0 = _pair(0.0, e)
    assert a0 == 0.0 and abs(p0 + 1.0 / e) <= 1e-12 / e
    for u in (0.5, 1.0):
        lo = _pair(u * h * (1 - 1e-10), e)
        hi = _pair(u * h * (1 + 1e-10), e)
        assert abs(lo[0] - hi[0]) <= 1e-8 * abs(hi[0]) and abs(lo[1] - hi[1]) <= 1e-8 * abs(hi[1])


def test_spline_force_is_minus_gradient_and_mass_is_enclosed():
    """a(r) = -dphi/dr (central differences), and r^2 a(r) -- the kernel's
    enclosed mass -- grows from 0 to m at r = h."""
    e = 0.01
    h = 2.8 * e
    for u in (0.1, 0.3, 0.45, 0.55, 0.7, 0.95):
        r, d = u * h, 1e-6 * h
        a, _ = _pair(r, e)
        dp = (_pair(r + d, e)[1] - _pair(r - d, e)[1]) / (2 * d)
        assert abs(a - dp) <= 1e-6 * abs(a), (u, a, dp)
    enc = [(_pair(u * h, e)[0]) * (u * h) ** 2 for u in np.linspace(0.05, 1.0, 20)]
    assert np.all(np.diff(enc) > 0) and abs(enc[-1] - 1.0) < 1e-12


def test_spline_tree_matches_direct(plummer_case):
    """The tree with spline softening at small theta equals the spline direct
    sum; at theta 0.5 it stays within 1e-3 at p99."""
    p32, m32, _, _ = plummer_case
    ad, pd = oracle.direct(p32.astype(np.float64), m32.astype(np.float64), 0.01, kind=1)
    T = oracle.Tree(p32, m32, 16, 32)
    a, p, _, _ = T.forces(1e-6, 0.01, kind=1)
    assert oracle.rel_err(a, ad).max() < 1e-12
    np.testing.assert_allclose(p, pd, rtol=1e-12)
    a, _, _, _ = T.forces(0.5, 0.01, kind=1)
    assert oracle.percentile(oracle.rel_err(a, ad), 0.99) <= 1e-3


def test_a_hard_worked_example():
    """Eq. 13 against the value the paper prints (tests/golden/a_hard.txt), the
    closed form mu/(M1+M2) = M1 M2/(M1+M2)^2 for unequal masses, and its
    independence of the mass unit."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "a_hard.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for m1, m2, r, a in rows:
        assert oracle.a_hard(float(m1), float(m2), float(r)) == pytest.approx(float(a), rel=1e-15)
    assert oracle.a_hard(1.0, 3.0, 2.0) == pytest.approx(3.0 / 16.0 * 2.0 / 4.0, rel=1e-15)
    assert oracle.a_hard(7e-3, 2e-3, 0.3) == pytest.approx(oracle.a_hard(7.0, 2.0, 0.3), rel=1e-14)
