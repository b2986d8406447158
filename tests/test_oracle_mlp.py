"""Pins for the oracle of the learned cell-force correction: bfloat16
rounding against hand-derived values, the analytic backward against finite
differences, Adam against its closed form on one step, and the cell
residual against the special cases that fix it."""
import numpy as np
import pytest

import ics
import oracle


def test_bf16_round_hand_values():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 3.0e38, 1 + 2 ** -7], dtype=np.float32)
    # spacing near 1 is 2^-7: 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-8 -> 1 + 2^-6
    r = oracle.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2 ** -6 and r[3] == -2.5 and r[5] == 1 + 2 ** -7
    assert abs(r[4] / 3.0e38 - 1) < 2 ** -8


def _round8(v):
    """Nearest value with 8 significant bits (bfloat16's), ties to even,
    written from frexp: an implementation independent of oracle.bf16_round."""
    import math
    m, e = math.frexp(v)                 # v = m 2^e, 0.5 <= |m| < 1
    q = m * 256.0                        # 8 significant bits
    fl = math.floor(q)
    r = fl + 1 if (q - fl > 0.5 or (q - fl == 0.5 and fl % 2 == 1)) else fl
    return math.ldexp(r / 256.0, e)


def test_mlp_forward_rounding_points_one_row_by_hand():
    """One row through a network whose only nonzero path is x0 -> h1_0 -> h2_0
    -> y0: the input and the weights 1 + 2^-9 round to 1 in bfloat16, and the
    hidden activations silu(1) and silu(2 h1 + b) are rounded to 8 significant
    bits (b = -1.4609375 + 2^-5 puts the second layer's input near 0, where the
    first rounding is not hidden by the second), so y0 = r(silu(2 r(silu(1)) +
    b)) + 1/4 exactly; every other output is its bias. Without the roundings
    the same row gives the plain FP64 value."""
    import math
    p = {k: np.zeros(v) for k, v in (("W1", (16, 64)), ("b1", 64), ("W2", (64, 64)), ("b2", 64), ("W3", (64, 8)),
                                     ("b3", 8))}
    a = 1 + 2 ** -9
    p["W1"][0, 0] = a
    p["W2"][0, 0] = 2.0
    b = -1.4609375 + 2 ** -5
    p["b2"][0] = b
    p["W3"][0, 0] = a
    p["b3"][:3] = [0.25, -0.5, 0.125]
    X = np.zeros((1, 16))
    X[0, 0] = a
    silu = lambda z: z / (1.0 + math.exp(-z))
    h1 = _round8(silu(1.0))
    h2 = _round8(silu(2.0 * h1 + b))
    y, _ = oracle.mlp_forward(p, X, rounding=True)
    assert h1 != silu(1.0) and h2 != silu(2.0 * h1 + b)        # both roundings change the value
    assert _round8(silu(2.0 * silu(1.0) + b)) != h2             # and the first is visible after the second
    # the other hidden units are silu(0) = 0 and add nothing
    np.testing.assert_array_equal(y[0], [h2 + 0.25, -0.5, 0.125])
    y0, _ = oracle.mlp_forward(p, X, rounding=False)
    z1 = a * a
    np.testing.assert_allclose(y0[0], [silu(2.0 * silu(z1) + b) * a + 0.25, -0.5, 0.125], rtol=1e-14)


def _params(seed):
    g = ics.rng(seed)
    p = {"W1": g.normal(0, 0.3, (16, 64)), "b1": g.normal(0, 0.1, 64), "W2": g.normal(0, 0.15, (64, 64)),
         "b2": g.normal(0, 0.1, 64), "W3": g.normal(0, 0.15, (64, 8)), "b3": g.normal(0, 0.1, 8)}
    p["W1"][11:] = 0.0
    p["W3"][:, 3:] = 0.0
    p["b3"][3:] = 0.0
    return p


def test_mlp_backward_matches_finite_differences():
    g = ics.rng(3)
    p = _params(4)
    X = np.zeros((32, 16))
    X[:, :14] = g.normal(0, 1, (32, 14))
    T = g.normal(0, 0.3, (32, 3))
    loss, grad = oracle.mlp_loss_grad(p, X, T, rounding=False)
    h = 1e-6
    for k, idx in [("W1", (3, 7)), ("b1", (5,)), ("W2", (10, 20)), ("b2", (63,)), ("W3", (4, 2)), ("b3", (1,))]:
        q = {a: b.copy() for a, b in p.items()}
        q[k][idx] += h
        lp, _ = oracle.mlp_loss_grad(q, X, T, rounding=False)
        q[k][idx] -= 2 * h
        lm, _ = oracle.mlp_loss_grad(q, X, T, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[k][idx]) <= 1e-6 * max(1e-3, abs(fd)), (k, fd, grad[k][idx])


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (oracle.silu(z + h) - oracle.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(oracle.silu_grad(z), fd, atol=1e-8)


def test_adam_first_step_is_sign_times_lr():
    """After one step from zero moments, the bias-corrected update is
    -lr g / (|g| + eps) per entry."""
    p = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -4.0, 1e-3])}
    st = {}
    q = oracle.adam_step({"a": p["a"].copy()}, g, st, lr=0.01)
    np.testing.assert_allclose(q["a"], p["a"] - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8), rtol=1e-12)


def test_cell_residual_special_cases():
    """A one-star cell has no residual (it is its own monopole); a far target
    sees a residual that falls faster than the quadrupole term."""
    w = ics.plummer(2000, 9)
    T = oracle.Tree(w.pos.astype(np.float32), w.mass.astype(np.float32), 1, 1)
    one = [c for c in range(T.ncell) if T.cells[c, 2] == 1][0]
    x = np.array([T.moments[one, 1] + 0.3, T.moments[one, 2], T.moments[one, 3]])
    np.testing.assert_allclose(oracle.cell_residual(T, one, x, 0.0), 0.0, atol=1e-12)
    big = [c for c in range(T.ncell) if T.cells[c, 2] > 50][-1]
    com = T.moments[big, 1:4]
    s = T.L / 2.0 ** T.cells[big, 0]
    res = [np.linalg.norm(oracle.cell_residual(T, big, com + np.array([k * s, 0.3 * s, 0.0]), 0.0))
           for k in (4.0, 8.0)]
    assert res[0] / res[1] > 12.0   # octupole ~ (s/r)^5 relative scaling of the force: ~32x per doubling
    f, norm = oracle.cell_features(T, big, com + np.array([4 * s, 0.0, 0.0]), 0.0)
    assert abs(np.linalg.norm(f[:3]) - 1) < 1e-12 and abs(f[3] - 0.25) < 1e-12 and f[4] == 0.0


def test_splitmix64_published_outputs():
    """The first outputs of SplitMix64 from state 0 (state advancing by the
    golden-ratio increment), as published with the generator."""
    g = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(g) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * g) % (1 << 64)) == 0x06C45D188009454F


def test_minibatch_rows_uniform_and_in_range():
    """The draw covers 0..n-1 uniformly (chi-square over 16 bins) and is a
    function of (seed, step, row) only."""
    n = 1000
    r = np.concatenate([oracle.minibatch_rows(7, k, 500, n) for k in range(8)])
    assert r.min() >= 0 and r.max() < n
    h = np.bincount(r * 16 // n, minlength=16)
    chi2 = ((h - r.size / 16) ** 2 / (r.size / 16)).sum()
    assert chi2 < 40.0                                    # 15 degrees of freedom: p ~ 5e-4
    np.testing.assert_array_equal(oracle.minibatch_rows(7, 3, 500, n), r[1500:2000])
    assert not np.array_equal(oracle.minibatch_rows(8, 3, 500, n), r[1500:2000])


def test_mlp_train_lowers_the_loss_of_a_learnable_target():
    """Trained on targets a small network of the same shape produces, the
    loop's loss falls by more than 10x within 300 steps."""
    tp = _params(41)
    X = np.zeros((512, 16))
    X[:, :14] = ics.rng(42).normal(0, 1, (512, 14))
    T, _ = oracle.mlp_forward(tp, X, rounding=False)
    start = _params(43)
    for k in start:
        start[k] = 0.3 * start[k]
    losses, _ = oracle.mlp_train(start, X, T, steps=300, batch=64, lr=3e-3, seed=5, rounding=False)
    assert np.mean(losses[-20:]) < 0.1 * np.mean(losses[:5])


def _traceless_brute(pos, m):
    """Traceless third moment of point masses about their centre of mass, by
    plain summation (independent of oracle.cell_octupole)."""
    com = (pos * m[:, None]).sum(0) / m.sum()
    d = pos - com
    O = np.zeros((3, 3, 3))
    for j in range(len(m)):
        for a in range(3):
            for b in range(3):
                for c in range(3):
                    O[a, b, c] += m[j] * d[j, a] * d[j, b] * d[j, c]
    t = np.array([O[a, 0, 0] + O[a, 1, 1] + O[a, 2, 2] for a in range(3)])
    for a in range(3):
        for b in range(3):
            for c in range(3):
                O[a, b, c] -= ((a == b) * t[c] + (a == c) * t[b] + (b == c) * t[a]) / 5.0
    return O


def test_octupole_feature_collinear_closed_form():
    """Two masses on the x axis (one leaf, and again as two one-star children
    of the root): O_xxx = sum m d^3, the traceless part has O_xxx (2/5) and
    O_xyy = O_xzz = -O_xxx / 5. Seen along x at distance R, v = (2/5) O_xxx x^
    is radial and the feature is (5/2)(3 - 7)(2/5) O_xxx x^ / (M R^3) =
    -4 O_xxx x^ / (M R^3); seen along y, v = -(1/5) O_xxx x^ is tangential and
    the feature is (5/2) 3 (-1/5) O_xxx x^ / (M R^3) = -1.5 O_xxx x^ / (M R^3)."""
    pos = np.array([[-0.3, 0.0, 0.0], [0.5, 0.0, 0.0]], dtype=np.float32)
    m = np.array([1.0, 3.0], dtype=np.float32)
    x64 = pos.astype(np.float64)[:, 0]
    com = (m * x64).sum() / m.sum()
    Oxxx = float((m * (x64 - com) ** 3).sum())
    for n_leaf in (4, 1):                   # one leaf, or a root with two one-star children
        T = oracle.Tree(pos.T.copy(), m, n_leaf, 32)
        assert (T.cells[0, 4] == 0) == (n_leaf == 4)
        M, R = 4.0, 10.0
        fx, _ = oracle.cell_features(T, 0, np.array([com + R, 0.0, 0.0]), 0.0)
        fy, _ = oracle.cell_features(T, 0, np.array([com, R, 0.0]), 0.0)
        np.testing.assert_allclose(fx[11:14], [-4.0 * Oxxx / (M * R ** 3), 0.0, 0.0], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(fy[11:14], [-1.5 * Oxxx / (M * R ** 3), 0.0, 0.0], rtol=1e-12, atol=1e-15)


def test_octupole_from_children_with_quadrupoles_is_exact():
    """A root with two children, each a leaf of two equal masses placed
    symmetrically about the child's centre of mass (no third moment of its
    own but a quadrupole): the children-based octupole equals the brute-force
    traceless third moment of the four stars."""
    cA, eA = np.array([-0.5, -0.4, -0.3]), np.array([0.1, 0.05, -0.02])
    cB, eB = np.array([0.4, 0.3, 0.45]), np.array([-0.05, 0.1, 0.08])
    pos = np.array([cA + eA, cA - eA, cB + eB, cB - eB], dtype=np.float32)
    m = np.array([1.0, 1.0, 2.0, 2.0], dtype=np.float32)
    T = oracle.Tree(pos.T.copy(), m, 2, 32)
    assert T.cells[0, 4] == 2 and all(T.cells[k, 4] == 0 and T.cells[k, 2] == 2 for k in (1, 2))
    ref = _traceless_brute(pos.astype(np.float64), m.astype(np.float64))
    np.testing.assert_allclose(oracle.cell_octupole(T, 0), ref, atol=1e-12 * np.abs(ref).max())


def test_octupole_feature_predicts_the_quadrupole_residual():
    """Far from a lopsided cell, the quadrupole expansion's residual in the
    output's units (residual |r|^2 / M) is the octupole feature, radial and
    tangential parts alike: the relative mismatch of the whole vector falls as
    s/r (the next order), and along the line of sight the residual is
    -10 O^T(r^, r^, r^) / r^5 written from the tensor directly."""
    g = ics.rng(77)
    pos = g.uniform(-0.5, 0.5, (3, 40)).astype(np.float32)
    pos[0, :10] += 0.3                                      # lopsided: a real octupole
    m = g.uniform(0.5, 1.5, 40).astype(np.float32)
    T = oracle.Tree(pos, m, 64, 64)                          # one leaf
    com = T.moments[0, 1:4]
    rh = np.array([0.6, -0.48, 0.64])
    O = _traceless_brute(pos.T.astype(np.float64), m.astype(np.float64))
    mis, vec = [], []
    for R in (20.0, 40.0):
        x = com + R * rh
        res = oracle.cell_residual(T, 0, x, 0.0)
        f, norm = oracle.cell_features(T, 0, x, 0.0)
        pred = -10.0 * float(np.einsum("abc,a,b,c->", O, rh, rh, rh)) / R ** 5
        mis.append(abs(res @ rh - pred) / abs(pred))
        vec.append(np.linalg.norm(res / norm - f[11:14]) / np.linalg.norm(f[11:14]))
    assert mis[0] < 0.1 and 1.6 < mis[0] / mis[1] < 2.4, mis
    assert vec[0] < 0.1 and 1.6 < vec[0] / vec[1] < 2.4, vec
