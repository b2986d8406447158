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
    X[:, :11] = g.normal(0, 1, (32, 11))
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
