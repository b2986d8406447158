"""Checks on the seeded input generators (not the method): the samples follow
the models the paper uses (Sect. 3) and are reproducible."""
import math

import numpy as np
import pytest

import ics


def test_hernquist_df_reproduces_density():
    """rho(r) = 4 pi int_0^vesc f(psi - v^2/2) v^2 dv for the closed-form DF."""
    from scipy.integrate import quad
    for r in (0.01, 0.3, 1.0, 5.0):
        psi = float(ics.hernquist_potential(r))
        val = 4 * math.pi * quad(lambda v: v * v * float(ics.hernquist_df(psi - 0.5 * v * v)), 0,
                                 math.sqrt(2 * psi), limit=200)[0]
        assert val == pytest.approx(float(ics.hernquist_density(r)), rel=1e-6)


def test_hernquist_sample_profile_and_virial():
    p = ics.hernquist(1 << 16, seed=2)
    r = np.linalg.norm(p.pos, axis=0)
    # half of the (truncated) mass inside the radius enclosing u = 0.495
    s = math.sqrt(0.495)
    assert np.median(r) == pytest.approx(s / (1 - s), rel=0.03)
    K = 0.5 * (p.mass * (p.vel ** 2).sum(0)).sum()
    assert K == pytest.approx(1 / 12, rel=0.05)
    assert p.mass.sum() == pytest.approx(1.0, rel=1e-12)


def test_plummer_sample_half_mass_radius():
    p = ics.plummer(1 << 14, seed=1)
    r = np.linalg.norm(p.pos, axis=0)
    assert np.median(r) == pytest.approx(1 / math.sqrt(2 ** (2 / 3) - 1), rel=0.04)


def test_reproducible_and_seeded():
    a = ics.hernquist(1000, seed=5)
    b = ics.hernquist(1000, seed=5)
    c = ics.hernquist(1000, seed=6)
    np.testing.assert_array_equal(a.pos, b.pos)
    assert not np.array_equal(a.pos, c.pos)


def test_smbh_setups():
    bh = ics.circular_bh()
    assert bh.vel[0, 1] == pytest.approx(math.sqrt((1 / 9) / 0.5))
    b = ics.central_binary()
    np.testing.assert_allclose(b.com, 0.0, atol=1e-18)
    np.testing.assert_allclose(b.com_vel, 0.0, atol=1e-18)
    rel = b.pos[0] - b.pos[1]
    vrel = b.vel[0] - b.vel[1]
    E = 0.5 * vrel @ vrel - 0.01 / np.linalg.norm(rel)
    assert -0.01 / (2 * E) == pytest.approx(0.01, rel=1e-12)        # semi-major axis
    sizes = ics.ensemble_sizes()
    assert sizes.shape == (64,) and sizes.min() >= 8192 and sizes.max() <= 524288


def test_hernquist_constants_the_paper_prints():
    """Sect. 3's model in code units (G = M = a = 1): the half-mass radius
    1 + sqrt(2) = 2.41 and the circular speed 0.28 at r = 0.1 that the paper
    quotes, from the generator's density by quadrature (not from the
    enclosed-mass formula the sampler inverts), and the sample's mass
    fraction inside the half-mass radius (truncated at u = 0.99: 0.5 / 0.99)."""
    from scipy.integrate import quad

    def mass(r):
        return quad(lambda s: 4 * math.pi * s * s * float(ics.hernquist_density(s)), 0, r, limit=200)[0]

    r_half = 1 + math.sqrt(2)
    assert mass(r_half) == pytest.approx(0.5, rel=1e-9)
    assert r_half == pytest.approx(2.41, abs=0.005)
    assert math.sqrt(mass(0.1) / 0.1) == pytest.approx(0.28, abs=0.01)
    p = ics.hernquist(1 << 16, seed=3)
    frac = float((np.linalg.norm(p.pos, axis=0) < r_half).mean())
    assert frac == pytest.approx(0.5 / 0.99, abs=0.01)
