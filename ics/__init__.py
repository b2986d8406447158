"""Seeded synthetic initial conditions for the tree-gravity path.

This module is shared by the GPU path's tests/bench and by the CPU oracle's
tests. It holds only the *inputs*: samples of the stellar systems the paper
simulates (Sect. 3: Hernquist spheres of unit mass and scale radius, G = 1,
equal-mass stars; SMBHs on circular orbits or as a bound pair) and of a
Plummer sphere. None of the gravity method's arithmetic (keys, tree,
multipoles, forces, integration) is here.

Random numbers come from numpy's Philox4x32-10 counter-based bit generator
(Salmon et al. 2011), seeded per workload, so a given seed gives the same
samples on x86_64 and aarch64.

All arrays are float64; callers that feed an FP32 kernel cast them once and
give the *same* cast values to the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Particles", "Chain", "Workload", "rng", "plummer", "hernquist",
    "hernquist_df", "hernquist_density", "hernquist_potential",
    "circular_bh", "central_binary", "plummer_workload", "hernquist_bh_workload",
    "hernquist_binary_workload", "ensemble_sizes", "subsample",
]


def rng(seed: int) -> np.random.Generator:
    """Philox4x32-10 generator for ``seed`` (platform independent)."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


@dataclass
class Particles:
    """Equal-mass field stars, FP64. ``pos``/``vel`` are (3, n)."""
    pos: np.ndarray
    vel: np.ndarray
    mass: np.ndarray

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


@dataclass
class Chain:
    """A regularised subsystem (one SMBH, or an SMBH pair), FP64.

    ``pos``/``vel`` are (k, 3). The chain's centre of mass is the particle the
    tree code sees (Sect. 2)."""
    mass: np.ndarray
    pos: np.ndarray
    vel: np.ndarray

    @property
    def total_mass(self) -> float:
        return float(self.mass.sum())

    @property
    def com(self) -> np.ndarray:
        return (self.mass[:, None] * self.pos).sum(0) / self.mass.sum()

    @property
    def com_vel(self) -> np.ndarray:
        return (self.mass[:, None] * self.vel).sum(0) / self.mass.sum()


@dataclass
class Workload:
    name: str
    stars: Particles
    chain: Chain | None
    eps_star: float
    theta: float
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# Plummer sphere, G = M = b = 1 (Aarseth, Henon & Wielen 1974 sampling)
# --------------------------------------------------------------------------
def plummer(n: int, seed: int, umax: float = 0.999) -> Particles:
    """Plummer sphere of unit mass and unit scale length.

    Radius from the inverse cumulative mass M(<r) = r^3/(1+r^2)^{3/2}
    (u drawn in (0, umax]), isotropic directions, speed q*v_esc with q drawn
    by von Neumann rejection from q^2 (1-q^2)^{7/2}, v_esc = sqrt(2)(1+r^2)^{-1/4}.
    The sample is shifted to its centre-of-mass frame."""
    g = rng(seed)
    u = g.uniform(0.0, 1.0, n) * umax
    u = np.where(u <= 0.0, umax * 1e-12, u)
    r = 1.0 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    pos = _isotropic(g, n) * r
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = g.uniform(0.0, 1.0, todo.size)
        yy = g.uniform(0.0, 0.1, todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    vel = _isotropic(g, n) * (q * vesc)
    mass = np.full(n, 1.0 / n)
    pos -= pos.mean(axis=1, keepdims=True)
    vel -= vel.mean(axis=1, keepdims=True)
    return Particles(pos, vel, mass)


def _isotropic(g: np.random.Generator, n: int) -> np.ndarray:
    cz = g.uniform(-1.0, 1.0, n)
    ph = g.uniform(0.0, 2.0 * math.pi, n)
    sz = np.sqrt(1.0 - cz * cz)
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz])


# --------------------------------------------------------------------------
# Hernquist (Dehnen gamma = 1) sphere, G = M = a = 1 (Sect. 3)
# --------------------------------------------------------------------------
def hernquist_density(r):
    """rho(r) = M a / (2 pi r (r + a)^3) with M = a = 1."""
    r = np.asarray(r, dtype=np.float64)
    return 1.0 / (2.0 * math.pi * r * (1.0 + r) ** 3)


def hernquist_potential(r):
    """Relative potential psi(r) = -Phi(r) = G M / (r + a) with G = M = a = 1."""
    return 1.0 / (1.0 + np.asarray(r, dtype=np.float64))


def hernquist_df(e):
    """Isotropic distribution function f(E) of the Hernquist model.

    ``e`` is the relative (binding) energy, 0 <= e <= 1 in units G = M = a = 1.
    Closed form of Hernquist (1990, ApJ 356, 359): with q = sqrt(e),
    f = [3 asin q + q sqrt(1-q^2) (1-2q^2)(8q^4-8q^2-3)] / (sqrt(2) (2 pi)^3 (1-q^2)^{5/2}).
    The tests check it against the density it must reproduce."""
    e = np.clip(np.asarray(e, dtype=np.float64), 0.0, 1.0 - 1e-15)
    q = np.sqrt(e)
    q2 = q * q
    num = 3.0 * np.arcsin(q) + q * np.sqrt(1.0 - q2) * (1.0 - 2.0 * q2) * (8.0 * q2 * q2 - 8.0 * q2 - 3.0)
    return num / (math.sqrt(2.0) * (2.0 * math.pi) ** 3 * (1.0 - q2) ** 2.5)


def hernquist(n: int, seed: int, umax: float = 0.99, chunk: int = 1 << 19) -> Particles:
    """Equal-mass Hernquist sphere, unit total mass and scale radius.

    Radii from the inverse cumulative mass M(<r) = r^2/(1+r)^2 with the
    enclosed-mass fraction u drawn in [0, umax] (truncation at
    r_max = sqrt(umax)/(1-sqrt(umax)), about 99 for umax = 0.99); the star
    mass is 1/n so the truncated sample still has unit mass. Speeds are drawn
    from the isotropic distribution function of the untruncated model,
    p(v | r) ~ v^2 f(psi(r) - v^2/2), by rejection under a per-star bound
    (1.25 x the maximum on a 48-point grid). Directions are isotropic."""
    g = rng(seed)
    u = g.uniform(0.0, 1.0, n) * umax
    s = np.sqrt(u)
    r = s / (1.0 - s)
    pos = _isotropic(g, n) * r
    speed = np.empty(n)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        speed[lo:hi] = _hernquist_speeds(g, r[lo:hi])
    vel = _isotropic(g, n) * speed
    mass = np.full(n, 1.0 / n)
    return Particles(pos, vel, mass)


def _hernquist_speeds(g: np.random.Generator, r: np.ndarray) -> np.ndarray:
    psi = hernquist_potential(r)
    vesc = np.sqrt(2.0 * psi)
    grid = (np.arange(1, 49) - 0.5) / 48.0                        # fractions of v_esc
    vg = vesc[:, None] * grid[None, :]
    gmax = (vg * vg * hernquist_df(psi[:, None] - 0.5 * vg * vg)).max(axis=1) * 1.25
    out = np.empty(r.shape[0])
    todo = np.arange(r.shape[0])
    while todo.size:
        v = g.uniform(0.0, 1.0, todo.size) * vesc[todo]
        y = g.uniform(0.0, 1.0, todo.size) * gmax[todo]
        ok = y < v * v * hernquist_df(psi[todo] - 0.5 * v * v)
        out[todo[ok]] = v[ok]
        todo = todo[~ok]
    return out


# --------------------------------------------------------------------------
# SMBHs
# --------------------------------------------------------------------------
def circular_bh(m_bh: float = 0.005, r: float = 0.5) -> Chain:
    """One SMBH on a circular orbit of radius r in the Hernquist potential of
    the stars: position (r,0,0), velocity (0, sqrt(M(<r)/r), 0), M(<r) = r^2/(1+r)^2."""
    menc = r * r / (1.0 + r) ** 2
    v = math.sqrt(menc / r)
    return Chain(np.array([m_bh]), np.array([[r, 0.0, 0.0]]), np.array([[0.0, v, 0.0]]))


def central_binary(m: float = 0.005, a: float = 0.01, e: float = 0.1) -> Chain:
    """Equal-mass SMBH pair with semi-major axis a and eccentricity e, centre of
    mass at rest at the origin, started at apocentre along x (separation
    a(1+e)) with relative speed sqrt(G M_b (1-e) / (a (1+e))) along y."""
    sep = a * (1.0 + e)
    vrel = math.sqrt(2.0 * m * (1.0 - e) / (a * (1.0 + e)))
    pos = np.array([[0.5 * sep, 0.0, 0.0], [-0.5 * sep, 0.0, 0.0]])
    vel = np.array([[0.0, 0.5 * vrel, 0.0], [0.0, -0.5 * vrel, 0.0]])
    return Chain(np.array([m, m]), pos, vel)


# --------------------------------------------------------------------------
# Named workloads (the shapes the paper's runs have)
# --------------------------------------------------------------------------
def plummer_workload(n: int = 4096, seed: int = 1) -> Workload:
    """Plummer sphere N=4096, eps=0.01, theta=0.5; no SMBH."""
    return Workload(f"plummer_n{n}", plummer(n, seed), None, 0.01, 0.5,
                    {"dt": 1e-3, "nsteps": 100, "seed": seed})


def hernquist_bh_workload(n: int = 1 << 20, seed: int = 2) -> Workload:
    """Hernquist sphere with one SMBH (m=0.005) on a circular orbit at r=0.5;
    eps_star=0.005; stars within 0.02 of the SMBH are its FP64 perturbers."""
    return Workload(f"hernquist_bh_n{n}", hernquist(n, seed), circular_bh(), 0.005, 0.5,
                    {"pert_radius": 0.02, "dt": 1e-3, "seed": seed})


def hernquist_binary_workload(n: int = 1 << 22, seed: int = 3) -> Workload:
    """Hernquist sphere with a central SMBH pair (a=0.01, e=0.1, m=0.005 each);
    the 256 nearest stars to the pair's centre of mass are its perturbers."""
    return Workload(f"hernquist_binary_n{n}", hernquist(n, seed), central_binary(), 0.005, 0.5,
                    {"pert_k": 256, "dt": 1e-3, "seed": seed})


def ensemble_sizes(members: int = 64, lo: int = 8192, hi: int = 524288, seed: int = 4) -> np.ndarray:
    """Member sizes log-uniform in [lo, hi] (the paper's N-dependence runs)."""
    g = rng(seed)
    return np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), members))).astype(np.int64)


def subsample(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices of range(n), sorted, seeded."""
    k = min(k, n)
    return np.sort(rng(seed).choice(n, size=k, replace=False)).astype(np.int64)


def ensemble_workload(members: int = 64, lo: int = 8192, hi: int = 524288, seed: int = 4,
                      sizes: np.ndarray | None = None) -> dict:
    """Ensemble of independent Hernquist realisations of uneven N (log-uniform
    sizes), each with a central SMBH pair (a = 0.01, e = 0.1, m = 0.005 each),
    stored one after another. Member k uses seed 1000 + k. Returns a dict with
    pos/vel (3, N), mass (N,), offsets (members + 1,), chain_m (2 members,),
    chain_x/chain_v (2 members, 3)."""
    if sizes is None:
        sizes = ensemble_sizes(members, lo, hi, seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    pos, vel, mass = [], [], []
    for k, n in enumerate(sizes):
        p = hernquist(int(n), 1000 + k)
        pos.append(p.pos)
        vel.append(p.vel)
        mass.append(p.mass)
    b = central_binary()
    m = len(sizes)
    return {"pos": np.concatenate(pos, 1), "vel": np.concatenate(vel, 1), "mass": np.concatenate(mass),
            "offsets": np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64), "sizes": sizes,
            "chain_m": np.tile(b.mass, m), "chain_x": np.tile(b.pos, (m, 1)), "chain_v": np.tile(b.vel, (m, 1))}
