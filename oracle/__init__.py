"""CPU FP64 oracle for the tree-gravity path (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package; the CUDA library never imports, links or calls it, and it shares no
code with it. The heavy loops are plain C in ``orc.c`` (built here with gcc,
OpenMP, ``-ffp-contract=off``); this module marshals numpy arrays and adds the
few steps that are one line of numpy (the leapfrog kick/drift, the energy and
momentum sums, error percentiles).

Every function cites the part of the paper it restates; the readings of the
points the paper leaves open are documented in ``orc.c``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_LOCK = threading.Lock()
_LIB = None


def build(force: bool = False) -> str:
    """Compile ``orc.c`` into ``_build/liborc.so`` (gcc, FP64, OpenMP)."""
    src = os.path.join(_HERE, "orc.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", src, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = C.CDLL(build())
            _declare(_LIB)
    return _LIB


_d = C.POINTER(C.c_double)
_f = C.POINTER(C.c_float)
_i64 = C.POINTER(C.c_int64)
_u64 = C.POINTER(C.c_uint64)


def _declare(L):
    L.orc_direct.argtypes = [C.c_int64, _d, _d, _d, _d, _d, C.c_int64, _i64, _d, _d, _d, _d, C.c_int32]
    L.orc_bounds.argtypes = [C.c_int64, _f, _f, _f, _d, _d, _d]
    L.orc_keys.argtypes = [C.c_int64, _f, _f, _f, _d, C.c_double, _u64]
    L.orc_sort.argtypes = [C.c_int64, _u64, _u64, _i64]
    L.orc_tree_build.argtypes = [C.c_int64, _f, _f, _f, _f, C.c_int32, C.c_int32]
    L.orc_tree_build.restype = C.c_void_p
    L.orc_tree_free.argtypes = [C.c_void_p]
    L.orc_tree_sizes.argtypes = [C.c_void_p, _i64]
    L.orc_tree_bounds.argtypes = [C.c_void_p, _d]
    L.orc_tree_keys.argtypes = [C.c_void_p, _u64, _i64]
    L.orc_tree_cells.argtypes = [C.c_void_p, _i64]
    L.orc_tree_moments.argtypes = [C.c_void_p, _d]
    L.orc_tree_groups.argtypes = [C.c_void_p, _i64]
    L.orc_tree_forces.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                  _f, _f, _f, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d, _i64, C.c_int64, _i64,
                                  C.c_float, _f, _f, _f, C.c_int32, _d, C.POINTER(C.c_int8)]
    L.orc_perturber.argtypes = [C.c_int32, _d, _d, C.c_int32, _d, _d, _d, _d, _d, _d, _d]
    L.orc_chain_moments.argtypes = [C.c_int32, _d, _d, _d]
    L.orc_knn.argtypes = [C.c_int64, _f, _f, _f, _f, C.c_int64, _i64]
    L.orc_knn.restype = C.c_int64
    L.orc_radius.argtypes = [C.c_int64, _f, _f, _f, _f, C.c_float, C.c_int64, _i64]
    L.orc_radius.restype = C.c_int64
    L.orc_influence.argtypes = [C.c_int64, _f, _f, _f, _f, _f, _f, _f, _f, C.c_double, C.c_int64, _d]
    L.orc_tidal.argtypes = [C.c_int64, _f, _f, _f, _f, _f, C.c_float, C.c_float, C.c_float, C.c_int64, _i64]
    L.orc_tidal.restype = C.c_int64
    L.orc_absorb.argtypes = [C.c_int64, _f, _f, _f, C.c_int32, _d, _d, C.c_int64, _i64, _d]
    L.orc_absorb.restype = C.c_int64


def _p(a, ty):
    return a.ctypes.data_as(ty)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# Direct sum
# ---------------------------------------------------------------------------
def direct(pos, mass, eps, targets=None, kind=0):
    """Direct-summation acceleration and potential (G = 1, Plummer softening,
    Sect. 3; kind = 1: spline softening of Plummer-equivalent length eps, the
    cubic-spline field with h = 2.8 eps) on ``targets`` (indices; default all)
    from all particles.

    ``pos`` (3, n) float64, ``mass`` (n,), ``eps`` scalar or (n,) where 0 marks
    an unsoftened particle (the chain centre of mass, Sect. 2/3). Pair
    softening is max(eps_i, eps_j), 0 if either is 0. Returns (acc (3, nt), pot (nt,))."""
    pos = _c(pos, np.float64)
    n = pos.shape[1]
    m = _c(mass, np.float64)
    e = _c(np.broadcast_to(np.asarray(eps, dtype=np.float64), (n,)), np.float64)
    t = np.arange(n, dtype=np.int64) if targets is None else _c(targets, np.int64)
    x, y, z = (_c(pos[a], np.float64) for a in range(3))
    out = [np.zeros(t.shape[0]) for _ in range(4)]
    lib().orc_direct(n, _p(x, _d), _p(y, _d), _p(z, _d), _p(m, _d), _p(e, _d), t.shape[0], _p(t, _i64),
                     *[_p(o, _d) for o in out], int(kind))
    return np.stack(out[:3]), out[3]


# ---------------------------------------------------------------------------
# Keys and sort
# ---------------------------------------------------------------------------
def bounds(pos32):
    """(min[3], L, scale) of FP32 positions (3, n)."""
    x, y, z = (_c(pos32[a], np.float32) for a in range(3))
    lo = np.zeros(3)
    L = C.c_double()
    s = C.c_double()
    lib().orc_bounds(x.shape[0], _p(x, _f), _p(y, _f), _p(z, _f), _p(lo, _d), C.byref(L), C.byref(s))
    return lo, L.value, s.value


def keys(pos32):
    """63-bit Morton keys of FP32 positions (3, n), unsorted, caller order."""
    x, y, z = (_c(pos32[a], np.float32) for a in range(3))
    lo, L, s = bounds(pos32)
    k = np.zeros(x.shape[0], dtype=np.uint64)
    lib().orc_keys(x.shape[0], _p(x, _f), _p(y, _f), _p(z, _f), _p(lo, _d), s, _p(k, _u64))
    return k


def stable_sort(key):
    """Stable sort of keys; returns (sorted keys, permutation: sorted slot -> index)."""
    key = _c(key, np.uint64)
    sk = np.zeros_like(key)
    perm = np.zeros(key.shape[0], dtype=np.int64)
    lib().orc_sort(key.shape[0], _p(key, _u64), _p(sk, _u64), _p(perm, _i64))
    return sk, perm


# ---------------------------------------------------------------------------
# Tree
# ---------------------------------------------------------------------------
class Tree:
    """The oracle octree of FP32 stars (positions (3, n), masses (n,)).

    Attributes after construction (numpy arrays):
      key, perm         sorted keys and sorted slot -> caller index
      cells [ncell, 9]  level, first, count, child, nchild, parent, ox, oy, oz
      moments [ncell,10] M, com x/y/z, Q xx, yy, zz, xy, xz, yz (FP64)
      groups [ngroup,8] first, count, box lo x/y/z, box hi x/y/z (grid units)
      lo, L, scale      bounding cube
    """

    def __init__(self, pos32, mass32, n_leaf: int = 16, group: int = 32):
        self.x, self.y, self.z = (_c(pos32[a], np.float32) for a in range(3))
        self.m = _c(mass32, np.float32)
        self.n = self.x.shape[0]
        self.n_leaf, self.group = n_leaf, group
        self._h = lib().orc_tree_build(self.n, _p(self.x, _f), _p(self.y, _f), _p(self.z, _f), _p(self.m, _f),
                                       n_leaf, group)
        sz = np.zeros(3, dtype=np.int64)
        lib().orc_tree_sizes(self._h, _p(sz, _i64))
        self.ncell, self.ngroup = int(sz[1]), int(sz[2])
        b = np.zeros(5)
        lib().orc_tree_bounds(self._h, _p(b, _d))
        self.lo, self.L, self.scale = b[:3].copy(), float(b[3]), float(b[4])
        self.key = np.zeros(self.n, dtype=np.uint64)
        self.perm = np.zeros(self.n, dtype=np.int64)
        lib().orc_tree_keys(self._h, _p(self.key, _u64), _p(self.perm, _i64))
        self.cells = np.zeros((self.ncell, 9), dtype=np.int64)
        lib().orc_tree_cells(self._h, _p(self.cells, _i64))
        self.moments = np.zeros((self.ncell, 10))
        lib().orc_tree_moments(self._h, _p(self.moments, _d))
        self.groups = np.zeros((self.ngroup, 8), dtype=np.int64)
        lib().orc_tree_groups(self._h, _p(self.groups, _i64))
        # FP64 copies of the stars in key order
        self.x_sorted = self.x[self.perm].astype(np.float64)
        self.y_sorted = self.y[self.perm].astype(np.float64)
        self.z_sorted = self.z[self.perm].astype(np.float64)
        self.m_sorted = self.m[self.perm].astype(np.float64)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree_free(h)
            self._h = None

    def forces(self, theta: float, eps_star: float, quadrupole: bool = True,
               extra_pos32=None, extra_mass=None, extra_eps=None, counts: bool = False, targets=None, rel=None,
               kind: int = 0, extra_quad=None, quad_skip=None):
        """Tree acceleration/potential on every star (caller order), FP64.

        Walk under the box-box opening-angle test at ``theta``; ``extra_*``
        are particles outside the tree (chain centres of mass; eps 0 =
        unsoftened) that act on the stars and each other directly and feel the
        tree through their own walk. Returns (acc (3,n), pot (n,), xacc (3,k),
        xpot (k,)[, counts (n,2) = P2P, M2P interactions]). With ``targets``
        (caller indices) only those stars are computed; the rest of the
        returned arrays is zero. With ``rel = (alpha, aref)`` the stars' groups
        use the relative opening criterion (see ``forces_rel``); groups whose
        smallest reference |a| is 0 and the extra particles use theta. ``kind``
        1: spline softening of the stars (see ``direct``; accepted cells closer
        than h = 2.8 eps act as softened monopoles). ``extra_quad`` (k, 6)
        gives each extra particle a traceless quadrupole (xx, yy, zz, xy, xz,
        yz) about its position, whose field it adds wherever it acts (a chain
        seen from outside: ``chain_moments``) except on the stars whose caller
        indices ``quad_skip`` lists (the chain's perturbers, which feel the
        resolved members through ``perturber`` instead)."""
        k = 0 if extra_mass is None else int(np.asarray(extra_mass).shape[0])
        ex = np.zeros((3, max(k, 1)), dtype=np.float32)
        xm = np.zeros(max(k, 1))
        xe = np.zeros(max(k, 1))
        if k:
            ex[:, :k] = np.asarray(extra_pos32, dtype=np.float32)
            xm[:k] = np.asarray(extra_mass, dtype=np.float64)
            xe[:k] = np.asarray(extra_eps, dtype=np.float64)
        exx, exy, exz = (_c(ex[a], np.float32) for a in range(3))
        xq = None
        if extra_quad is not None and k:
            xq = _c(np.asarray(extra_quad, dtype=np.float64).reshape(k, 6), np.float64)
        skip = None
        if quad_skip is not None:
            skip = np.zeros(max(self.n, 1), dtype=np.int8)
            skip[np.asarray(quad_skip, dtype=np.int64)] = 1
        ar = [_c(np.asarray(rel[1][a], dtype=np.float32), np.float32) for a in range(3)] if rel is not None else None
        out = [np.zeros(self.n) for _ in range(4)]
        xout = [np.zeros(max(k, 1)) for _ in range(4)]
        cnt = np.zeros((self.n, 2), dtype=np.int64) if counts else None
        lib().orc_tree_forces(self._h, float(np.float32(theta)), float(eps_star), int(quadrupole), k,
                              _p(exx, _f), _p(exy, _f), _p(exz, _f), _p(xm, _d), _p(xe, _d),
                              *[_p(o, _d) for o in out], *[_p(o, _d) for o in xout],
                              _p(cnt, _i64) if counts else None,
                              -1 if targets is None else len(targets),
                              None if targets is None else _p(_c(targets, np.int64), _i64),
                              float(np.float32(rel[0])) if rel is not None else 0.0,
                              *([_p(v, _f) for v in ar] if rel is not None else [None, None, None]), int(kind),
                              None if xq is None else _p(xq, _d),
                              None if skip is None else skip.ctypes.data_as(C.POINTER(C.c_int8)))
        res = (np.stack(out[:3]), out[3], np.stack(xout[:3])[:, :k], xout[3][:k])
        return res + (cnt,) if counts else res


    def forces_rel(self, alpha: float, eps_star: float, aref, quadrupole: bool = True, counts: bool = False,
                   targets=None, theta: float = 0.5):
        """Tree acceleration/potential (caller order, FP64) under the relative
        opening criterion (Sect. 3's "Gadget" criterion, Gadget-2 reading):
        a cell of mass M and side s at box distance d is used when
        M s^2 <= alpha |a| d^4, |a| the smallest reference magnitude of the
        group (``aref``: FP32 reference accelerations (3, n), caller order;
        magnitudes taken in FP32), and the group lies outside the cell's box
        grown by s/10 per side; a group whose smallest |a| is 0 uses theta.
        Returns (acc (3,n), pot (n,)[, counts (n,2)])."""
        r = self.forces(theta, eps_star, quadrupole, counts=counts, targets=targets, rel=(alpha, aref))
        return (r[0], r[1], r[4]) if counts else (r[0], r[1])


# ---------------------------------------------------------------------------
# Chain / perturber coupling (Sect. 2, Eq. 3)
# ---------------------------------------------------------------------------
def chain_moments(chain_mass, chain_pos):
    """Total mass, centre of mass and traceless quadrupole of a chain about its
    centre of mass, Q_ab = sum_k m_k (3 d_a d_b - |d|^2 delta_ab), d = x_k -
    com (the two-term expansion of Sect. 1 applied to the chain's members).
    Returns dict M, com (3,), Q (6,) = (xx, yy, zz, xy, xz, yz)."""
    cm = _c(chain_mass, np.float64)
    cx = _c(chain_pos, np.float64).reshape(-1)
    out = np.zeros(10)
    lib().orc_chain_moments(cm.shape[0], _p(cm, _d), _p(cx, _d), _p(out, _d))
    return {"M": float(out[0]), "com": out[1:4].copy(), "Q": out[4:10].copy()}


def perturber(chain_mass, chain_pos, pert_mass, pert_pos):
    """Unsoftened FP64 couplings of a chain (k members, pos (k,3)) and its
    perturbers (p, pos (p,3)), Sect. 2 and Eq. 3. Returns dict with a_pert
    (p,3), pot_pert (p,), a_chain (k,3), pot_chain (k,), corr (3,) = Eq. 3
    correction, sub (3,) = perturbers' direct terms on the centre-of-mass
    particle, corr_pot, sub_pot, com (3,), M."""
    cm = _c(chain_mass, np.float64)
    cx = _c(chain_pos, np.float64).reshape(-1)
    pm = _c(pert_mass, np.float64)
    px = _c(pert_pos, np.float64).reshape(-1)
    nch, npt = cm.shape[0], pm.shape[0]
    ap = np.zeros(3 * max(npt, 1))
    pp = np.zeros(max(npt, 1))
    ac = np.zeros(3 * max(nch, 1))
    pc = np.zeros(max(nch, 1))
    out = np.zeros(12)
    lib().orc_perturber(nch, _p(cm, _d), _p(cx, _d), npt, _p(pm, _d), _p(px, _d), _p(ap, _d), _p(pp, _d),
                        _p(ac, _d), _p(pc, _d), _p(out, _d))
    return {"a_pert": ap[:3 * npt].reshape(npt, 3), "pot_pert": pp[:npt],
            "a_chain": ac[:3 * nch].reshape(nch, 3), "pot_chain": pc[:nch],
            "corr": out[0:3].copy(), "sub": out[3:6].copy(), "corr_pot": float(out[6]),
            "sub_pot": float(out[7]), "com": out[8:11].copy(), "M": float(out[11])}


def knn(pos32, centre32, k):
    """Indices of the k stars nearest to centre (FP32 distances, ties by index)."""
    x, y, z = (_c(pos32[a], np.float32) for a in range(3))
    c = _c(centre32, np.float32)
    out = np.zeros(max(k, 1), dtype=np.int64)
    got = lib().orc_knn(x.shape[0], _p(x, _f), _p(y, _f), _p(z, _f), _p(c, _f), k, _p(out, _i64))
    return out[:got]


def radius(pos32, centre32, r2_32):
    """Indices (ascending) of stars with FP32 squared distance below r2."""
    x, y, z = (_c(pos32[a], np.float32) for a in range(3))
    c = _c(centre32, np.float32)
    n = x.shape[0]
    out = np.zeros(max(n, 1), dtype=np.int64)
    got = lib().orc_radius(n, _p(x, _f), _p(y, _f), _p(z, _f), _p(c, _f), np.float32(r2_32), n, _p(out, _i64))
    return out[:got]


def a_hard(m1, m2, r_infl):
    """Semi-major axis at which an SMBH binary becomes hard (Eq. 13, Sect. 5):
    a_hard = mu / (M1 + M2) * r_infl / 4 with the reduced mass
    mu = (1/M1 + 1/M2)^-1 and r_infl the influence radius of the pair. The
    method starts its chain with a radius of a few a_hard (Sect. 5). FP64."""
    m1, m2, r_infl = float(m1), float(m2), float(r_infl)
    mu = 1.0 / (1.0 / m1 + 1.0 / m2)
    return mu / (m1 + m2) * r_infl / 4.0


def chain_start_radius(pos32, vel32, mass32, centre32, m_bh, alpha, beta, eps, n_sigma=50):
    """The chain's start radius of Eq. 1, r_chain,0 = max(alpha r_infl, beta eps),
    r_infl = min(r(<2 M_bh), G M_bh / sigma^2), sigma the velocity dispersion
    of the n_sigma nearest stars (see orc_influence for the exact rule).
    Returns dict r2m, sigma, r_sigma, r_infl, r_chain0."""
    x, y, z = (_c(pos32[a], np.float32) for a in range(3))
    vx, vy, vz = (_c(vel32[a], np.float32) for a in range(3))
    m = _c(mass32, np.float32)
    c = _c(centre32, np.float32)
    out = np.zeros(3)
    lib().orc_influence(x.shape[0], *[_p(a, _f) for a in (x, y, z, vx, vy, vz, m, c)], float(m_bh), int(n_sigma),
                        _p(out, _d))
    r_infl = min(out[0], out[2])
    return {"r2m": out[0], "sigma": out[1], "r_sigma": out[2], "r_infl": r_infl,
            "r_chain0": max(alpha * r_infl, beta * eps)}


def tidal(pos32, mass32, centre32, mchain32, gamma, rcrit):
    """Indices (ascending) of the stars that pass the tidal perturber
    criterion of Eq. 2, r_j < (2 m_j / (gamma M))^(1/3) r_crit, decided in FP64
    without a cube root on the FP32 squared distances."""
    x, y, z = (_c(pos32[a], np.float32) for a in range(3))
    m = _c(mass32, np.float32)
    c = _c(centre32, np.float32)
    n = x.shape[0]
    out = np.zeros(max(n, 1), dtype=np.int64)
    got = lib().orc_tidal(n, _p(x, _f), _p(y, _f), _p(z, _f), _p(m, _f), _p(c, _f), np.float32(mchain32),
                          np.float32(gamma), np.float32(rcrit), n, _p(out, _i64))
    return out[:got]


def absorb(pos32, chain_mass, chain_pos):
    """Eq. 4: indices (ascending) of the stars closer to the chain's centre of
    mass than the chain radius (its largest member distance), decided in FP64
    on squared distances (see orc_absorb). Returns (idx, r_chain)."""
    x, y, z = (_c(pos32[a], np.float32) for a in range(3))
    cm = _c(chain_mass, np.float64)
    cx = _c(chain_pos, np.float64).reshape(-1)
    n = x.shape[0]
    out = np.zeros(max(n, 1), dtype=np.int64)
    o2 = np.zeros(2)
    got = lib().orc_absorb(n, _p(x, _f), _p(y, _f), _p(z, _f), cm.shape[0], _p(cm, _d), _p(cx, _d), n, _p(out, _i64),
                           _p(o2, _d))
    return out[:got], float(o2[0])


def chain_escape(mass, pos, vel, massive, designated, r_chain0, gamma, n_absorbing):
    """Escape from the chain (Eq. 5) and the membership rules around it
    (Sect. 2, Sect. 3), FP64 on the members in index order:
      - c, v_c: the members' centre-of-mass position and velocity;
      - member k recedes if (d . u) > 0 with d = x_k - c, u = v_k - v_c, summed
        (d_x u_x + d_y u_y) + d_z u_z, and escapes if also
        (d_x d_x + d_y d_y) + d_z d_z > r_esc^2, r_esc = gamma r_chain0 (Eq. 5);
      - absorption goes first: while perturbers are being absorbed
        (n_absorbing > 0) escapes wait, unless the chain radius (largest member
        distance) exceeds the escape radius by more than 5 %;
      - the chain ends if fewer than 2 members remain, or if the designated
        massive member escapes and no other massive member remains; if another
        does, the most massive remaining massive member (lowest index on ties)
        becomes the designated one.
    Returns dict escape (bool array), terminate, designated, r_chain, r_escape."""
    m = np.asarray(mass, np.float64)
    x = np.asarray(pos, np.float64).reshape(-1, 3)
    v = np.asarray(vel, np.float64).reshape(-1, 3)
    k = m.shape[0]
    M = 0.0
    c = [0.0, 0.0, 0.0]
    vc = [0.0, 0.0, 0.0]
    for i in range(k):
        M += m[i]
        for a in range(3):
            c[a] += m[i] * x[i, a]
            vc[a] += m[i] * v[i, a]
    for a in range(3):
        c[a] = c[a] / M if M > 0 else 0.0
        vc[a] = vc[a] / M if M > 0 else 0.0
    r_esc = gamma * r_chain0
    re2 = r_esc * r_esc
    rc2 = 0.0
    cand = np.zeros(k, dtype=bool)
    for i in range(k):
        d = [x[i, a] - c[a] for a in range(3)]
        u = [v[i, a] - vc[a] for a in range(3)]
        d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
        du = (d[0] * u[0] + d[1] * u[1]) + d[2] * u[2]
        rc2 = max(rc2, d2)
        cand[i] = d2 > re2 and du > 0.0
    grown = 1.05 * r_esc
    esc = cand if (n_absorbing <= 0 or rc2 > grown * grown) else np.zeros(k, dtype=bool)
    terminate = int(k - int(esc.sum()) < 2)
    des = int(designated)
    if esc[des]:
        rest = [i for i in range(k) if massive[i] and not esc[i]]
        if rest:
            des = max(rest, key=lambda i: (m[i], -i))
        else:
            terminate = 1
    return {"escape": esc, "terminate": terminate, "designated": des, "r_chain": math.sqrt(rc2), "r_escape": r_esc}


# ---------------------------------------------------------------------------
# Integration and diagnostics
# ---------------------------------------------------------------------------
def energy(pos, vel, mass, pot):
    """FP64 totals (Sect. 3/4 energy diagnostic): E_kin = sum m v^2/2,
    E_pot = sum m phi / 2, momentum P = sum m v, angular momentum
    L = sum m x cross v. Exactly rounded sums (math.fsum)."""
    import math
    pos, vel = np.asarray(pos, np.float64), np.asarray(vel, np.float64)
    m, p = np.asarray(mass, np.float64), np.asarray(pot, np.float64)
    ek = math.fsum(0.5 * m * (vel * vel).sum(0))
    ep = math.fsum(0.5 * m * p)
    P = [math.fsum(m * vel[a]) for a in range(3)]
    Lv = np.cross(pos.T, vel.T).T
    Lm = [math.fsum(m * Lv[a]) for a in range(3)]
    return {"ekin": ek, "epot": ep, "etot": ek + ep, "P": np.array(P), "L": np.array(Lm)}


def kdk(pos, vel, acc, dt, force_fn, nsteps=1):
    """Kick-drift-kick leapfrog with a global step (the integrator used here
    in place of the paper's DKD block steps): v += a dt/2; x += v dt;
    a = force_fn(x); v += a dt/2. Returns (pos, vel, acc)."""
    pos, vel, acc = pos.copy(), vel.copy(), acc.copy()
    for _ in range(nsteps):
        vel = vel + 0.5 * dt * acc
        pos = pos + dt * vel
        acc = force_fn(pos)
        vel = vel + 0.5 * dt * acc
    return pos, vel, acc


def block_levels(acc32, vel32, level, n, max_level, dt_max, tau_acc, tau_vel, eps, start=False):
    """New time-step levels (block time steps, Sect. 2; criteria of Sect. 3)
    of the stars active at substep n: dt = min(tau_acc sqrt(eps / |a|),
    tau_vel eps / |v|) in FP64 from the FP32 components (sums in the order
    (x x + y y) + z z), level = the smallest l in [0, L] with dt_max 2^-l <= dt;
    unless start, a coarser level only where its step boundary is at n (else
    the coarsest such level between). Inactive stars keep theirs."""
    a = np.asarray(acc32, dtype=np.float32).astype(np.float64)
    v = np.asarray(vel32, dtype=np.float32).astype(np.float64)
    tau_acc, tau_vel, eps = (float(np.float32(t)) for t in (tau_acc, tau_vel, eps))
    L = int(max_level)
    level = np.asarray(level, dtype=np.int64).copy()
    out = level.copy()
    for i in range(level.shape[0]):
        if not start and n % (1 << (L - level[i])) != 0:
            continue
        a2 = (a[0, i] * a[0, i] + a[1, i] * a[1, i]) + a[2, i] * a[2, i]
        v2 = (v[0, i] * v[0, i] + v[1, i] * v[1, i]) + v[2, i] * v[2, i]
        dt = math.inf
        if a2 > 0:
            dt = tau_acc * math.sqrt(eps / math.sqrt(a2))
        if v2 > 0:
            dt = min(dt, (tau_vel * eps) / math.sqrt(v2))
        lv, step = 0, float(dt_max)
        while lv < L and step > dt:
            step *= 0.5
            lv += 1
        if not start:
            while lv < level[i] and n % (1 << (L - lv)) != 0:
                lv += 1
        out[i] = lv
    return out


def block_kdk(pos, vel, force_fn, level, max_level, dt_max, nsub, adapt=None):
    """Block time steps in kick-drift-kick form (Sect. 2: stars on a hierarchy
    of step levels), FP64. Star i has step dt_max / 2^level[i]; a substep of
    dt_min = dt_max / 2^L drifts every star; the stars whose step ends then
    (substep count a multiple of 2^(L - level)) take the force of the new
    positions (force_fn(pos, active) -> acc (3, n), only the active columns
    are used), their closing half kick, a new level (adapt = (tau_acc,
    tau_vel, eps): block_levels on the FP32-rounded acc and velocity; None:
    fixed) and the opening half kick. Starts with forces on every star, levels
    and opening kicks. Returns (pos, vel, acc, level, active updates)."""
    pos, vel = np.array(pos, dtype=np.float64), np.array(vel, dtype=np.float64)
    level = np.asarray(level, dtype=np.int64).copy()
    L = int(max_level)
    n_all = pos.shape[1]
    acc = np.asarray(force_fn(pos, np.ones(n_all, bool)), dtype=np.float64)

    def new_levels(lv, n, start):
        if adapt is None:
            return lv
        return block_levels(acc.astype(np.float32), vel.astype(np.float32), lv, n, L, dt_max, *adapt, start=start)

    level = new_levels(level, 0, True)
    vel = vel + acc * (0.5 * dt_max * 2.0 ** -level)
    updates = 0
    dt_min = dt_max * 2.0 ** -L
    for n in range(1, nsub + 1):
        pos = pos + vel * dt_min
        active = (n % (1 << (L - level))) == 0
        updates += int(active.sum())
        a_new = np.asarray(force_fn(pos, active), dtype=np.float64)
        acc[:, active] = a_new[:, active]
        vel[:, active] += acc[:, active] * (0.5 * dt_max * 2.0 ** -level[active])
        level = new_levels(level, n, False)
        vel[:, active] += acc[:, active] * (0.5 * dt_max * 2.0 ** -level[active])
    return pos, vel, acc, level, updates


def rel_err(a, ref):
    """Per-particle relative error |a - ref| / |ref| of (3, n) vectors."""
    a, ref = np.asarray(a, np.float64), np.asarray(ref, np.float64)
    return np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)


def percentile(e, p):
    """Nearest-rank percentile: sorted ascending, index ceil(p n) - 1."""
    import math
    s = np.sort(np.asarray(e, np.float64))
    if s.size == 0:
        return float("nan")
    return float(s[max(0, math.ceil(p * s.size) - 1)])


# ---------------------------------------------------------------------------
# Learned cell-force correction (not in the paper): features, targets, MLP
# ---------------------------------------------------------------------------
MLP_IN, MLP_IN_PAD, MLP_HID, MLP_OUT, MLP_OUT_PAD = 14, 16, 64, 3, 8


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64:
    the float32 value's low 16 bits are rounded away."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _sym3(Q6):
    return np.array([[Q6[0], Q6[3], Q6[4]], [Q6[3], Q6[1], Q6[5]], [Q6[4], Q6[5], Q6[2]]])


def cell_octupole(tree, cell):
    """Traceless third moment of a cell about its centre of mass, the term the
    quadrupole expansion leaves out (the next order of Sect. 1's expansion).
    A leaf: from its stars, O_abc = sum_j m_j d_a d_b d_c (d = x_j - com). An
    internal cell: from its children k (centre-of-mass offsets D_k, masses M_k,
    traceless quadrupoles Q_k), O_abc = sum_k [M_k D_a D_b D_c + (D_a Q_k,bc +
    D_b Q_k,ac + D_c Q_k,ab) / 3], the children's own third moments left out
    (the trace parts of the children's second moments drop out of the
    traceless part). Then O^T_abc = O_abc - (delta_ab t_c + delta_ac t_b +
    delta_bc t_a) / 5 with t_a = O_akk. Returns O^T (3, 3, 3)."""
    c = tree.cells[cell]
    com = tree.moments[cell, 1:4]
    O = np.zeros((3, 3, 3))
    if c[4] == 0:      # a leaf: its stars
        first, count = c[1], c[2]
        d = np.stack([tree.x_sorted[first:first + count], tree.y_sorted[first:first + count],
                      tree.z_sorted[first:first + count]]) - com[:, None]
        O = np.einsum("j,aj,bj,cj->abc", tree.m_sorted[first:first + count], d, d, d)
    else:
        for k in range(c[3], c[3] + c[4]):
            mk = tree.moments[k]
            Mk, D, Qk = mk[0], mk[1:4] - com, _sym3(mk[4:10])
            O += Mk * np.einsum("a,b,c->abc", D, D, D)
            O += (np.einsum("a,bc->abc", D, Qk) + np.einsum("b,ac->abc", D, Qk) + np.einsum("c,ab->abc", D, Qk)) / 3.0
    t = np.einsum("akk->a", O)
    I = np.eye(3)
    return O - (np.einsum("ab,c->abc", I, t) + np.einsum("ac,b->abc", I, t) + np.einsum("bc,a->abc", I, t)) / 5.0


def cell_features(tree, cell, x, eps):
    """Features of one (target at x, accepted cell) pair: r/|r| (3), s/|r|,
    eps/|r|, Q/(M s^2) (xx, yy, zz, xy, xz, yz), and the octupole term of the
    cell's acceleration in the output's units (3): the next order of Sect. 1's
    expansion, whose potential is -(5/2) O^T(r^, r^, r^) / |r|^4 with O^T the
    traceless third moment (cell_octupole), has the acceleration
    (5/2) [3 O^T(., r^, r^) - 7 r^ O^T(r^, r^, r^)] / |r|^5, and times |r|^2 / M
    that is (5/2) [3 v - 7 r^ (r^ . v)] / (M |r|^3) with v = O^T(., r^, r^).
    r = x - com, s the cell side; also returns the normalisation M/|r|^2 of the
    output."""
    mo = tree.moments[cell]
    M, com, Q = mo[0], mo[1:4], mo[4:10]
    lev = tree.cells[cell, 0]
    s = tree.L / 2.0 ** lev
    r = np.asarray(x, dtype=np.float64) - com
    d = np.linalg.norm(r)
    rh = r / d
    v = np.einsum("abc,b,c->a", cell_octupole(tree, cell), rh, rh)
    g = 2.5 * (3.0 * v - 7.0 * rh * (rh @ v)) / (M * d ** 3)
    f = np.concatenate([rh, [s / d, eps / d], Q / (M * s * s), g])
    return f, M / (d * d)


def cell_residual(tree, cell, x, eps):
    """Exact softened force of the cell's stars on x minus the cell's softened
    monopole + quadrupole force (the quantity the network learns)."""
    c = tree.cells[cell]
    first, count = c[1], c[2]
    xs = np.stack([tree.x_sorted[first:first + count], tree.y_sorted[first:first + count],
                   tree.z_sorted[first:first + count]])
    ms = tree.m_sorted[first:first + count]
    dx = xs - np.asarray(x, dtype=np.float64)[:, None]
    r2 = (dx * dx).sum(0) + eps * eps
    exact = (ms * r2 ** -1.5 * dx).sum(1)
    mo = tree.moments[cell]
    M, com = mo[0], mo[1:4]
    q = mo[4:10]
    Q = np.array([[q[0], q[3], q[4]], [q[3], q[1], q[5]], [q[4], q[5], q[2]]])
    r = np.asarray(x, dtype=np.float64) - com
    rho2 = r @ r + eps * eps
    rinv = rho2 ** -0.5
    Qr = Q @ r
    rqr = r @ Qr
    quad = -M * r * rinv ** 3 + Qr * rinv ** 5 - 2.5 * rqr * r * rinv ** 7
    return exact - quad


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def mlp_forward(params, X, rounding=True):
    """Forward pass in FP64 with the rounding points of the BF16 tensor-core
    path: inputs, weights and hidden activations rounded to bfloat16, biases
    and sums exact (rounding=False: plain FP64 everywhere). params: W1 (16,64),
    b1 (64,), W2 (64,64), b2, W3 (64,8), b3 (8,) (padded rows/columns zero).
    Returns (Y (n,3), cache)."""
    rnd = bf16_round if rounding else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3 = (rnd(params[k]) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (np.asarray(params[k], np.float64) for k in ("b1", "b2", "b3"))
    X0 = rnd(X)
    Z1 = X0 @ W1 + b1
    H1 = rnd(silu(Z1))
    Z2 = H1 @ W2 + b2
    H2 = rnd(silu(Z2))
    Y = H2 @ W3 + b3
    return Y[:, :MLP_OUT], dict(X0=X0, Z1=Z1, H1=H1, Z2=Z2, H2=H2, W2=W2, W3=W3)


def mlp_loss_grad(params, X, T, rounding=True):
    """Mean squared error over the batch and the 3 outputs, and its analytic
    gradient with respect to every parameter (straight-through the bfloat16
    roundings)."""
    Y, c = mlp_forward(params, X, rounding)
    n = X.shape[0]
    D = Y - T
    loss = float((D * D).sum() / (n * MLP_OUT))
    dY = np.zeros((n, MLP_OUT_PAD))
    dY[:, :MLP_OUT] = 2.0 * D / (n * MLP_OUT)
    g = {}
    g["W3"] = c["H2"].T @ dY
    g["b3"] = dY.sum(0)
    dZ2 = (dY @ c["W3"].T) * silu_grad(c["Z2"])
    g["W2"] = c["H1"].T @ dZ2
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ c["W2"].T) * silu_grad(c["Z1"])
    g["W1"] = c["X0"].T @ dZ1
    g["b1"] = dZ1.sum(0)
    return loss, g


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of FP64 master parameters in place;
    state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k], dtype=np.float64))
        v = state.setdefault("v_" + k, np.zeros_like(params[k], dtype=np.float64))
        g = grads[k]
        m[...] = b1 * m + (1 - b1) * g
        v[...] = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


# ---------------------------------------------------------------------------
# Training loop of the network (not in the paper): seeded minibatches + Adam
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 output for the counter value x (Steele, Lea & Flood 2014):
    z = x + 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds and a final
    xor-shift, all modulo 2^64 (Python integers)."""
    z = (int(x) + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def minibatch_rows(seed, step, batch, n):
    """Rows of minibatch `step`: row i is floor(h n / 2^64) with
    h = splitmix64(seed + step * batch + i) (64-bit wrap-around)."""
    return np.array([(splitmix64((int(seed) + int(step) * int(batch) + i) & _M64) * int(n)) >> 64
                     for i in range(batch)], dtype=np.int64)


def mlp_train(params, X, T, steps, batch, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, seed=0, rounding=True):
    """Adam on minibatches drawn by minibatch_rows: for each step the loss and
    analytic gradient of mlp_loss_grad on the drawn rows, then adam_step.
    Returns (losses, params) with params updated (FP64)."""
    state, losses = {}, []
    params = {k: np.array(v, dtype=np.float64) for k, v in params.items()}
    for k in range(steps):
        rows = minibatch_rows(seed, k, batch, X.shape[0])
        loss, g = mlp_loss_grad(params, X[rows], T[rows], rounding)
        losses.append(loss)
        params = adam_step(params, g, state, lr, b1, b2, eps)
    return losses, params
