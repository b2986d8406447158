"""Shared helpers for the GPU parity tests (inputs and comparisons only)."""
import numpy as np

import ics
import oracle


def to_dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def stars32(pos, mass):
    p32 = np.ascontiguousarray(pos, dtype=np.float32)
    m32 = np.ascontiguousarray(mass, dtype=np.float32)
    return p32, m32


def gpu_tree(ctx, p32, m32):
    import torch
    x, y, z = (to_dev(p32[a]) for a in range(3))
    m = to_dev(m32)
    ctx.build_tree(x, y, z, m)
    torch.cuda.synchronize()
    return x, y, z, m


def gpu_cells_as_oracle(view):
    """GPU cell arrays in the oracle's [ncell, 9] layout."""
    cb = view["cbox"].cpu().numpy().astype(np.int64)
    cl = view["clink"].cpu().numpy().astype(np.int64)
    par = view["cparent"].cpu().numpy().astype(np.int64)
    nch = cl[:, 1] - cl[:, 0]
    child = np.where(nch > 0, cl[:, 0], -1)
    return np.stack([cb[:, 3], cl[:, 2], cl[:, 3] - cl[:, 2], child, nch, par, cb[:, 0], cb[:, 1], cb[:, 2]], 1)


def sorted_groups(g):
    """Groups [ngroup, 8] (first, count, box lo x/y/z, box hi x/y/z) ordered by first star."""
    g = np.asarray(g, dtype=np.int64).reshape(-1, 8)
    return g[np.argsort(g[:, 0], kind="stable")]


def hernquist32(n, seed):
    w = ics.hernquist(n, seed)
    return stars32(w.pos, w.mass)


def err_stats(a, ref):
    e = oracle.rel_err(a, ref)
    return oracle.percentile(e, 0.5), oracle.percentile(e, 0.99), float(e.max())


def gpu_cell_centres(view):
    """Geometric cell centres in FP32, computed as librv does:
    lo + (o + side/2) * unit with each operation rounded once."""
    b = view["bounds"].cpu().numpy()
    cb = view["cbox"].cpu().numpy()
    lo = b[:3].astype(np.float32)
    unit = np.float32(b[3] / 2097152.0)
    half = (2.0 ** (20 - cb[:, 3].astype(np.float64))).astype(np.float32)
    out = np.empty((cb.shape[0], 3), dtype=np.float32)
    for a in range(3):
        out[:, a] = lo[a] + (cb[:, a].astype(np.float32) + half) * unit
    return out


def gpu_com(view):
    """Absolute centres of mass (FP64) from the GPU's centre-relative records."""
    g = view["cmom"].cpu().numpy().astype(np.float64)
    return gpu_cell_centres(view).astype(np.float64) + g[:, 1:4]
