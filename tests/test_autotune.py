"""Autotuner: cache keys and candidate grid on the host; on the GPU, a tuned
choice is one of the candidates, is the fastest of its table, and is reused
from the cache."""
import os

import numpy as np
import pytest

import ics


def test_cache_key_and_grid():
    from paper_1507_01009_gb300 import autotune as at
    assert at.bucket(1) == 0 and at.bucket(1024) == 10 and at.bucket(1025) == 11
    k1 = at.cache_key("GB300", 1 << 20, 1, 0.5, True)
    k2 = at.cache_key("GB300", (1 << 20) - 5, 1, 0.5, True)
    assert k1 == k2 and k1 != at.cache_key("GB300", 1 << 20, 64, 0.5, True)
    grid = at.candidates()
    assert len(grid) == len(at.GRID_GROUP) * len(at.GRID_LEAF) * len(at.GRID_TILE)
    assert all(c["tile"] % 32 == 0 and c["group"] <= 64 for c in grid)


def test_cache_roundtrip(tmp_path):
    from paper_1507_01009_gb300 import autotune as at
    p = str(tmp_path / "a.json")
    at.save_cache({"k": {"config": {"group": 32}, "table": []}}, p)
    assert at.load_cache(p)["k"]["config"]["group"] == 32
    assert at.load_cache(str(tmp_path / "missing.json")) == {}


@pytest.mark.gpu
def test_autotune_picks_fastest_and_caches(tmp_path):
    import torch
    from paper_1507_01009_gb300 import autotune as at
    w = ics.hernquist(1 << 15, 3)
    p32 = w.pos.astype(np.float32)
    x, y, z = (torch.from_numpy(np.ascontiguousarray(p32[a])).cuda() for a in range(3))
    m = torch.from_numpy(w.mass.astype(np.float32)).cuda()
    grid = at.candidates(groups=(32, 16), leaves=(8, 16), tiles=(64,))
    path = str(tmp_path / "tune.json")
    r = at.autotune(x, y, z, m, theta=0.5, eps_star=0.005, grid=grid, reps=2, cache_path=path)
    assert not r["cached"] and r["config"] in [dict(group=c["group"], n_leaf=c["n_leaf"], tile=c["tile"]) for c in grid]
    best = min(r["table"], key=lambda t: t["total_ms"])
    assert r["config"]["group"] == best["group"] and r["config"]["n_leaf"] == best["n_leaf"]
    r2 = at.autotune(x, y, z, m, theta=0.5, eps_star=0.005, grid=grid, reps=2, cache_path=path)
    assert r2["cached"] and r2["config"] == r["config"]
    assert os.path.exists(path)
