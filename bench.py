"""Benchmark: tree-force particles/s on one GB300 at p99 relative force
error <= 1e-3 against the FP64 direct sum.

Default workload (the largest configuration the metric names that fits one
GPU): a Hernquist (Dehnen gamma = 1) galaxy of 2^24 equal-mass stars, total
mass 1, scale radius 1, isotropic velocities from the distribution function;
star softening 0.005; opening angle 0.8 with quadrupoles (the tree of the
learned-correction configuration). One step = the whole force path once:
kick/drift, tree build (bounds, keys, sort, topology, multipoles, groups),
tree walk, kick, FP64 energy/momentum totals, replayed from a CUDA graph.
Reported beside the value: the learned cell-force correction (the network is
trained first, untimed, on samples the code generates) as a force pass at
theta 0.8 and at theta 1.0, the plain tree's force pass at the same angles,
the network kernel's tensor-core roofline, and the tree build's HBM roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload learned|hernquist_bh|hernquist_bh_relmac|hernquist_bh_block|hernquist_binary|plummer|ensemble]

Other workloads: `hernquist_bh` (2^20 stars plus one SMBH of mass 0.005 on a
circular orbit at r = 0.5, its FP64 perturbers within r < 0.02, theta 0.5),
`hernquist_bh_block` (the same on block time steps: levels 0..4 below
dt_max = 1/64 from tau_acc = tau_vel = 0.3, walks of the groups holding an
active star; particles = active star updates), `hernquist_bh_relmac` (the
same with the relative opening criterion the paper's runs use, tolerance
1e-3, the previous step's accelerations as references), `hernquist_binary`
(2^22 stars, central SMBH pair, 256 nearest perturbers, the pair's
quadrupole on the other stars), `plummer` (4096 stars), `ensemble` (64
independent Hernquist realisations, sizes log-uniform in 8192..524288, each
with a central SMBH pair, all members in one build and one walk per step).
Every step except the block scheme's is captured once as a CUDA graph and
replayed (--no-graph launches its kernels one by one). Each workload fixes
its tree (leaf size, walk group); the autotuner picks the interaction tile,
and a wider sweep over (group, leaf, tile) is reported beside.

Under torchrun (N > 1) every rank runs its own realisation (replicas: no
data exchange); the value is the sum of particles over ranks / max time.
--impl reference times the CPU oracle (FP64, all host cores) on the same
workload: its tree of all stars is built once (timed, reported), and each
step walks a fresh seeded sample of 8192 stars on it; ms_per_step is the
measured wall time of a step, and the value is the whole-pass throughput
n / (build + n x walk time per star) with the scale stated in the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tree-force particles/s on 1 GB300 at p99 rel. force err ≤1e-3 vs FP64 direct"
UNIT = "particles/s"
FLOP_P2P, FLOP_M2P = 20, 54   # per interaction, counted from the walk kernel's source
L2_FLUSH_BYTES = 256 << 20
WALK_PROFILE = os.path.join(ROOT, "profiles", "walk_tree_k_hernquist_n4194304_theta0.8.md")


def _dist():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def make_workload(name: str, rank: int = 0, stars: int | None = None) -> dict:
    """The workload `name`; `stars` (default workload only) scales its galaxy
    down, e.g. for a profiler capture of the same kernels on a smaller case."""
    import ics
    base = 1000 * rank
    if name == "learned":
        ns = int(stars) if stars else 1 << 24
        w = ics.hernquist(ns, seed=5 + base)
        d = dict(pos=w.pos, vel=w.vel, mass=w.mass, offsets=None, chain_m=None, chain_x=None, chain_v=None,
                 pert_mode=0, pert_radius=0.0, pert_k=0)
        cfg = {"workload": f"hernquist_gamma1_n{ns}", "n_stars": ns}
    elif name in ("hernquist_bh", "hernquist_bh_relmac", "hernquist_bh_block"):
        w = ics.hernquist_bh_workload(1 << 20, seed=2 + base)
        d = dict(pos=w.stars.pos, vel=w.stars.vel, mass=w.stars.mass, offsets=None, chain_m=w.chain.mass,
                 chain_x=w.chain.pos, chain_v=w.chain.vel, pert_mode=1, pert_radius=0.02, pert_k=0)
        cfg = {"workload": "hernquist_gamma1_n1048576_smbh", "n_stars": 1 << 20, "smbh_mass": 0.005,
               "smbh_orbit_r": 0.5, "perturber_radius": 0.02}
    elif name == "hernquist_binary":
        w = ics.hernquist_binary_workload(1 << 22, seed=3 + base)
        d = dict(pos=w.stars.pos, vel=w.stars.vel, mass=w.stars.mass, offsets=None, chain_m=w.chain.mass,
                 chain_x=w.chain.pos, chain_v=w.chain.vel, pert_mode=2, pert_radius=0.0, pert_k=256)
        cfg = {"workload": "hernquist_gamma1_n4194304_smbh_binary", "n_stars": 1 << 22, "binary_a": 0.01,
               "binary_e": 0.1, "smbh_mass": 0.005, "perturbers": "256 nearest",
               "chain_field_beyond_perturbers": "centre of mass + quadrupole"}
    elif name == "plummer":
        w = ics.plummer_workload(4096, seed=1 + base)
        d = dict(pos=w.stars.pos, vel=w.stars.vel, mass=w.stars.mass, offsets=None, chain_m=None, chain_x=None,
                 chain_v=None, pert_mode=0, pert_radius=0.0, pert_k=0)
        cfg = {"workload": "plummer_n4096", "n_stars": 4096}
    elif name == "ensemble":
        e = ics.ensemble_workload(64, seed=4 + base)
        d = dict(pos=e["pos"], vel=e["vel"], mass=e["mass"], offsets=e["offsets"], chain_m=e["chain_m"],
                 chain_x=e["chain_x"], chain_v=e["chain_v"], pert_mode=2, pert_radius=0.0, pert_k=256)
        cfg = {"workload": "ensemble64_hernquist_gamma1_smbh_binary", "n_stars": int(e["offsets"][-1]),
               "members": 64, "member_sizes": "log-uniform 8192..524288 (seed 4)", "perturbers": "256 nearest",
               "chain_field_beyond_perturbers": "centre of mass + quadrupole"}
    else:
        raise ValueError(name)
    d["eps"] = 0.01 if name == "plummer" else 0.005
    d["theta"] = 0.8 if name == "learned" else 0.5
    d["dt"] = 1e-3
    d["name"] = name
    d["n"] = int(d["mass"].shape[0])
    # the workload's tree (both arms build the same one); the walk's tile is tuned
    d["n_leaf"], d["group"] = (16, 32) if name == "plummer" else (24, 64)
    star_mb = 44 * d["n"] / 1e6   # x, y, z, vx, vy, vz, m, ax, ay, az, pot (FP32)
    cfg["l2"] = (f"star arrays {star_mb:.1f} MB" + (" (larger than the 129 MB L2)" if star_mb > 129 else "") + "; " +
                 "GPU arm: 256 MiB written between timed steps (L2 flush)")
    # the paper's runs open cells by a relative ("Gadget") criterion with tolerance 1e-3 (Sect. 3)
    d["mac"], d["alpha"] = (1, 1e-3) if name.endswith("_relmac") else (0, 1e-3)
    cfg.update({"eps_star": d["eps"], "theta": d["theta"], "quadrupole": True, "dt": 1e-3,
                "n_leaf": d["n_leaf"], "walk_group": d["group"]})
    if d["mac"] == 1:
        cfg.update({"workload": cfg["workload"] + "_relative_mac", "mac": "relative (M s^2 <= alpha |a| d^4)",
                    "alpha": d["alpha"], "theta_for_first_pass_and_smbh": 0.5})
    # block time steps (Sect. 2 hierarchy; tau 0.3 as the paper's stars, Sect. 3)
    d["block"] = dict(dt_max=1.0 / 64, L=4, tau=0.3) if name.endswith("_block") else None
    if d["block"]:
        cfg.update({"workload": cfg["workload"] + "_block_steps", "dt_max": 1.0 / 64, "max_level": 4,
                    "tau_acc": 0.3, "tau_vel": 0.3,
                    "metric_note": "particles = active star force updates; one step = dt_max = 16 substeps"})
        cfg.pop("dt", None)
    d["config"] = cfg
    return d


def member_ranges(d):
    off = d["offsets"] if d["offsets"] is not None else np.array([0, d["n"]])
    return [(int(off[k]), int(off[k + 1])) for k in range(len(off) - 1)]


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index, self.samples, self.proc, self.thread = index, [], None, None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for p in self.samples:
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for name, v in zip(names, p[3:]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reported baseline; never tuned)
# ---------------------------------------------------------------------------
REF_SAMPLE = 8192   # stars walked per oracle step (both the reference arm and the cpu_baseline leg)


class OracleRun:
    """The CPU oracle on a workload, with the workload's tree (leaf size, walk
    group) and the same method as the GPU path (each chain's centre of mass an
    unsoftened extra particle carrying the chain's quadrupole). The trees of
    the members are built once, timed; each step walks a seeded sample of
    stars on them and is timed. full_pass_s() scales both to one pass over
    all stars."""

    def __init__(self, d, max_stars=1 << 24):
        import oracle
        self.d = d
        p32 = d["pos"].astype(np.float32)
        m32 = d["mass"].astype(np.float32)
        self.ranges = [(s, e) for (s, e) in member_ranges(d) if e > s]
        chosen, tot = [], 0
        for (s, e) in self.ranges:
            if chosen and tot + (e - s) > max_stars:
                break
            chosen.append((s, e))
            tot += e - s
        self.chosen, self.tot = chosen, tot
        t0 = time.perf_counter()
        self.trees = [oracle.Tree(p32[:, s:e], m32[s:e], d["n_leaf"], d["group"]) for (s, e) in chosen]
        self.build_s = time.perf_counter() - t0
        self.p32 = p32

    def step(self, sample, seed):
        """Walks of `sample` stars spread over the built members; returns (seconds, stars walked)."""
        import ics
        import oracle
        d = self.d
        per = max(1, sample // len(self.chosen))
        walked, t = 0, 0.0
        for k, ((s, e), T) in enumerate(zip(self.chosen, self.trees)):
            tg = ics.subsample(e - s, min(per, e - s), seed=seed * 1000 + k)
            rel = None
            if d.get("mac") == 1:
                # references for the relative criterion: the Hernquist field -x / (r (r + 1)^2) (G = M = a = 1)
                x = self.p32[:, s:e].astype(np.float64)
                r = np.maximum(np.linalg.norm(x, axis=0), 1e-12)
                rel = (d["alpha"], (-x / (r * (r + 1.0) ** 2)).astype(np.float32))
            t0 = time.perf_counter()
            if d["chain_m"] is not None:
                nch = len(d["chain_m"]) // len(self.ranges)
                mi = member_ranges(d).index((s, e))
                mom = oracle.chain_moments(d["chain_m"][mi * nch:(mi + 1) * nch], d["chain_x"][mi * nch:(mi + 1) * nch])
                xq = [mom["Q"]] if nch > 1 else None
                T.forces(d["theta"], float(np.float32(d["eps"])), True, mom["com"].astype(np.float32).reshape(3, 1),
                         np.array([float(np.float32(mom["M"]))]), [0.0], targets=tg, rel=rel, extra_quad=xq)
            else:
                T.forces(d["theta"], float(np.float32(d["eps"])), True, targets=tg, rel=rel)
            t += time.perf_counter() - t0
            walked += len(tg)
        return t, walked

    def full_pass_s(self, walk_s, walked):
        return self.build_s * self.d["n"] / self.tot + walk_s * self.d["n"] / walked

    def describe(self, walked):
        return (f"oracle trees (n_leaf {self.d['n_leaf']}, group {self.d['group']}) of {len(self.chosen)} member(s) "
                f"({self.tot} stars, built once in {self.build_s:.2f} s) + walks of {walked} seeded stars per step; "
                f"whole pass = build x {self.d['n'] / self.tot:.3f} + walk x {self.d['n'] / walked:.1f}")


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    d = make_workload(args.workload, 0, args.stars)
    orc = OracleRun(d)
    for i in range(args.warmup):
        orc.step(REF_SAMPLE, seed=100 + i)
    step_s, walked = [], 0
    for i in range(args.steps):
        t, walked = orc.step(REF_SAMPLE, seed=i)
        step_s.append(t)
    walk_s = float(np.mean(step_s))
    value = d["n"] / orc.full_pass_s(walk_s, walked)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * walk_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": d["config"],
            "step": f"oracle walk of {walked} sampled stars (measured wall time)",
            "scale": {"build_s": orc.build_s, "build_scale": d["n"] / orc.tot, "walk_scale": d["n"] / walked,
                      "whole_pass_s": orc.full_pass_s(walk_s, walked)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": orc.describe(walked)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def _walk_traffic(n):
    """DRAM bytes per walk launch on n stars of the default workload's galaxy
    from the committed ncu summary (captured on a smaller galaxy of the same
    kind and scaled by the stars: the traffic grows with them), if it was
    taken on the current walk.cu (else None)."""
    import hashlib
    import re
    try:
        txt = open(WALK_PROFILE).read()
        src = open(os.path.join(ROOT, "paper_1507_01009_gb300", "csrc", "walk.cu"), "rb").read()
    except OSError:
        return None
    h = hashlib.sha256(src).hexdigest()[:16]
    m = re.search(r"walk.cu sha256 prefix: `([0-9a-f]+)`", txt)
    t = re.search(r"= \*\*([0-9.]+) MB per launch\*\*", txt)
    c = re.search(r"captured stars: `([0-9]+)`", txt)
    if not m or not t or not c or m.group(1) != h:
        return None
    return float(t.group(1)) * 1e6 * n / float(c.group(1))


def max_over_ranks(ms: float, device=None) -> float:
    """Largest timed-region duration over all ranks (the job's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, stars_per_rank: int, steps: int, total_ms: float) -> float:
    """Whole-job particles/s: every rank advances its own realisation (replicas)."""
    return world * stars_per_rank * steps / (total_ms / 1e3)


def _rel_err(a, ref):
    """Per-body relative error |a - ref| / |ref| of (3, k) vectors."""
    return np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)


def _p99(e):
    """Nearest-rank 99th percentile: sorted ascending, index ceil(0.99 k) - 1."""
    s = np.sort(np.asarray(e, np.float64))
    return float(s[max(0, math.ceil(0.99 * s.size) - 1)]) if s.size else float("nan")


def p99_vs_direct(d, S, sample=2048, seed=77):
    """p99 relative acceleration error of the current GPU forces against the
    fully resolved FP64 direct sum (the library's rv_direct_fp64, on the GPU)
    over each sampled star's own member: stars softened, every chain member
    an unsoftened body of its own (no chain model)."""
    import ics
    from paper_1507_01009_gb300 import rv
    xs = np.stack([t.cpu().numpy() for t in (S.x, S.y, S.z)]).astype(np.float64)
    a = np.stack([t.cpu().numpy() for t in (S.ax, S.ay, S.az)]).astype(np.float64)
    m32 = S.m.cpu().numpy().astype(np.float64)
    eps = float(np.float32(d["eps"]))
    ranges = member_ranges(d)
    tg = ics.subsample(d["n"], sample, seed=seed)
    cx = S.chain_x.cpu().numpy().reshape(-1, 3) if S.chain_x is not None else None
    errs = []
    for k, (s, e) in enumerate(ranges):
        t = tg[(tg >= s) & (tg < e)]
        if len(t) == 0:
            continue
        pos, mass, epsv = xs[:, s:e], m32[s:e], np.full(e - s, eps)
        if cx is not None:
            nch = S.n_chain
            cm = d["chain_m"][k * nch:(k + 1) * nch]
            pos = np.concatenate([pos, cx[k * nch:(k + 1) * nch].T], 1)
            mass = np.concatenate([mass, cm])
            epsv = np.concatenate([epsv, np.zeros(nch)])
        ad, _ = rv.direct_fp64(pos, mass, epsv, t - s)
        errs.append(_rel_err(a[:, t], ad))
    return _p99(np.concatenate(errs))


P99_BOUND = 1e-3   # the metric's accuracy condition


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1507_01009_gb300 import rv

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    d = make_workload(args.workload, rank, args.stars)
    n = d["n"]
    # every step but the block scheme's is captured once as a CUDA graph and replayed
    use_graph = args.workload not in ("hernquist_bh_block",) and not args.no_graph
    blk = d["block"]

    # the walk's interaction tile: the autotuner's pick for the workload's tree (untimed); a wider
    # sweep over (group, leaf, tile) is reported beside
    from paper_1507_01009_gb300 import autotune
    p32 = d["pos"].astype(np.float32)
    xs = [torch.from_numpy(np.ascontiguousarray(p32[a])).to(dev) for a in range(3)]
    ms = torch.from_numpy(d["mass"].astype(np.float32)).to(dev)
    tkw = dict(offsets=d["offsets"], theta=d["theta"], eps_star=float(np.float32(d["eps"])), reps=2, cache_path=None)
    tuned = autotune.autotune(*xs, ms, grid=autotune.candidates(groups=(d["group"],), leaves=(d["n_leaf"],),
                                                                 tiles=autotune.GRID_TILE), **tkw)
    wide = autotune.autotune(*xs, ms, grid=autotune.candidates(groups=(32, 64), leaves=(8, 16, 24, 32),
                                                                tiles=(64, 96, 128, 256)), **tkw) if not args.no_sweep else None
    tune = tuned["config"]
    if d["name"] != "learned":
        del xs, ms
    ctx = rv.Context(n, theta=d["theta"], eps_star=float(np.float32(d["eps"])), mac=d["mac"], alpha=d["alpha"],
                     **tune)
    S = rv.System(d["pos"], d["vel"], d["mass"], chain_m=d["chain_m"], chain_x=d["chain_x"], chain_v=d["chain_v"],
                  pert_mode=d["pert_mode"], pert_radius=d["pert_radius"], pert_k=d["pert_k"],
                  member_offsets=d["offsets"])
    M = S.n_members
    energy_out = torch.zeros(10 * M, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev) if use_graph else torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    B = rv.Blocks(n, blk["dt_max"], blk["L"], tau_acc=blk["tau"], tau_vel=blk["tau"],
                  eps=float(np.float32(d["eps"]))) if blk else None

    def step():
        if use_graph:
            ctx.kdk_step_graph(S, d["dt"], 1, energy_out=energy_out, stream=stream)
        elif blk:
            ctx.block_steps(S, B, 2 ** blk["L"], stream=stream)      # one dt_max: ends at a sync point
            ctx.energy(S, out=energy_out, stream=stream)
        else:
            ctx.kdk_step(S, d["dt"], 1, stream=stream)
            ctx.energy(S, out=energy_out, stream=stream)

    with torch.cuda.stream(stream):
        if blk:
            ctx.block_start(S, B, stream=stream)
        else:
            ctx.system_forces(S, stream=stream)
        ctx.energy(S, out=energy_out, stream=stream)
        e_first = energy_out.view(M, 10)[:, 2].sum().item()   # total energy before the first step
        for _ in range(max(3, args.warmup)):
            step()
    ctx.sync_status(stream=stream)

    # ---- timed region: exactly K steps, CUDA events on the launching stream, L2 flushed before each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    b0 = ctx.block_count() if blk else 0
    ctx.profile_walk(not blk)   # block steps: walks of varying size, timed as full walks below
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 255)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = ctx.launch_count() - l0
    walk_total_ms, walk_launches = ctx.walk_time()
    ctx.profile_walk(False)
    sampler.stop()
    ctx.sync_status(stream=stream)
    e_last = energy_out.view(M, 10)[:, 2].sum().item()   # after the last timed step
    n_steps = max(3, args.warmup) + args.steps
    energy_drift = {"rel": (e_last - e_first) / abs(e_first), "steps": n_steps,
                    "dt": (blk["dt_max"] if blk else d["dt"]), "E0": e_first}
    total_ms = max_over_ranks(float(np.sum([a.elapsed_time(b) for a, b in ev])), dev)
    ms_per_step = total_ms / args.steps
    if blk:   # particles = active star force updates
        upd = ctx.block_count() - b0
        value = job_throughput(ws, upd / args.steps, args.steps, total_ms)
    else:
        value = job_throughput(ws, n, args.steps, total_ms)
    p99 = p99_vs_direct(d, S) if rank == 0 else None

    # ---- dominant kernel: the walk. Its launches inside the timed steps were timed
    # with CUDA events on the launching stream (not possible inside a replayed
    # graph: then a separate loop of build + walk on the same stream is timed).
    n_p2p, n_m2p = ctx.walk_stats()
    flop = FLOP_P2P * n_p2p + FLOP_M2P * n_m2p
    if walk_launches > 0:
        walk_ms = walk_total_ms / walk_launches
        walk_src = "walk launches inside the timed steps"
    else:
        pairs = []
        off = d["offsets"] if d["offsets"] is not None else [0, n]
        ref = tuple(t.clone() for t in (S.ax, S.ay, S.az))   # relative criterion: the step's references
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ctx.build_tree_members(off, S.x, S.y, S.z, S.m, stream=stream)
                flush.fill_(k & 255)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if d["mac"] == 1:
                    ctx.tree_forces_rel(d["alpha"], ref, out=(S.ax, S.ay, S.az, S.pot), stream=stream)
                else:
                    ctx.tree_forces_members(out=(S.ax, S.ay, S.az, S.pot), stream=stream)
                e1.record(stream)
                pairs.append((e0, e1))
        torch.cuda.synchronize()
        ctx.sync_status(stream=stream)
        walk_ms = float(np.mean([a.elapsed_time(b) for a, b in pairs]))
        n_p2p, n_m2p = ctx.walk_stats()
        flop = FLOP_P2P * n_p2p + FLOP_M2P * n_m2p
        walk_src = ("separate build + full walk loop (block steps walk only the active groups); extra particles "
                    "omitted" if blk else
                    "separate build + walk loop, same criterion (steps replayed from a CUDA graph); extra particles "
                    "omitted")
    achieved = flop / (walk_ms / 1e3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * 2 * 2.07e9 / 1e12   # FP32 lanes x FMA x max SM clock
    traffic = _walk_traffic(n) if d["name"] == "learned" else None
    roofline = {"bound": "alu", "kernel": "walk_tree_k", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_note": ("dram read + write bytes per launch from the committed ncu capture of the same "
                                 "walk.cu on the 2^22-star galaxy, scaled by the stars" if traffic else None),
                "peak_note": f"{sms} SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz (derived, not measured)",
                "walk_ms": walk_ms, "walk_timing": walk_src, "flop_per_launch": float(flop),
                "interactions_per_star": float((n_p2p + n_m2p) / max(n, 1)),
                "walk_share_of_step": walk_ms / ms_per_step}
    roof_build = build_roofline(ctx, d, S, stream, flush, args.steps, ms_per_step)

    # ---- end to end through the public API with host (pinned) buffers
    # the state a step reads (positions, velocities, the forces its first kick
    # uses) goes in every step and the state it leaves comes back, with the
    # energy totals; the masses are constant and the potentials are reduced on
    # the device into the energy totals
    # (rows x, y, z, vx, vy, vz, ax, ay, az of the System's state block: one
    # copy each way)
    dev_state = S.state[:9]
    host_state = torch.empty((9, n), dtype=torch.float32, pin_memory=True)
    host_state.copy_(dev_state.cpu())
    e_host = torch.empty(10 * M, dtype=torch.float64, pin_memory=True)
    h2d = 4 * n * 9
    d2h = 4 * n * 9 + 80 * M
    lv_host = None
    if blk:   # the levels are state of the block scheme too
        lv_host = torch.empty(n, dtype=torch.int8, pin_memory=True)
        lv_host.copy_(B.level.cpu())
        h2d += n
        d2h += n
    e2e_ms = []
    with torch.cuda.stream(stream):
        # untimed warm-up of the same loop: the first copies into and out of the
        # freshly pinned host buffers pay a one-time setup cost (~30 ms measured)
        for k in range(max(3, args.warmup) + args.steps):
            flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dev_state.copy_(host_state, non_blocking=True)
            if blk:
                B.level.copy_(lv_host, non_blocking=True)
            step()
            host_state.copy_(dev_state, non_blocking=True)
            if blk:
                lv_host.copy_(B.level, non_blocking=True)
            e_host.copy_(energy_out, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if k >= max(3, args.warmup):
                e2e_ms.append(e0.elapsed_time(e1))
    ctx.sync_status(stream=stream)
    e2e_val = ws * (upd / args.steps if blk else n) / (float(np.mean(e2e_ms)) / 1e3)

    separate = None
    if d["name"] == "ensemble" and rank == 0:
        separate = ensemble_separate(d, tune, args.steps, args.warmup, flush)

    learned, roof_net = None, None
    if d["name"] == "learned" and rank == 0 and not args.no_learned:
        del S, ctx
        torch.cuda.empty_cache()
        learned, roof_net = learned_leg(d, xs, ms, tune, flush, args.steps, max(3, args.warmup))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        orc = OracleRun(d)
        orc.step(REF_SAMPLE, seed=2)                      # warm-up
        st = [orc.step(REF_SAMPLE, seed=3 + k) for k in range(2)]
        cs, walked = float(np.mean([t for t, _ in st])), st[0][1]
        cpu = {"value": n / orc.full_pass_s(cs, walked), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": orc.describe(walked) + "; 1 warm-up + 2 timed walks",
               "measured_s": orc.build_s + 3 * cs}

    if rank == 0:
        cfg = dict(d["config"])   # the workload, identical in the reference arm's line
        run = {"tile": tune["tile"],
               "step": ("16 block substeps (drift, perturber select, build, walk of active groups, fp64 "
                        "perturber/chain, kicks and levels of active stars) + energy" if blk else
                        "kdk + perturber select + build + walk + fp64 perturber/chain + energy"
                        if d["chain_m"] is not None else "kdk + build + walk + energy"),
               "parallelism": f"replicas{ws}" if ws > 1 else "single", "graph_captured": bool(use_graph)}
        tuning = {"tile_grid_walk_ms": {str(r["tile"]): round(r["walk_ms"], 3) for r in tuned["table"]}}
        if wide is not None:
            best = min(wide["table"], key=lambda r: r["total_ms"])
            tuning["wide_sweep_build_plus_walk_ms"] = {f'{r["group"]}/{r["n_leaf"]}/{r["tile"]}':
                                                       round(r["total_ms"], 3) for r in wide["table"]}
            tuning["wide_sweep_best"] = {k: best[k] for k in ("group", "n_leaf", "tile")}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
                "run": run, "p99_rel_err_vs_fp64_direct": p99, "meets_p99": bool(p99 is not None and p99 <= P99_BOUND),
                "clocks": sampler.summary(),
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": float(np.mean(e2e_ms)), "ms_per_step_median": float(np.median(e2e_ms)),
                        "ms_per_step_max": float(np.max(e2e_ms))},
                "gpu_launches": int(launches), "roofline": roofline, "roofline_build": roof_build,
                "cpu_baseline": cpu, "energy_drift": energy_drift, "autotune": tuning}
        if separate is not None:
            line["batched_vs_separate"] = {"batched_particles_per_s": value, "batched_ms_per_step": ms_per_step,
                                           "separate": separate, "speedup": value / separate["particles_per_s"]}
        if learned is not None:
            line["learned_correction"] = learned
            line["roofline_network"] = roof_net
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# learned cell-force correction: tree at theta 0.8 + network, 2^24 stars
# ---------------------------------------------------------------------------
def ensemble_separate(d, tune, steps, warmup, flush):
    """The ensemble's members stepped one after another, each as its own
    single-galaxy system (its own context, the same tree parameters, tile and
    criterion, its own captured KDK step with its SMBH pair and perturbers):
    the plain tree the batched form is compared with, in particles/s over the
    same stars. Timed like the batched steps (CUDA events on the launching
    stream, L2 flush before each step of all members)."""
    import torch
    from paper_1507_01009_gb300 import rv
    off = d["offsets"]
    M = len(off) - 1
    nch = len(d["chain_m"]) // M
    eps = float(np.float32(d["eps"]))
    stream = torch.cuda.Stream()
    members = []
    for k in range(M):
        a, b = int(off[k]), int(off[k + 1])
        ctx = rv.Context(b - a, theta=d["theta"], eps_star=eps, mac=d["mac"], alpha=d["alpha"], **tune)
        S = rv.System(d["pos"][:, a:b], d["vel"][:, a:b], d["mass"][a:b], chain_m=d["chain_m"][k * nch:(k + 1) * nch],
                      chain_x=d["chain_x"][k * nch:(k + 1) * nch], chain_v=d["chain_v"][k * nch:(k + 1) * nch],
                      pert_mode=d["pert_mode"], pert_radius=d["pert_radius"], pert_k=d["pert_k"])
        members.append((ctx, S, torch.zeros(10, dtype=torch.float64, device="cuda")))
    with torch.cuda.stream(stream):
        for ctx, S, eo in members:
            ctx.system_forces(S, stream=stream)
        for _ in range(max(3, warmup)):
            for ctx, S, eo in members:
                ctx.kdk_step_graph(S, d["dt"], 1, energy_out=eo, stream=stream)
    torch.cuda.synchronize()
    ev = []
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for ctx, S, eo in members:
                ctx.kdk_step_graph(S, d["dt"], 1, energy_out=eo, stream=stream)
            e1.record(stream)
            ev.append((e0, e1))
    torch.cuda.synchronize()
    for ctx, S, eo in members:
        ctx.sync_status(stream=stream)
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    return {"particles_per_s": d["n"] / (ms / 1e3), "ms_per_step": ms, "members": M,
            "how": "each member its own context and captured step, members one after another on one stream"}


def build_roofline(ctx, d, S, stream, flush, reps, ms_per_step):
    """The tree build (bounding cube, keys, radix sort, permutation, topology,
    groups, moments: all HBM-bound) timed alone with CUDA events on its
    stream, an L2 flush before each, against the measured HBM copy bandwidth.
    Algorithmic bytes per build: per star the cube's 12 B read; keys 16 B read
    and 8 B (key) + 16 B (the packed star) written; each of the sort's passes
    (7 of 9 bits for 63-bit keys, one more on the member when there are
    several) 12 B read + 8 B (the up-sweep's key) + 12 B written; the
    permutation 4 B + 16 B read and 16 B written; the topology 8 B read; the
    moments 16 B read; per cell 42 B written by the topology and 48 B read +
    48 B written by the moments."""
    import torch
    off = d["offsets"] if d["offsets"] is not None else [0, S.n]
    ev = []
    with torch.cuda.stream(stream):
        for k in range(max(4, reps)):
            flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.build_tree_members(off, S.x, S.y, S.z, S.m, stream=stream)
            e1.record(stream)
            ev.append((e0, e1))
    torch.cuda.synchronize()
    ctx.sync_status(stream=stream)
    ms = float(np.median([a.elapsed_time(b) for a, b in ev[1:]]))
    n, ncell, _ = ctx.tree_sizes()
    passes = 7 + (1 if len(off) > 2 else 0)
    per_star = 12 + 40 + passes * 32 + 36 + 8 + 16
    nbytes = n * per_star + ncell * (42 + 96)
    gbs = nbytes / (ms / 1e3) / 1e9
    hbm = _measured_peaks().get("hbm_gbs")
    peak = hbm or 6800.0
    return {"bound": "hbm", "kernels": f"bounds, keys, sort ({passes} passes), gather, topology, groups, moments",
            "ms": ms, "bytes": float(nbytes), "bytes_per_star": nbytes / max(n, 1), "cells": ncell,
            "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "traffic": None,
            "share_of_step": ms / ms_per_step,
            "peak_note": "hbm_gbs of MEASURED_PEAKS.json (copy)" if hbm else "fallback 6.8 TB/s"}


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def learned_leg(d, xs, ms, tune, flush, steps, warmup):
    """The learned cell-force correction beside the plain tree, as force
    passes (build + walk [+ pair record + network + correction]) on the
    workload's stars: at the workload's theta and at theta 1.0 (where the
    plain tree misses p99 1e-3). At each angle a fresh network is trained
    first (untimed) on 2^20 samples the code generates at that angle (400 Adam
    steps of 8192 rows). p99 against the FP64 direct sum on 2048 seeded
    stars; the network kernel alone is timed on the recorded pairs' row count."""
    import torch
    import ics
    from paper_1507_01009_gb300 import rv
    n = d["n"]
    eps = float(np.float32(d["eps"]))
    x, y, z = xs
    m = ms
    ctx = rv.Context(n, theta=d["theta"], eps_star=eps, n_leaf=d["n_leaf"], group=d["group"], tile=tune["tile"])
    tg = ics.subsample(n, 2048, seed=17)
    ad, _ = rv.direct_fp64(d["pos"].astype(np.float32).astype(np.float64),
                           d["mass"].astype(np.float32).astype(np.float64), eps, tg)

    def p99(o):
        a = np.stack([u[tg].cpu().numpy() for u in o[:3]]).astype(np.float64)
        return _p99(_rel_err(a, ad))

    def timed(fn):
        for _ in range(warmup):
            o = fn()
        torch.cuda.synchronize()
        t = []
        for k in range(steps):
            flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            o = fn()
            e1.record()
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        ctx.sync_status()
        return float(np.mean(t)), o

    out, net_rows, net = {}, 0, None
    for th, trec in ((d["theta"], 0.7), (1.0, 0.7)):
        ctx.build_tree(x, y, z, m)
        fx, ft, _ = rv.mlp_samples(ctx, th, eps, 1 << 20, seed=7)
        net = rv.Mlp(seed=8)
        losses = net.train(fx, ft, steps=400, batch=8192, lr=2e-3, seed=2)
        del fx, ft

        def learned_pass():
            ctx.build_tree(x, y, z, m)
            return rv.tree_forces_mlp(ctx, net, th, trec, eps, pair_cap=1 << 28)

        def plain_pass():
            ctx.build_tree(x, y, z, m)
            return ctx.tree_forces(theta=th, eps_star=eps)

        t_l, o_l = timed(learned_pass)
        npairs = int(o_l[5].item())
        net_rows = max(net_rows, npairs)
        p_l = p99(o_l)
        del o_l
        t_p, o_p = timed(plain_pass)
        p_p = p99(o_p)
        del o_p
        out[f"theta_{th}"] = {
            "plain": {"ms": t_p, "particles_per_s": n / (t_p / 1e3), "p99": p_p, "meets_p99": p_p <= P99_BOUND},
            "learned": {"ms": t_l, "particles_per_s": n / (t_l / 1e3), "p99": p_l, "meets_p99": p_l <= P99_BOUND,
                        "theta_rec": trec, "pairs": npairs, "train_loss_first_last": [losses[0], losses[-1]]}}
    # the network kernel alone (tcgen05, bf16) on as many rows as the largest pair record
    feats = torch.zeros((max(net_rows, 1), 16), dtype=torch.float32, device="cuda")
    t_net = []
    for k in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.forward(feats)
        e1.record()
        e1.synchronize()
        t_net.append(e0.elapsed_time(e1))
    del feats
    flop_row = 2 * (14 * 64 + 64 * 64 + 64 * 3)   # the network's own multiply-adds (padding not counted)
    tflops = net_rows * flop_row / (float(np.median(t_net[1:])) / 1e3) / 1e12
    peaks = _measured_peaks()
    bf16 = peaks.get("bf16_tflops")
    roof = {"bound": "tensor", "kernel": "mlp_forward_tc_k (tcgen05, bf16 operands, fp32 accumulate)",
            "rows": net_rows, "flop_per_row": flop_row, "ms": float(np.median(t_net[1:])), "achieved": tflops,
            "peak": bf16 or 1900.0, "unit": "TFLOP/s", "frac": tflops / (bf16 or 1900.0), "traffic": None,
            "peak_note": "bf16_tflops of MEASURED_PEAKS.json (burst)" if bf16 else "fallback 1.9 PFLOP/s bf16"}
    # the epilogue's special-function unit: one tanh per hidden activation
    # (2 x 64 a row) at one warp instruction (32 results) per clock per SM, the
    # XU pipe's peak as ncu counts it on GB300 (152 SMs, 2.07 GHz maximum clock)
    sfu_ms = net_rows * 2 * 64 / (32 * 152 * 2.07e9) * 1e3
    roof["sfu_bound"] = {"ms": sfu_ms, "frac": sfu_ms / roof["ms"], "tflops_at_bound": net_rows * flop_row / sfu_ms / 1e9,
                         "note": "time the tanh operations alone take on the SFU pipe; frac = that / measured ms"}
    del ctx
    torch.cuda.empty_cache()
    return out, roof


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="learned",
                    choices=["learned", "hernquist_bh", "hernquist_bh_relmac", "hernquist_bh_block", "hernquist_binary",
                             "plummer", "ensemble"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the wide (group, leaf, tile) sweep")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-correction leg")
    ap.add_argument("--stars", type=int, default=None,
                    help="stars of the default workload's galaxy (default 2^24), e.g. a smaller case to profile")
    ap.add_argument("--no-graph", action="store_true", help="launch every kernel of a step (no CUDA graph)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
