"""Benchmark: tree-force particles/s on one GB300 at p99 relative force
error <= 1e-3 against the FP64 direct sum.

Workload: Hernquist (Dehnen gamma = 1) galaxy, 2^20 equal-mass stars of total
mass 1 and scale radius 1, plus one SMBH of mass 0.005 on a circular orbit at
r = 0.5; star softening 0.005; SMBH-star forces unsoftened, FP64 for the
stars within 0.02 of the SMBH; opening angle 0.5 with quadrupoles.

One step = the whole force path once: kick/drift, perturber selection, tree
build (keys, sort, topology, multipoles, groups), tree walk, FP64 perturber
coupling and chain hand-off, kick, FP64 energy/momentum totals.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own realisation (replicas: no
data exchange); the value is the sum of particles over ranks / max time.
--impl reference times the CPU oracle (FP64, all host cores) on the same
workload, on a bounded sample per step.
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
N_STARS = 1 << 20
THETA, EPS, PERT_R, DT = 0.5, 0.005, 0.02, 1e-3
FLOP_P2P, FLOP_M2P = 20, 54   # per interaction, counted from the walk kernel's source
L2_FLUSH_BYTES = 256 << 20


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload_config(n_ranks):
    return {"workload": f"hernquist_gamma1_n{N_STARS}_smbh", "n_stars": N_STARS, "smbh_mass": 0.005,
            "smbh_orbit_r": 0.5, "eps_star": EPS, "theta": THETA, "quadrupole": True, "n_leaf": 16,
            "walk_group": 32, "tile": 64, "perturber_radius": PERT_R, "dt": DT,
            "step": "kdk + perturber select + build + walk + fp64 perturber/chain + energy",
            "parallelism": f"replicas{n_ranks}" if n_ranks > 1 else "single",
            "l2": "flushed (256 MiB write) before every timed step"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
def oracle_step_time(p32, m32, bh_pos32, bh_mass, sample, seed=0):
    """Seconds for one oracle force pass on this workload, from a bounded
    sample: full tree build + tree walk for `sample` stars, scaled to all
    stars. Returns (seconds per full pass, description)."""
    import ics
    import oracle
    n = p32.shape[1]
    tg = ics.subsample(n, sample, seed=seed)
    t0 = time.perf_counter()
    T = oracle.Tree(p32, m32, 16, 32)
    t1 = time.perf_counter()
    T.forces(THETA, float(np.float32(EPS)), True, bh_pos32, np.array([bh_mass]), [0.0], targets=tg)
    t2 = time.perf_counter()
    full = (t1 - t0) + (t2 - t1) * n / len(tg)
    return full, f"oracle tree build of all {n} stars + walk of {len(tg)} sampled stars, walk time scaled x{n / len(tg):.1f}"


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import ics
    w = ics.hernquist_bh_workload(N_STARS, seed=2)
    p32 = w.stars.pos.astype(np.float32)
    m32 = w.stars.mass.astype(np.float32)
    bh = w.chain.pos.T.astype(np.float32)
    sample = 16384
    for i in range(args.warmup):
        oracle_step_time(p32, m32, bh, float(np.float32(w.chain.mass[0])), sample, seed=100 + i)
    times, desc = [], ""
    for i in range(args.steps):
        t, desc = oracle_step_time(p32, m32, bh, float(np.float32(w.chain.mass[0])), sample, seed=i)
        times.append(t)
    ms = 1e3 * float(np.mean(times))
    value = N_STARS / (ms / 1e3)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _workload_config(1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    import ics
    from paper_1507_01009_gb300 import rv

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = ics.hernquist_bh_workload(N_STARS, seed=2 + 1000 * rank)
    p32 = w.stars.pos.astype(np.float32)
    v32 = w.stars.vel.astype(np.float32)
    m32 = w.stars.mass.astype(np.float32)
    ctx = rv.Context(N_STARS, theta=THETA, eps_star=float(np.float32(EPS)), n_leaf=16, group=32, tile=64)
    S = rv.System(p32, v32, m32, chain_m=w.chain.mass, chain_x=w.chain.pos, chain_v=w.chain.vel, pert_mode=1,
                  pert_radius=PERT_R)
    energy_out = torch.zeros(10, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        ctx.kdk_step(S, DT, 1)
        ctx.energy(S, out=energy_out)

    ctx.system_forces(S)
    for _ in range(max(3, args.warmup)):
        step()
    ctx.sync_status()

    # ---- timed region: exactly K steps, each timed with CUDA events, L2 flushed before each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    for k in range(args.steps):
        flush.fill_(k & 255)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = ctx.launch_count() - l0
    sampler.stop()
    ctx.sync_status()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(np.sum(step_ms))
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = ws * N_STARS * args.steps / (total_ms / 1e3)

    # ---- accuracy of the forces the timed steps produced (current state) vs FP64 direct
    p99 = None
    if rank == 0:
        import oracle
        xs = np.stack([t_.cpu().numpy() for t_ in (S.x, S.y, S.z)]).astype(np.float64)
        a = np.stack([t_.cpu().numpy() for t_ in (S.ax, S.ay, S.az)]).astype(np.float64)
        cx = S.chain_x.cpu().numpy().reshape(-1, 3).T
        allp = np.concatenate([xs, cx], 1)
        allm = np.concatenate([m32.astype(np.float64), w.chain.mass])
        epsv = np.concatenate([np.full(N_STARS, float(np.float32(EPS))), [0.0]])
        tg = ics.subsample(N_STARS, 2048, seed=77)
        ad, _ = oracle.direct(allp, allm, epsv, targets=tg)
        p99 = oracle.percentile(oracle.rel_err(a[:, tg], ad), 0.99)

    # ---- dominant kernel (tree walk): CUDA events around rv_tree_forces on the launching stream
    walk_ms, flops = [], []
    xyzm = torch.tensor([[float(S.chain_x[0]), float(S.chain_x[1]), float(S.chain_x[2]), float(S.chain_m[0])]],
                        dtype=torch.float32, device=dev)
    xeps = torch.zeros(1, dtype=torch.float32, device=dev)
    outs = (S.ax, S.ay, S.az, S.pot)
    for k in range(args.steps):
        ctx.build_tree(S.x, S.y, S.z, S.m)
        flush.fill_(k & 255)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.tree_forces(extra_xyzm=xyzm, extra_eps=xeps, out=outs)
        e1.record(stream)
        e1.synchronize()
        walk_ms.append(e0.elapsed_time(e1))
        n_p2p, n_m2p = ctx.walk_stats()
        flops.append(FLOP_P2P * n_p2p + FLOP_M2P * n_m2p)
    ctx.sync_status()
    walk_s = float(np.mean(walk_ms)) / 1e3
    achieved = float(np.mean(flops)) / walk_s / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * 2 * 2.07e9 / 1e12   # FP32 lanes x FMA x max SM clock
    roofline = {"bound": "alu", "kernel": "walk_tree_k", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_note": f"{sms} SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz",
                "walk_ms": float(np.mean(walk_ms)), "flop_per_launch": float(np.mean(flops)),
                "interactions_per_star": float((n_p2p + n_m2p) / N_STARS),
                "walk_share_of_step": float(np.mean(walk_ms)) / ms_per_step}

    # ---- end to end through the public API with host (pinned) buffers
    host = {k_: torch.empty(N_STARS, dtype=torch.float32, pin_memory=True)
            for k_ in ("x", "y", "z", "vx", "vy", "vz", "m", "ax", "ay", "az", "pot")}
    for k_, arr in zip(("x", "y", "z"), p32):
        host[k_].copy_(torch.from_numpy(np.ascontiguousarray(arr)))
    for k_, arr in zip(("vx", "vy", "vz"), v32):
        host[k_].copy_(torch.from_numpy(np.ascontiguousarray(arr)))
    host["m"].copy_(torch.from_numpy(m32))
    for k_ in ("ax", "ay", "az", "pot"):
        host[k_].copy_(getattr(S, k_).cpu())
    e_host = torch.empty(10, dtype=torch.float64, pin_memory=True)
    ins = ("x", "y", "z", "vx", "vy", "vz", "m", "ax", "ay", "az")
    outs_h = ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "pot")
    h2d = 4 * N_STARS * len(ins)
    d2h = 4 * N_STARS * len(outs_h) + 80
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 255)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k_ in ins:
            getattr(S, k_).copy_(host[k_], non_blocking=True)
        step()
        for k_ in outs_h:
            host[k_].copy_(getattr(S, k_), non_blocking=True)
        e_host.copy_(energy_out, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    ctx.sync_status()
    e2e_val = ws * N_STARS / (float(np.mean(e2e_ms)) / 1e3)

    # ---- CPU oracle on this machine's host cores (bounded sample), rank 0 at N = 1 only
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sec, desc = oracle_step_time(p32, m32, w.chain.pos.T.astype(np.float32), float(np.float32(w.chain.mass[0])),
                                     65536, seed=3)
        cpu = {"value": N_STARS / sec, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _workload_config(ws), "p99_rel_err_vs_fp64_direct": p99,
                "clocks": sampler.summary(),
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": float(np.mean(e2e_ms))},
                "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
