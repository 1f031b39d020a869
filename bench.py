#!/usr/bin/env python
"""Benchmark: KIFMM long-range force evaluation on one GB300 per rank.

One step = one pass of the whole hot path over one system: set_sources (bounding
cube, Morton keys, radix sort, octree, U/V/W/X lists) + evaluate (P2M, M2M,
M2L, P2L, L2L, L2P/M2P, P2P, scatter) for the default workload, the
1M-sphere DEM Coulomb packing (RSA to solid fraction 0.4, radii U[0.5, 1.5]
mm, charges N(0, (1e-12 C)^2), p = 6, leaf cap 128, FP32 inputs/outputs).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line on rank 0.  A single system does not shard: with N > 1
every rank evaluates its own replica (no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mparticles/s per KIFMM force eval at 1M, rel-L2 err<=1e-5; speedup vs plain FP32"
UNIT = "Mparticles/s"
EPS0 = 8.8541878128e-12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA x max clock

WORKLOADS = {
    "c2": dict(name="dem-coulomb-rsa-1M", n=1_000_000, p=6, leaf_cap=128, max_depth=20, seed=1001),
    "c2-small": dict(name="dem-coulomb-rsa-64k", n=65_536, p=6, leaf_cap=128, max_depth=20, seed=1001),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=os.environ.get("KIFMM_BENCH_PRECISION", "fp32"))
    ap.add_argument("--accuracy-targets", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def make_inputs(w):
    from workloads import generators as G
    x, q, meta = G.dem_coulomb(w["n"], w["seed"])
    return x, q, meta


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def algorithmic_work(plan, w, n):
    """Algorithmic units per evaluate for the roofline: M2L flops 2 n_s^2 |V|,
    P2P pairs (sum over leaves of n_B times the U-list source count, minus the
    self pairs), tree-build bytes."""
    info = plan.tree_info()
    ns = 6 * (w["p"] - 1) ** 2 + 2
    m2l_flops = 2.0 * ns * ns * info["n_v"]
    t = plan.tree()
    ptr, idx = plan.list("U")
    cnt = t["count"]
    src = np.add.reduceat(cnt[idx], ptr[:-1]) if idx.size else np.zeros(len(cnt))
    src = np.where(np.diff(ptr) > 0, src, 0)
    pairs = float(np.sum(cnt * src) - n)
    # tree: bbox read 16 B, keys read 12 B + write 16 B, 8 sort passes x (read 12 + 12 + write 12) B, gather 36 B
    tree_bytes = n * (16 + 28 + 8 * 36 + 36)
    return {"m2l_flops": m2l_flops, "p2p_pairs": pairs, "tree_bytes": float(tree_bytes), "info": info}


def roofline_for(stage, ms_per_call, work, precision, peaks):
    hbm, bf16, bf16_s, kind = peaks
    if stage == "m2l":
        flops = work["m2l_flops"]
        ach = flops / (ms_per_call * 1e-3) / 1e12
        if precision.startswith("mixed"):
            peak = bf16_s if precision == "mixed_fp16" else bf16_s / 2
            return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": None, "kernel": "m2l", "peak_source": f"{kind} bf16 sustained (fp16 same rate)"}
        return {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "m2l_simt",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    if stage == "p2p":
        flops = 20.0 * work["p2p_pairs"]
        ach = flops / (ms_per_call * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "p2p",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz; 20 flop per pair"}
    if stage == "tree":
        gbs = work["tree_bytes"] / (ms_per_call * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": None, "kernel": "tree", "peak_source": f"{kind} copy bandwidth"}
    return None


def cpu_baseline_leg(x, q, w, n_targets, seed=0, sample_frac=0.5):
    """CPU leg (the only place the benchmark runs the oracle): time the FP64
    oracle KIFMM on a bounded sample of the workload (the corner sub-cube
    holding sample_frac of the particles), and compute FP64 direct-sum
    reference values on sampled targets for the accuracy figures."""
    from oracle import oracle as O
    O.build()
    lo = x.min(axis=0)
    side = (x.max(axis=0) - lo).max()
    cut = side * sample_frac ** (1.0 / 3.0)
    sel = np.all(x - lo < cut, axis=1)
    xs, qs = x[sel], q[sel]
    t0 = time.perf_counter()
    tree = O.sort_and_tree(xs, w["leaf_cap"], w["max_depth"])
    lst = O.lists(tree)
    ops = O.operators(w["p"])
    t1 = time.perf_counter()
    O.kifmm(xs, qs, p=w["p"], tree=tree, lst=lst, ops=ops)
    t2 = time.perf_counter()
    cores = len(os.sched_getaffinity(0))
    base = {"value": xs.shape[0] / (t2 - t0 - 0.0) / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"corner sub-cube with {xs.shape[0]} of {x.shape[0]} particles; FP64 oracle tree+lists+KIFMM, "
                      f"p={w['p']}, M={w['leaf_cap']} ({t2 - t0:.1f} s; operator precompute excluded)"}
    rng = np.random.default_rng(seed)
    idx = rng.choice(x.shape[0], size=min(n_targets, x.shape[0]), replace=False)
    pd, gd = O.direct(x, q, x[idx])
    return base, idx, pd, gd


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, as it stands, on a bounded sample of
    the same workload per step (rank 0 only)."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    w = WORKLOADS[args.workload]
    x, q, meta = make_inputs(w)
    lo = x.min(axis=0)
    side = (x.max(axis=0) - lo).max()
    frac = 0.1
    cut = side * frac ** (1.0 / 3.0)
    sel = np.all(x - lo < cut, axis=1)
    xs, qs = x[sel], q[sel]
    ops = O.operators(w["p"])

    def step():
        tree = O.sort_and_tree(xs, w["leaf_cap"], w["max_depth"])
        lst = O.lists(tree)
        O.kifmm(xs, qs, p=w["p"], tree=tree, lst=lst, ops=ops)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = xs.shape[0] / dt / 1e6
    cores = len(os.sched_getaffinity(0))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w["name"], "n": w["n"], "p": w["p"], "leaf_cap": w["leaf_cap"],
                      "parallelism": "host cores (OpenMP)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"corner sub-cube with {xs.shape[0]} of {x.shape[0]} particles per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2512_09478_gb300 import Plan
    dist = world > 1
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = WORKLOADS[args.workload]
    x, q, meta = make_inputs(w)
    n = x.shape[0]
    coef = 1.0 / EPS0
    xt = torch.tensor(x, dtype=torch.float32, device=dev)
    qt = torch.tensor(q, dtype=torch.float32, device=dev)
    plan = Plan(p=w["p"], leaf_cap=w["leaf_cap"], max_depth=w["max_depth"], precision=args.precision, coef=coef,
                n_max=n, dtype=torch.float32)
    pot = torch.empty(n, dtype=torch.float32, device=dev)
    grad = torch.empty(n, 3, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.set_sources(xt, qt)
        plan.evaluate(pot, grad)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    work = algorithmic_work(plan, w, n)
    plan.profile(True)
    plan.profile_read()
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evict the previous step's working set from L2 (not timed)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    prof = plan.profile_read()
    plan.profile(False)
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = t.item()
    ms_per_step = total_ms / args.steps
    value = world * n / (ms_per_step * 1e-3) / 1e6

    # end to end: pinned host inputs -> device -> set_sources + evaluate -> host outputs
    e2e = None
    if not args.no_e2e:
        hx = torch.tensor(x, dtype=torch.float32).pin_memory()
        hq = torch.tensor(q, dtype=torch.float32).pin_memory()
        hpot = torch.empty(n, dtype=torch.float32).pin_memory()
        hgrad = torch.empty(n, 3, dtype=torch.float32).pin_memory()
        dx = torch.empty_like(xt)
        dq = torch.empty_like(qt)

        def e2e_step():
            dx.copy_(hx, non_blocking=True)
            dq.copy_(hq, non_blocking=True)
            plan.set_sources(dx, dq)
            plan.evaluate(pot, grad)
            hpot.copy_(pot, non_blocking=True)
            hgrad.copy_(grad, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, 10))
        e_ms = 0.0
        for k in range(ke):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            torch.cuda.synchronize()
            e_ms += a.elapsed_time(b)
        e2e = {"value": world * n / (e_ms / ke * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(hx.numel() * 4 + hq.numel() * 4),
               "d2h_bytes_per_step": int(hpot.numel() * 4 + hgrad.numel() * 4)}

    if rank != 0:
        return
    # dominant stage and its roofline
    calls = prof["calls"]
    per_call = {k: prof["ms"][k] / max(calls[k], 1) for k in prof["ms"] if calls[k] > 0}
    dominant = max(per_call, key=lambda k: prof["ms"][k])
    peaks = measured_peaks()
    roof = roofline_for(dominant, per_call[dominant], work, args.precision, peaks)
    other = {s: roofline_for(s, per_call[s], work, args.precision, peaks) for s in ("m2l", "p2p", "tree")
             if s in per_call}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w["name"], "n": n, "p": w["p"], "leaf_cap": w["leaf_cap"],
                      "precision": args.precision, "parallelism": f"replicas x{world}" if world > 1 else "1 gpu",
                      "l2": "flushed between steps (256 MiB write)",
                      "rsa_solid_fraction": round(meta["solid_fraction"], 4),
                      "boxes": work["info"]["n_boxes"], "max_level": work["info"]["max_level"]},
           "roofline": roof, "stage_rooflines": other,
           "stages_ms": {k: round(v / args.steps, 4) for k, v in prof["ms"].items() if calls[k] > 0},
           "gpu_launches": int(prof["launches"]), "clocks": clk, "e2e": e2e}
    if not args.no_cpu_baseline:
        base, idx, pd, gd = cpu_baseline_leg(x, q, w, args.accuracy_targets)
        out["cpu_baseline"] = base
        p_gpu = pot.double().cpu().numpy()[idx] * EPS0  # back to Eq. 3 units for the comparison
        g_gpu = grad.double().cpu().numpy()[idx] * EPS0
        f_ref = -q[idx, None] * gd
        f_gpu = -q[idx, None] * g_gpu
        out["accuracy"] = {"targets": int(idx.size), "vs": "FP64 direct sum",
                           "rel_l2_pot": rel_l2(p_gpu, pd), "rel_l2_grad": rel_l2(g_gpu, gd),
                           "rel_l2_force": rel_l2(f_gpu, f_ref)}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if "RANK" in os.environ else 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
