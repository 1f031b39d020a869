#!/usr/bin/env python
"""Benchmark: KIFMM long-range force evaluation on one GB300 per rank.

One step = one pass of the whole hot path.  Default workload (c2): the
1M-sphere DEM Coulomb packing (RSA to solid fraction 0.4, radii U[0.5, 1.5]
mm, charges N(0, (1e-12 C)^2), p = 6, leaf cap 128, FP32 inputs/outputs);
a step is set_sources (bounding cube, Morton keys, radix sort, octree,
U/V/W/X lists) + evaluate (P2M, M2M, M2L, P2L, L2L, leaf pseudo-inverses,
L2P/M2P/P2P, scatter).  Other workloads:
  c3  200k rigid clumps x 4 charges: the step adds the clump force/torque reduce;
  c5  64 independent systems of 10k..200k particles: the tree is built once and
      each step replays one captured CUDA graph of update_sources + evaluate.

    python bench.py [--gpus N --steps K --warmup W] [--workload c2|c3|c5] [--impl reference]

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
    # p_accurate: the lowest surface order whose FP64 KIFMM meets rel-L2 <= 1e-5
    # on forces on this packing (4.0e-6 at p = 7 against 3.0e-5 at p = 6)
    "c2": dict(kind="rsa", name="dem-coulomb-rsa-1M", n=1_000_000, p=6, leaf_cap=128, max_depth=20, seed=1001,
               p_accurate=7),
    # 1/8 of C2: the same leaf occupancy (about 30 points) one level higher
    "c2-small": dict(kind="rsa", name="dem-coulomb-rsa-125k", n=125_000, p=6, leaf_cap=128, max_depth=20, seed=1001),
    "c2-64k": dict(kind="rsa", name="dem-coulomb-rsa-64k", n=65_536, p=6, leaf_cap=128, max_depth=20, seed=1001),
    "c3": dict(kind="clumps", name="rigid-clumps-200k-x4", n=800_000, clumps=200_000, p=6, leaf_cap=128,
               max_depth=20, seed=1002),
    "c4": dict(kind="plummer", name="gravity-plummer-4M", n=4_000_000, p=8, leaf_cap=128, max_depth=12, seed=1003,
               oracle_frac=0.03, ref_frac=0.005, compare="fp64"),
    "c5": dict(kind="batched", name="batched-64-systems-10k-200k", systems=64, p=6, leaf_cap=64, max_depth=20,
               seed=1004, ref_frac=0.1),
}
WORKLOADS["c2"]["compare"] = "fp32"


# DRAM bytes (read + write) of the dominant kernels per step on the 1M DEM
# packing (M2L: its one launch; leaf kernel: its three tile variants), from an
# ncu capture of the timed steps with the DRAM byte counters and the duration
# only (profiles/dram_traffic_c2_dem_coulomb_1M.md).  A figure is reported
# only while the kernel's sources are byte-identical to the ones captured
# (sha256 over the listed files); otherwise the roofline's traffic is null.
_M2L_SRC = ("paper_2512_09478_gb300/csrc/m2l_tc.cu", "paper_2512_09478_gb300/csrc/tc_ptx.cuh",
            "paper_2512_09478_gb300/csrc/common.cuh", "paper_2512_09478_gb300/csrc/internal.h")
_LEAF_SRC = ("paper_2512_09478_gb300/csrc/fmm.cu", "paper_2512_09478_gb300/csrc/common.cuh",
             "paper_2512_09478_gb300/csrc/internal.h")
TRAFFIC = {
    ("dem-coulomb-rsa-1M", "m2l"): (_M2L_SRC, "2930bb808ea1995153aa528a283826ff0089836c0692b1a886b3579915bdf02c", 96189952),
    ("dem-coulomb-rsa-1M", "p2p"): (_LEAF_SRC, "878cc63175916d94552a1ff20aace24ffec7bd61c66ecd4b34b2f350e9ae4b9d", 76453120),
}


def traffic_for(workload, stage):
    import hashlib
    ent = TRAFFIC.get((workload, stage))
    if ent is None:
        return None
    paths, sha, nbytes = ent
    m = hashlib.sha256()
    try:
        for path in paths:
            with open(os.path.join(ROOT, path), "rb") as f:
                m.update(f.read())
    except OSError:
        return None
    return nbytes if m.hexdigest() == sha else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=os.environ.get("KIFMM_BENCH_PRECISION", "mixed_fp16"))
    ap.add_argument("--accuracy-targets", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed tile shapes (default: the library tunes them on the first, untimed, evaluate)")
    ap.add_argument("--m2l-eps-compare", type=float, default=1e-5,
                    help="also time the same step with the compressed M2L at this eps (0: skip)")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--m2l-variant", default=None,
                    help="pin the tensor-core M2L variant as producers,tiles,stages (e.g. 2,2,3) instead of tuning it")
    ap.add_argument("--compare", default="auto",
                    help="also time this precision on the same workload (auto: the workload's comparison "
                         "path, none: skip)")
    return ap.parse_args()


def make_inputs(w):
    """Positions, charges and metadata of a workload.  Coulomb workloads carry
    SI charges (coef 1/eps0); the batched workload is in Eq. 3 units."""
    from workloads import generators as G
    if w["kind"] == "rsa":
        x, q, meta = G.dem_coulomb(w["n"], w["seed"])
        meta.update(coef=1.0 / EPS0, offsets=[0, len(x)])
    elif w["kind"] == "clumps":
        x, q, off, centres = G.clumps(w["clumps"], w["seed"])
        meta = {"clump_offsets": off, "centres": centres, "coef": 1.0 / EPS0, "offsets": [0, len(x)]}
    elif w["kind"] == "plummer":
        # G = 1: masses as charges with coef -4 pi (Eq. 4 read as attractive)
        x, q = G.plummer(w["n"], w["seed"])
        meta = {"coef": -4.0 * np.pi, "offsets": [0, len(x)]}
    else:
        x, q, off = G.batched(w["systems"], w["seed"])
        meta = {"coef": 1.0, "offsets": [int(v) for v in off]}
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
    near-field pairs (sum over leaves of n_B times the U-list source count,
    minus the self pairs), tree-build bytes."""
    info = plan.tree_info()
    ns = 6 * (w["p"] - 1) ** 2 + 2
    m2l_flops = 2.0 * ns * ns * info["n_v"]
    t = plan.tree()
    ptr, idx = plan.list("U")
    cnt = t["count"]
    src = np.add.reduceat(cnt[idx], ptr[:-1]) if idx.size else np.zeros(len(cnt))
    src = np.where(np.diff(ptr) > 0, src, 0)
    pairs = float(np.sum(cnt * src) - n)
    # the leaf kernel also evaluates n_s pseudo-sources per target for L2P and
    # per W-list box for M2P
    wptr, _ = plan.list("W")
    leaf_pairs = pairs + ns * float(n) + ns * float(np.sum(cnt * np.diff(wptr)))
    # tree: bbox read 16 B, keys read 12 B + write 16 B, each radix pass the
    # library ran x (read 12 B for the histogram + read 12 B and write 12 B in
    # the scatter), gather 36 B
    tree_bytes = n * (16 + 28 + info["sort_passes"] * 36 + 36)
    return {"m2l_flops": m2l_flops, "p2p_pairs": pairs, "leaf_pairs": leaf_pairs, "tree_bytes": float(tree_bytes),
            "info": info}


def roofline_for(stage, ms_per_call, work, precision, peaks):
    hbm, bf16, bf16_s, kind = peaks
    if stage == "m2l":
        flops = work["m2l_flops"]
        ach = flops / (ms_per_call * 1e-3) / 1e12
        if precision.startswith("mixed"):
            # a ~1 ms kernel timed on its own launch: the burst peak (FP16 runs at the BF16 rate)
            return {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                    "traffic": None, "kernel": "k_m2l_tc",
                    "peak_source": f"{kind} bf16 burst (fp16 same rate); 3 split products, 1 counted"}
        return {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "k_ggemm<GatherM2L>",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    if stage == "p2p":
        flops = 20.0 * work["leaf_pairs"]
        ach = flops / (ms_per_call * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "k_leaf_all",
                "pairs": {"p2p": work["p2p_pairs"], "l2p_m2p": work["leaf_pairs"] - work["p2p_pairs"]},
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz; 20 flop per (pseudo-)source pair"}
    if stage == "tree":
        gbs = work["tree_bytes"] / (ms_per_call * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": None, "kernel": "set_sources", "peak_source": f"{kind} copy bandwidth"}
    return None


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_sample(x, q, meta, w, frac):
    """A bounded sample of the workload for the CPU legs: the corner sub-cube
    holding ``frac`` of the particles (c2, c3), or the leading systems holding
    about ``frac`` of them (c5)."""
    if w["kind"] == "batched":
        off = meta["offsets"]
        k = max(1, int(np.searchsorted(np.asarray(off[1:]), frac * off[-1])))
        return [(x[off[s]:off[s + 1]], q[off[s]:off[s + 1]]) for s in range(k)], f"systems 0..{k - 1}"
    if w["kind"] == "plummer":
        # the central cube holding about frac of the particles
        r = np.abs(x - np.median(x, axis=0)).max(axis=1)
        sel = r <= np.quantile(r, frac)
        return [(x[sel], q[sel])], "central cube"
    lo = x.min(axis=0)
    side = (x.max(axis=0) - lo).max()
    if frac >= 1.0:
        return [(x, q)], "whole workload"
    sel = np.all(x - lo < side * frac ** (1.0 / 3.0), axis=1)
    return [(x[sel], q[sel])], "corner sub-cube"


def cpu_baseline_leg(x, q, meta, w, n_targets, seed=0, frac=None):
    """CPU leg (the only place the benchmark runs the oracle): time the FP64
    oracle KIFMM on a bounded sample of the workload, and compute FP64
    direct-sum reference values on sampled targets for the accuracy figures."""
    from oracle import oracle as O
    O.build()
    frac = w.get("oracle_frac", 1.0) if frac is None else frac
    parts, what = _oracle_sample(x, q, meta, w, frac)
    ops = O.operators(w["p"])
    t0 = time.perf_counter()
    n_s = 0
    for xs, qs in parts:
        tree = O.sort_and_tree(xs, w["leaf_cap"], w["max_depth"])
        lst = O.lists(tree)
        O.kifmm(xs, qs, p=w["p"], tree=tree, lst=lst, ops=ops)
        n_s += xs.shape[0]
    t2 = time.perf_counter()
    cores = len(os.sched_getaffinity(0))
    base = {"value": n_s / (t2 - t0) / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what}: {n_s} of {x.shape[0]} particles; FP64 oracle tree+lists+KIFMM, "
                      f"p={w['p']}, M={w['leaf_cap']} ({t2 - t0:.1f} s; operator precompute excluded)"}
    rng = np.random.default_rng(seed)
    ref = {}
    # The accuracy reference sums over the FP32 inputs the device received, so
    # the figures measure the method, not the rounding of the caller's data.
    x = x.astype(np.float32).astype(np.float64)
    q = q.astype(np.float32).astype(np.float64)
    if w["kind"] == "clumps":
        off, cen = meta["clump_offsets"], meta["centres"].astype(np.float32).astype(np.float64)
        cl = np.sort(rng.choice(len(cen), size=min(256, len(cen)), replace=False))
        idx = np.concatenate([np.arange(off[c], off[c + 1]) for c in cl])
        pd, gd = O.direct(x, q, x[idx])
        loc = np.concatenate([[0], np.cumsum([off[c + 1] - off[c] for c in cl])])
        F, T = O.clump_reduce(x[idx], q[idx], gd, loc, cen[cl])
        ref.update(clumps=cl, F=F, T=T)
    elif w["kind"] == "batched":
        off = meta["offsets"]
        idx_l, pd_l, gd_l = [], [], []
        for s in rng.choice(len(off) - 1, size=4, replace=False):
            a, b = off[s], off[s + 1]
            t = a + rng.choice(b - a, size=min(512, b - a), replace=False)
            pd_s, gd_s = O.direct(x[a:b], q[a:b], x[t])
            idx_l.append(t)
            pd_l.append(pd_s)
            gd_l.append(gd_s)
        idx, pd, gd = np.concatenate(idx_l), np.concatenate(pd_l), np.concatenate(gd_l)
    else:
        idx = rng.choice(x.shape[0], size=min(n_targets, x.shape[0]), replace=False)
        pd, gd = O.direct(x, q, x[idx])
    ref.update(idx=idx, pot=pd, grad=gd)
    return base, ref


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, as it stands, on the same workload
    per step (rank 0 only): the whole workload for the DEM and clump cases
    (about 7 s per step on 16 cores at 1M), a bounded sample where that would
    take minutes per step (4M gravity, 64 batched systems)."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    w = WORKLOADS[args.workload]
    x, q, meta = make_inputs(w)
    parts, what = _oracle_sample(x, q, meta, w, w.get("ref_frac", 1.0))
    ops = O.operators(w["p"])
    n_s = sum(p[0].shape[0] for p in parts)

    def step():
        for xs, qs in parts:
            tree = O.sort_and_tree(xs, w["leaf_cap"], w["max_depth"])
            lst = O.lists(tree)
            O.kifmm(xs, qs, p=w["p"], tree=tree, lst=lst, ops=ops)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = n_s / dt / 1e6
    cores = len(os.sched_getaffinity(0))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w["name"], "n": int(x.shape[0]), "systems": len(meta["offsets"]) - 1,
                      "p": w["p"], "leaf_cap": w["leaf_cap"], "parallelism": "host cores (OpenMP)",
                      "same_workload": n_s == int(x.shape[0])},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{what}: {n_s} of {x.shape[0]} particles per step"},
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
    n_job = x.shape[0]
    coef, offsets = meta["coef"], meta["offsets"]
    sharded = w["kind"] == "batched" and world > 1
    if sharded:
        # whole systems per rank, largest first onto the least-loaded rank; no collective on the data path
        from paper_2512_09478_gb300 import shard
        assignment = shard.assign_largest_first(np.diff(offsets), world)
        x, q, offsets = shard.local_batch(x, q, offsets, assignment[rank])
    n_sys_job = len(meta["offsets"]) - 1
    meta = dict(meta, offsets=offsets)
    n = x.shape[0]
    n_sys = len(offsets) - 1
    xt = torch.tensor(x, dtype=torch.float32, device=dev)
    qt = torch.tensor(q, dtype=torch.float32, device=dev)
    plan = Plan(p=w["p"], leaf_cap=w["leaf_cap"], max_depth=w["max_depth"], precision=args.precision, coef=coef,
                n_max=n, n_systems_max=n_sys, dtype=torch.float32, autotune=not args.no_autotune)
    if args.m2l_variant:
        plan.set_m2l_tuning(*[int(v) for v in args.m2l_variant.split(",")])
    pot = torch.empty(n, dtype=torch.float32, device=dev)
    grad = torch.empty(n, 3, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    clumps = w["kind"] == "clumps"
    if clumps:
        coff = torch.tensor(meta["clump_offsets"], device=dev)
        cref = torch.tensor(meta["centres"], dtype=torch.float32, device=dev)
        force = torch.empty(len(meta["centres"]), 3, dtype=torch.float32, device=dev)
        torque = torch.empty_like(force)

    # Every timed step runs the whole path (tree, lists, evaluation) on new
    # positions: the steps alternate the packing and its mirror image
    # (x -> lo + hi - x, the same workload).  The plan builds its lists on
    # every set_sources; keeping them when the boxes are unchanged
    # (reuse_lists) is timed on its own below.
    lo, hi = xt.min(0).values, xt.max(0).values
    xs_alt = (xt, (lo + hi) - xt)
    cref_alt = (cref, (lo + hi) - cref) if clumps else (None, None)

    def eager_step(k=0):
        xk = xs_alt[k & 1]
        plan.set_sources(xk, qt, offsets)
        plan.evaluate(pot, grad)
        if clumps:
            plan.clump_reduce(coff, xk, qt, grad, cref_alt[k & 1], force, torque)

    graph = None
    if w["kind"] == "batched":
        # tree built once; each step refreshes the particles and evaluates, as one graph
        plan.set_sources(xt, qt, offsets)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):
                plan.update_sources(xt, qt)
                plan.evaluate(pot, grad)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        l0 = plan.profile_read()["launches"]
        with torch.cuda.graph(graph):
            plan.update_sources(xt, qt)
            plan.evaluate(pot, grad)
        launches_per_replay = plan.profile_read()["launches"]

        def step(k=0):
            graph.replay()
    else:
        step = eager_step

    for k in range(max(args.warmup, 3)):
        step(k)
    torch.cuda.synchronize()
    work = algorithmic_work(plan, w, n)
    if graph is None:
        plan.profile(True)
    plan.profile_read()
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if args.profile_region:
        torch.cuda.profiler.start()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evict the previous step's working set from L2 (not timed)
        evs[k][0].record(stream)
        step(k)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if args.profile_region:
        torch.cuda.profiler.stop()
    clk = clocks.stop()
    if dist:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    if graph is None:
        prof = plan.profile_read()
        plan.profile(False)
        launches = int(prof["launches"])
        prof_note = "stage events recorded in the timed steps"
        # untimed: both halves of the alternation built their lists, and the
        # outputs (checked for accuracy below) are the packing's own
        rebuilt = []
        for k in (1, 0):
            eager_step(k)
            rebuilt.append(plan.tree_info()["lists_reused"] == 0)
        torch.cuda.synchronize()
    else:
        launches = int(launches_per_replay) * args.steps
        # stage split from an uncaptured pass of the same evaluate (events cannot be read per replay)
        plan.profile(True)
        plan.profile_read()
        for _ in range(args.steps):
            plan.update_sources(xt, qt)
            plan.evaluate(pot, grad)
        prof = plan.profile_read()
        plan.profile(False)
        prof_note = "stage events from uncaptured passes of the same update_sources + evaluate"
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = t.item()
    ms_per_step = total_ms / args.steps
    units = n_job if sharded else world * n  # particles all ranks processed per step
    value = units / (ms_per_step * 1e-3) / 1e6

    # end to end through the public API: pinned host inputs -> device -> step -> host outputs
    e2e = None
    if not args.no_e2e:
        hxs = (xt.cpu().pin_memory(), xs_alt[1].cpu().pin_memory())   # the packing and its mirror image
        hq = torch.tensor(q, dtype=torch.float32).pin_memory()
        hpot = torch.empty(n, dtype=torch.float32).pin_memory()
        hgrad = torch.empty(n, 3, dtype=torch.float32).pin_memory()
        dx = torch.empty_like(xt)
        dq = torch.empty_like(qt)

        def e2e_step(k):
            dx.copy_(hxs[k & 1], non_blocking=True)
            dq.copy_(hq, non_blocking=True)
            plan.set_sources(dx, dq, offsets)
            plan.evaluate(pot, grad)
            if clumps:
                plan.clump_reduce(coff, dx, dq, grad, cref_alt[k & 1], force, torque)
            hpot.copy_(pot, non_blocking=True)
            hgrad.copy_(grad, non_blocking=True)

        for k in range(2):
            e2e_step(k)
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, 10))
        e_ms = 0.0
        for k in range(ke):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step(k)
            b.record(stream)
            torch.cuda.synchronize()
            e_ms += a.elapsed_time(b)
        if dist:
            t = torch.tensor([e_ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e_ms = t.item()
        e2e = {"value": units / (e_ms / ke * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(hxs[0].numel() * 4 + hq.numel() * 4),
               "d2h_bytes_per_step": int(hpot.numel() * 4 + hgrad.numel() * 4),
               "step": "set_sources + evaluate" + (" + clump_reduce" if clumps else "")}

    # second number: the tree reused across steps (update_sources + evaluate),
    # the long-range stride / reuse case; same L2 flush and events
    # untimed: the packing's own tree and outputs again (e2e may end on the
    # mirror image; a captured graph was recorded on this tree)
    eager_step(0)
    torch.cuda.synchronize()

    reuse = None
    if graph is None:
        def reuse_step():
            plan.update_sources(xt, qt)
            plan.evaluate(pot, grad)
            if clumps:
                plan.clump_reduce(coff, xt, qt, grad, cref, force, torque)

        for _ in range(3):
            reuse_step()
        torch.cuda.synchronize()
        kr = max(3, min(args.steps, 20))
        r_ms = 0.0
        for k in range(kr):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            reuse_step()
            b.record(stream)
            torch.cuda.synchronize()
            r_ms += a.elapsed_time(b)
        if dist:
            t = torch.tensor([r_ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            r_ms = t.item()
        reuse = {"value": units / (r_ms / kr * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": r_ms / kr, "steps": kr,
                 "step": "update_sources + evaluate" + (" + clump_reduce" if clumps else "") + " (tree frozen)"}

        # third number: refresh_sources (the device-side leaf test, one host
        # sync, then the kept tree's update) on positions jittered by 1e-6 of
        # the domain, alternating with the originals
        ext = (xt.max(0).values - xt.min(0).values).max()
        gj = torch.Generator(device=dev)
        gj.manual_seed(7)
        xj = xt + (torch.rand(xt.shape, generator=gj, device=dev, dtype=xt.dtype) - 0.5) * (2e-6 * ext)
        kept = 0

        def refresh_step(k):
            nonlocal kept
            kept += int(plan.refresh_sources(xj if k & 1 else xt, qt))
            plan.evaluate(pot, grad)
            if clumps:
                plan.clump_reduce(coff, xt, qt, grad, cref, force, torque)

        for k in range(3):
            refresh_step(k)
        torch.cuda.synchronize()
        kept = 0
        f_ms = 0.0
        for k in range(kr):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            refresh_step(k)
            b.record(stream)
            torch.cuda.synchronize()
            f_ms += a.elapsed_time(b)
        if dist:
            t = torch.tensor([f_ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            f_ms = t.item()
        kept_timed = kept
        # untimed: the outputs (checked for accuracy below) must again be those
        # of the unjittered positions
        refresh_step(0)
        torch.cuda.synchronize()
        reuse["refresh"] = {"value": units / (f_ms / kr * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": f_ms / kr,
                            "steps": kr, "tree_kept": kept_timed,
                            "step": "refresh_sources (skin 0.05, jitter 1e-6 of the domain) + evaluate"}

        # fourth number: set_sources on the same jittered alternation with a
        # reuse_lists plan; the tree is rebuilt every step and its lists are
        # kept when the boxes came out the same (own outputs: the accuracy
        # check below reads the benchmarked plan's)
        lplan = Plan(p=w["p"], leaf_cap=w["leaf_cap"], max_depth=w["max_depth"], precision=args.precision,
                     coef=coef, n_max=n, n_systems_max=n_sys, dtype=torch.float32, autotune=not args.no_autotune,
                     reuse_lists=True)
        pot_l, grad_l = torch.empty_like(pot), torch.empty_like(grad)
        if clumps:
            force_l, torque_l = torch.empty_like(force), torch.empty_like(torque)

        def lists_step(k):
            xk = xj if k & 1 else xt
            lplan.set_sources(xk, qt, offsets)
            lplan.evaluate(pot_l, grad_l)
            if clumps:
                lplan.clump_reduce(coff, xk, qt, grad_l, cref, force_l, torque_l)

        for k in range(3):
            lists_step(k)
        torch.cuda.synchronize()
        l_ms, kept_l = 0.0, 0
        for k in range(kr):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lists_step(k)
            b.record(stream)
            kept_l += lplan.tree_info()["lists_reused"]
            torch.cuda.synchronize()
            l_ms += a.elapsed_time(b)
        if dist:
            t = torch.tensor([l_ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            l_ms = t.item()
        torch.cuda.synchronize()
        lplan.close()
        reuse["lists_kept"] = {"value": units / (l_ms / kr * 1e-3) / 1e6, "unit": UNIT,
                               "ms_per_step": l_ms / kr, "steps": kr, "lists_kept": kept_l,
                               "step": "set_sources (reuse_lists plan; jitter 1e-6 of the domain, alternating) "
                                       "+ evaluate"}

    if rank != 0:
        return
    calls = prof["calls"]
    per_call = {k: prof["ms"][k] / max(calls[k], 1) for k in prof["ms"] if calls[k] > 0}
    # dominant single kernel: the M2L (k_m2l_tc / gathered GEMM) or the leaf kernel
    dominant = max((k for k in per_call if k in ("m2l", "p2p")), key=lambda k: prof["ms"][k])
    peaks = measured_peaks()
    roof = roofline_for(dominant, per_call[dominant], work, args.precision, peaks)
    other = {s: roofline_for(s, per_call[s], work, args.precision, peaks) for s in ("m2l", "p2p", "tree")
             if s in per_call}
    for s_name, r in list(other.items()) + [(dominant, roof)]:
        if r is not None and args.precision == "mixed_fp16":
            r["traffic"] = traffic_for(w["name"], s_name)
    cfg = {"workload": w["name"], "n": n_job, "systems": n_sys_job, "p": w["p"], "leaf_cap": w["leaf_cap"],
           "precision": args.precision,
           "parallelism": ("1 gpu" if world == 1 else
                           f"systems sharded over {world} gpus (largest first)" if sharded else f"replicas x{world}"),
           "l2": "flushed between steps (256 MiB write)", "boxes": work["info"]["n_boxes"],
           "max_level": work["info"]["max_level"],
           "step": ("graph replay of update_sources + evaluate (tree frozen)" if graph is not None else
                    "set_sources + evaluate" + (" + clump_reduce" if clumps else ""))}
    if graph is None:
        cfg["positions"] = "steps alternate the packing and its mirror image (x -> lo + hi - x)"
        cfg["lists_rebuilt_every_step"] = all(rebuilt)
    if "solid_fraction" in meta:
        cfg["rsa_solid_fraction"] = round(meta["solid_fraction"], 4)
    tun = plan.tuning()
    cfg["tiles"] = {"autotuned": tun["tuned_leaf"], "m2l_stages": tun["m2l_stages"],
                    "m2l_producer_warps": tun["m2l_producers"], "m2l_tiles_per_cta": tun["m2l_tiles"],
                    "leaf_tpl_x_groups_per_8_targets": ["%dx%d" % t for t in tun["leaf_tiles"]]}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "strong" if sharded else "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
           "roofline": roof, "stage_rooflines": other,
           "stages_ms": {k: round(v / max(calls[k], 1) * (calls[k] / args.steps), 4)
                         for k, v in prof["ms"].items() if calls[k] > 0},
           "stages_note": prof_note, "gpu_launches": launches, "clocks": clk, "e2e": e2e, "tree_reuse": reuse}
    ref = None
    if not args.no_cpu_baseline:
        base, ref = cpu_baseline_leg(x, q, meta, w, args.accuracy_targets)
        out["cpu_baseline"] = base
        out["accuracy"] = accuracy_of(ref, q, coef, pot, grad, force if clumps else None,
                                      torque if clumps else None)
    cmp_prec = w.get("compare") if args.compare == "auto" else (None if args.compare == "none" else args.compare)
    if cmp_prec and cmp_prec != args.precision:
        out["compare"] = compare_leg(args, w, cmp_prec, xt, qt, offsets, coef, n, n / (ms_per_step * 1e-3) / 1e6, stream, flush,
                                     clumps, (coff, cref) if clumps else None, ref, q)
    if w.get("p_accurate") and args.precision == "mixed_fp16":
        # the lowest surface order whose FP64 method error on this packing meets
        # the metric's rel-L2 <= 1e-5 for forces: the benchmarked path and the
        # plain FP32 path at that order, with their accuracy
        pa = w["p_accurate"]
        mixed_a = compare_leg(args, w, "mixed_fp16", xt, qt, offsets, coef, n, 0.0, stream, flush, clumps,
                              (coff, cref) if clumps else None, ref, q, p=pa)
        fp32_a = compare_leg(args, w, "fp32", xt, qt, offsets, coef, n, 0.0, stream, flush, clumps,
                             (coff, cref) if clumps else None, ref, q, p=pa)
        for leg in (mixed_a, fp32_a):
            leg.pop("speedup_of_benchmarked", None)
            leg.pop("m2l_ms", None)
        out["at_accuracy"] = {"p": pa, "value": mixed_a["value"], "unit": UNIT,
                              "ms_per_step": mixed_a["ms_per_step"], "precision": "mixed_fp16",
                              "accuracy": mixed_a.get("accuracy"), "fp32": fp32_a,
                              "speedup_vs_fp32": mixed_a["value"] / fp32_a["value"],
                              "step": "set_sources + evaluate"}
    if args.m2l_eps_compare > 0 and args.precision == "mixed_fp16":
        out["m2l_compressed"] = compare_leg(args, w, "mixed_fp16", xt, qt, offsets, coef, n,
                                            n / (ms_per_step * 1e-3) / 1e6, stream, flush, clumps,
                                            (coff, cref) if clumps else None, ref, q, m2l_eps=args.m2l_eps_compare)
    print(json.dumps(out), flush=True)


def accuracy_of(ref, q, coef, pot, grad, force=None, torque=None):
    """rel-L2 of the sampled outputs against the FP64 direct sums in ``ref``."""
    idx = ref["idx"]
    p_gpu = pot.double().cpu().numpy()[idx] / coef  # back to Eq. 3 units for the comparison
    g_gpu = grad.double().cpu().numpy()[idx] / coef
    q64 = q.astype(np.float32).astype(np.float64)
    acc = {"targets": int(idx.size), "vs": "FP64 direct sum over the FP32 inputs",
           "rel_l2_pot": rel_l2(p_gpu, ref["pot"]), "rel_l2_grad": rel_l2(g_gpu, ref["grad"]),
           "rel_l2_force": rel_l2(-q64[idx, None] * g_gpu, -q64[idx, None] * ref["grad"])}
    if force is not None:
        cl = ref["clumps"]
        acc["clumps"] = int(cl.size)
        acc["rel_l2_clump_force"] = rel_l2(force.double().cpu().numpy()[cl] / coef, ref["F"])
        acc["rel_l2_clump_torque"] = rel_l2(torque.double().cpu().numpy()[cl] / coef, ref["T"])
    return acc


def compare_leg(args, w, prec, xt, qt, offsets, coef, n, value, stream, flush, clumps, cl, ref, q, m2l_eps=0.0,
                p=None):
    """The same step with another precision of the library (plain FP32 SIMT
    M2L for the DEM workload, the FP64 path for gravity), or with the
    compressed M2L (m2l_eps > 0): its throughput, the speedup of the
    benchmarked configuration over it, and its accuracy."""
    import torch
    from paper_2512_09478_gb300 import Plan
    dt = torch.float64 if prec == "fp64" else torch.float32
    p = w["p"] if p is None else p
    plan = Plan(p=p, leaf_cap=w["leaf_cap"], max_depth=w["max_depth"], precision=prec, coef=coef,
                n_max=n, n_systems_max=len(offsets) - 1, dtype=dt, autotune=not args.no_autotune,
                m2l_eps=m2l_eps)
    x2, q2 = xt.to(dt), qt.to(dt)
    pot = torch.empty(n, dtype=dt, device=xt.device)
    grad = torch.empty(n, 3, dtype=dt, device=xt.device)
    if clumps:
        coff, cref = cl
        cref = cref.to(dt)
        force = torch.empty(cref.shape[0], 3, dtype=dt, device=xt.device)
        torque = torch.empty_like(force)

    # the packing and its mirror image in turn, as in the benchmarked step
    lo, hi = x2.min(0).values, x2.max(0).values
    xs_alt = (x2, (lo + hi) - x2)
    cref_alt = (cref, (lo + hi) - cref) if clumps else (None, None)

    def step(i):
        plan.set_sources(xs_alt[i & 1], q2, offsets)
        plan.evaluate(pot, grad)
        if clumps:
            plan.clump_reduce(coff, xs_alt[i & 1], q2, grad, cref_alt[i & 1], force, torque)

    for i in range(3):
        step(i)
    torch.cuda.synchronize()
    k = 3 if prec == "fp64" else max(3, min(args.steps, 10))
    ms = 0.0
    for i in range(k):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(i)
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
    step(0)   # untimed: the packing's own outputs for the accuracy check
    torch.cuda.synchronize()
    v = n / (ms / k * 1e-3) / 1e6
    res = {"precision": prec, "p": p, "value": v, "unit": UNIT, "ms_per_step": ms / k, "steps": k,
           "speedup_of_benchmarked": value / v, "io_dtype": "f64" if prec == "fp64" else "f32"}
    if m2l_eps > 0:
        res["m2l_eps"] = m2l_eps
        res["m2l_ranks_out_in"] = list(plan.tuning()["m2l_ranks"])
    if ref is not None:
        res["accuracy"] = accuracy_of(ref, q, coef, pot, grad, force if clumps else None,
                                      torque if clumps else None)
    return res


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
