#!/usr/bin/env python3
"""Benchmark of the GB300 falcON step: particle-steps/s on the paper-shaped disk.

Workload (one "step" = one full SBAB1 step of Sect. 4.1 through ncorp_step:
half kick, tree collision search, drift, key sort + octree build, climb with
P2M/M2M, dual-tree walk, M2L, descent, L2P + near field + external forces,
half kick): one synthetic moonlet disk of N = 1e5 (seed 2, the recipe of
paper_2310_20374_gb300/diskgen.py), falcON p = 6, theta_min = 0.5,
dt = 1e-3, mixed precision (FP32 expansions and near field, FP64 state,
geometry, keys and collision test).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {ncorp,reference}]

N > 1 runs under torchrun: every rank integrates its own replica disk (the
step has no exchange between disks), the timed region is bracketed by
barriers and the slowest rank's time is used.  --impl reference times the
CPU oracle (oracle/, plain C FP64) on the host, rank 0 only.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s, falcON p=6 gravity+collisions; p50/p99 step latency mixed-N"
UNIT = "particle-steps/s"
# DRAM bytes (read + write) of one k_eval launch, from ncu captures of the current
# kernel (dram__bytes_read.sum + dram__bytes_write.sum, mixed precision, leaf size
# 64), keyed by (N, p, theta_min); entries are removed whenever the kernel changes,
# until it is captured again.  Other workloads report null.  Empty: the captures
# (5.54e6 at N = 1e5, p = 6; 50.3e6 at N = 1e6, p = 4) were taken with the kernel
# at eight blocks per SM, before its launch bound became six.
EVAL_DRAM_BYTES_PER_LAUNCH = {}


def eval_traffic(n, p, theta, precision, leaf_size):
    if precision != "mixed" or leaf_size != 64 or THRESHOLDS_OVERRIDE:
        return None
    return EVAL_DRAM_BYTES_PER_LAUNCH.get((n, p, theta))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ncorp", choices=["ncorp", "reference"])
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--p", type=int, default=6)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--leaf-size", type=int, default=0, help="disk: leaf size s (0: the default for p)")
    ap.add_argument("--thresholds", default="", help="disk: N_cs,N_cc_pre,N_cc_post of the gravity walk at --p")
    ap.add_argument("--fused-walk", type=int, default=0, choices=[0, 1],
                    help="disk: one walk per step for gravity and the next step's collision pairs")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--resolve-f", type=float, default=0.0,
                    help="disk: 0 = colliding pairs reported (default); 1..2 = resolved with this f (Sect. 5)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="disk: time only the requested precision on workload 2 (no FP64/mixed twin, no workload 3)")
    ap.add_argument("--steps3", type=int, default=100, help="disk: timed steps of workload 3 (N = 1e6)")
    ap.add_argument("--workload", default="disk", choices=["disk", "ensemble", "serving", "standard"],
                    help="disk: one disk per GPU (default); ensemble: 64 disks of mixed size per GPU in one batch; "
                         "serving: disks arriving as a Poisson stream, each integrated for 100 steps")
    ap.add_argument("--serve-seconds", type=float, default=30.0, help="serving: length of the arrival window")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="serving: requests per second")
    ap.add_argument("--serve-budget", type=float, default=0.5,
                    help="serving: the batch's device-memory budget as a fraction of the free memory at the start")
    ap.add_argument("--serve-pool", type=int, default=600,
                    help="serving: distinct initial disks (later requests reuse them; 0: one per request)")
    ap.add_argument("--tick-steps", type=int, default=10, help="serving: most steps per ncorp_batch_run")
    ap.add_argument("--serve-log", default="",
                    help="serving: file to which the loop appends one JSON line per run and tick (flushed each time)")
    ap.add_argument("--steps4", type=int, default=50, help="default run: steps of the 64-disk ensemble")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), ws, int(os.environ.get("LOCAL_RANK", "0"))


def slowest_rank(dist, value, world, device="cuda"):
    """Max over the ranks of a per-rank time: the replicas' aggregate runs as long as the slowest rank."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, steps, world, seconds):
    """Whole-job particle-steps/s of `world` independent replicas timed by the slowest one."""
    return units_per_rank * steps * world / seconds


# Algorithmic work per stage of one step (the measurement table of the scope:
# bytes a stage must move per moonlet, or FLOPs per unit it must compute).
# HBM-bound stages: kdk = kick-drift (x, v, a read: 72 B; x, v written: 48 B)
# and the scatter of the new state to the caller's order (52 B read, 48 B
# written); sort = keys (24 B read, 24 B written), the nearly-sorted merge of
# (key, index) (36 B), the gather to tree order (~196 B); build = 16 B;
# climb = the moonlet pass of the geometry and of P2M (2 x 32 B); eval = L2P,
# near sums, external force and closing kick (~152 B).  ALU-bound stages, in
# the method's own units whatever the kernels evaluate: m2l = FLOPs per
# unordered well-separated pair (one D(R), both directions), by p; near =
# 30 FLOPs per unordered moonlet pair of the direct sums (one rsqrt); collide
# = 30 FLOPs per candidate pair of the collision test.  walk and descend are
# latency-bound chains (dependent generations; ancestor translations per
# leaf): no throughput bound.
STAGE_BYTES_PER_MOONLET = {"kdk": 220.0, "sort": 280.0, "build": 16.0, "climb": 64.0, "eval": 152.0}
M2L_FLOP_PER_PAIR = {3: 250.0, 4: 700.0, 6: 3200.0}
NEAR_FLOP_PER_PAIR = 30.0
COLLIDE_FLOP_PER_TEST = 30.0


FP32_PEAK_TFLOPS = None   # measured at the start of the run: the collision prefilters run in FP32 in both forms


def stage_rooflines(stage_ms, n, p, m2l_pairs, p2p_inter, col_tests, hbm_gbs, alu_tflops):
    """Per-stage fraction of roofline from per-step stage times (ms) and the step's work counters;
    alu_tflops is the measured FMA peak of the precision the near field and M2L run in (the collision
    prefilter is taken against the FP32 peak in both forms)."""
    out = {}
    for st, bpm in STAGE_BYTES_PER_MOONLET.items():
        ms = stage_ms.get(st, 0.0)
        if ms > 0:
            gbs = bpm * n / (ms * 1e-3) / 1e9
            out[st] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_gbs, "unit": "GB/s",
                       "frac": round(gbs / hbm_gbs, 4), "bytes_per_moonlet": bpm}
    flops = {"near": NEAR_FLOP_PER_PAIR * p2p_inter, "collide": COLLIDE_FLOP_PER_TEST * col_tests}
    if p in M2L_FLOP_PER_PAIR:
        flops["m2l"] = M2L_FLOP_PER_PAIR[p] * m2l_pairs
    for st, f in flops.items():
        ms = stage_ms.get(st, 0.0)
        if ms > 0 and f > 0:
            tf = f / (ms * 1e-3) / 1e12
            pk = FP32_PEAK_TFLOPS if (st == "collide" and FP32_PEAK_TFLOPS) else alu_tflops
            out[st] = {"bound": "alu", "achieved": round(tf, 3), "peak": round(pk, 2), "unit": "TFLOP/s",
                       "frac": round(tf / pk, 4), "flops_per_step": f}
    for st in ("walk", "descend"):
        if stage_ms.get(st, 0.0) > 0:
            out[st] = {"bound": "latency", "ms": round(stage_ms[st], 4)}
    return out


def measured_hbm_gbs(default=6800.0):
    """Measured copy bandwidth of the GB300s, else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError, TypeError):
        return default


def leaf_size_for(p):
    return 64 if p >= 4 else 32


def leaf_size_of(a, n, p):
    """Leaf size of a run of N = n at order p: --leaf-size for the main workload, else the default for p."""
    return a.leaf_size if a.leaf_size > 0 and n == a.n else leaf_size_for(p)


THRESHOLDS_OVERRIDE = {}   # p -> [N_cs, N_cc,pre, N_cc,post] given with --thresholds


def thresholds_for(p):
    if p in THRESHOLDS_OVERRIDE:
        return list(THRESHOLDS_OVERRIDE[p])
    return [256, 256, 512] if p >= 6 else [64, 8, 64]


def direct_sample_errors(pos, mass, acc_mutual, k=1000, seed=0):
    """Median and 99th percentile over a seeded sample of k moonlets of |a - a_direct| / |a_direct|, the
    mutual accelerations against FP64 direct summation (G = 1; coincident pairs contribute nothing)."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(pos), size=min(k, len(pos)), replace=False)
    ref = np.zeros((len(idx), 3))
    for j0 in range(0, len(pos), 20000):
        src, m = pos[j0:j0 + 20000], mass[j0:j0 + 20000]
        d = src[None, :, :] - pos[idx][:, None, :]
        r2 = np.einsum("ijk,ijk->ij", d, d)
        with np.errstate(divide="ignore"):
            w = np.where(r2 > 0.0, m[None, :] / (r2 * np.sqrt(r2)), 0.0)
        ref += np.einsum("ij,ijk->ik", w, d)
    diff = np.linalg.norm(acc_mutual[idx] - ref, axis=1)
    err = diff / np.linalg.norm(ref, axis=1)
    # the same difference relative to the total acceleration with the central body's pull (G = M_c = 1)
    x = pos[idx]
    total = ref - x / np.linalg.norm(x, axis=1)[:, None] ** 3
    err_t = diff / np.linalg.norm(total, axis=1)
    return {"median": float(np.median(err)), "p99": float(np.percentile(err, 99)),
            "median_of_total": float(np.median(err_t)), "p99_of_total": float(np.percentile(err_t, 99)),
            "sample": int(len(idx)),
            "note": "mutual accelerations (ncorp_accel) against FP64 direct summation on a seeded sample: "
                    "|a - a_direct| / |a_direct|, and the same difference over the total acceleration with the "
                    "central body"}


def measure_accuracy(ncorp, d, n, p, theta, precision, local, stream):
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_MIXED if precision == "mixed" else ncorp.NCORP_FP64
    cfg.leaf_size = leaf_size_for(p)
    cfg.n_cs, cfg.n_cc_pre, cfg.n_cc_post = thresholds_for(p)
    ctx = ncorp.ncorp_init(cfg, n, local, stream.cuda_stream)
    try:
        acc, mut = np.zeros((n, 3)), np.zeros((n, 3))
        ncorp.ncorp_accel(ctx, d["pos"], d["mass"], n, p, theta, acc, mut)
    finally:
        ncorp.ncorp_free(ctx)
    return direct_sample_errors(d["pos"], d["mass"], mut)


def workload_config(a, n=None, seed=None, p=None, theta=None, precision=None):
    n = a.n if n is None else n
    seed = a.seed if seed is None else seed
    p = a.p if p is None else p
    theta = a.theta if theta is None else theta
    precision = a.precision if precision is None else precision
    res = f", collisions resolved with f={a.resolve_f}" if a.resolve_f else ""
    return {"workload": f"1 disk x {n} moonlets per GPU (seed {seed}+rank), falcON p={p} theta_min={theta}, "
                        f"SBAB1 step dt={a.dt} with tree collision search{res}, {precision} precision",
            "n_per_gpu": n, "p": p, "theta_min": theta, "dt": a.dt,
            "leaf_size": leaf_size_of(a, n, p),
            "gravity_thresholds": thresholds_for(p), "collision_thresholds": [12, 0, 16],
            "precision": precision, "l2": "flushed by a 256 MiB device write before every timed step",
            "parallelism": "replicas (one independent disk per GPU)",
            **({"resolve_f": a.resolve_f} if a.resolve_f else {}),
            **({"fused_walk": 1} if a.fused_walk else {})}


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def physical_gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ---------------------------------------------------------------------------- GPU arm
def host_cores():
    """Cores of this host as the OS reports them (nproc, and lscpu's model line when available)."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Architecture", "Model name", "CPU(s)", "Thread(s) per core", "Core(s) per socket",
                             "Socket(s)", "CPU max MHz"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


def time_disk(a, ncorp, torch, ctx_args, d, n, p, theta, precision, steps, warmup, prof_steps, local, stream, flush):
    """Times `steps` resident ncorp_step calls of one disk (L2 flushed before each, CUDA events on the
    library's stream), then `prof_steps` directly launched steps with the stage timers on.  Returns the
    per-step times, counters of the last step, summed launches and the stage times per step."""
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_MIXED if precision == "mixed" else ncorp.NCORP_FP64
    cfg.leaf_size = leaf_size_of(a, n, p)
    cfg.n_cs, cfg.n_cc_pre, cfg.n_cc_post = thresholds_for(p)
    cfg.c_cs, cfg.c_cc_pre, cfg.c_cc_post = 12, 0, 16
    cfg.resolve_f = a.resolve_f
    cfg.fused_walk = a.fused_walk
    ctx = ncorp.ncorp_init(cfg, n, local, stream.cuda_stream)
    pos = torch.tensor(d["pos"], device="cuda")
    vel = torch.tensor(d["vel"], device="cuda")
    m = torch.tensor(d["mass"], device="cuda")
    R = torch.tensor(d["radius"], device="cuda")

    def step():
        ncorp.ncorp_step(ctx, pos, vel, m, R, n, p, theta, a.dt)

    try:
        for _ in range(max(warmup, 3)):
            step()
        ctx_args["barrier"]()
        step_ms, launches, graph_steps, found = [], 0, 0, 0
        last = {}
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            st = ncorp.ncorp_stats(ctx)
            launches += st["launches"]
            graph_steps += st["graph"]
            found += st["col_found"]
            last = st
        ctx_args["barrier"]()
        # stage times: more steps after the timed region, launched directly (profiled steps are never
        # replayed from a graph) with CUDA events around every stage on the stream it runs on
        ncorp.ncorp_profile(ctx, True)
        stage, prof = {}, {"m2l": 0, "p2p_interactions": 0, "col_tests": 0}
        for _ in range(prof_steps):
            flush.zero_()
            torch.cuda.synchronize()
            step()
            st = ncorp.ncorp_stats(ctx)
            for k in prof:
                prof[k] += st[k]
            for k, v in ncorp.ncorp_stage_times(ctx).items():
                stage[k] = stage.get(k, 0.0) + v
        ncorp.ncorp_profile(ctx, False)
    finally:
        ncorp.ncorp_free(ctx)
    return {"step_ms": step_ms, "launches": launches, "graph_steps": graph_steps, "found": found, "last": last,
            "stage": {k: v / prof_steps for k, v in stage.items()}, "prof": {k: v / prof_steps for k, v in prof.items()},
            "prof_steps": prof_steps}


def near_roofline(t, peak_tflops, precision, traffic):
    """Roofline of the dominant kernel, the near-field direct sums (k_eval): NEAR_FLOP_PER_PAIR per unordered
    moonlet pair of the step (the method's count, whatever the kernel evaluates) over the kernel's event-timed
    duration, against the measured FMA peak of its precision."""
    near_ms = t["stage"].get("near", 0.0)
    pairs = t["prof"]["p2p_interactions"]
    flops = NEAR_FLOP_PER_PAIR * pairs
    achieved = flops / (near_ms * 1e-3) / 1e12 if near_ms > 0 else 0.0
    return {"bound": "alu", "kernel": "k_eval (near-field direct sums per leaf)",
            "achieved": round(achieved, 3), "peak": round(peak_tflops, 2), "unit": "TFLOP/s",
            "frac": round(achieved / peak_tflops, 4) if peak_tflops else None, "traffic": traffic,
            "flops_per_launch": flops, "unordered_pairs_per_launch": pairs, "avg_launch_ms": round(near_ms, 4),
            "peak_note": f"measured {precision} FMA throughput of this GPU (ncorp_fma_peak, in-bounds FMA chains, "
                         f"best of 5 launches at the start of this run), 'of measured'"}


def summarize(a, t, n, steps, world, dist, hbm, peak_tflops, p):
    total = sum(t["step_ms"])
    t_max = slowest_rank(dist, total, world)
    last = {k: t["last"][k] for k in ("cells", "leaves", "depth", "m2l", "p2p_pairs", "p2p_self", "p2p_interactions",
                                      "walk_iters", "col_pairs", "col_self", "col_tests", "col_iters",
                                      "m2l_directed", "p2p_directed", "sort_path")}
    return {"value": round(replica_throughput(n, steps, world, t_max * 1e-3), 1), "unit": UNIT,
            "ms_per_step": round(t_max / steps, 4),
            "p50_step_ms": round(float(np.percentile(t["step_ms"], 50)), 4),
            "p99_step_ms": round(float(np.percentile(t["step_ms"], 99)), 4),
            "steps": steps, "graph_steps": t["graph_steps"], "gpu_launches": t["launches"],
            "colliding_pairs_per_step": t["found"] / steps, "tree_stats_last_step": last,
            "stage_ms_per_step": {k: round(v, 4) for k, v in t["stage"].items()},
            "stage_note": f"CUDA events around each stage, {t['prof_steps']} directly launched steps after the "
                          f"timed region",
            "stage_roofline": stage_rooflines(t["stage"], n, p, t["prof"]["m2l"], t["prof"]["p2p_interactions"],
                                              t["prof"]["col_tests"], hbm, peak_tflops)}


def run_gpu(a):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2310_20374_gb300 import diskgen, ncorp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    hbm = measured_hbm_gbs()
    sampler = ClockSampler(physical_gpu_index(local))
    peaks = {"fp32_tflops": ncorp.ncorp_fma_peak(local, ncorp.NCORP_MIXED, stream.cuda_stream) / 1e12,
             "fp64_tflops": ncorp.ncorp_fma_peak(local, ncorp.NCORP_FP64, stream.cuda_stream) / 1e12,
             "hbm_gbs": hbm, "how": "FMA: ncorp_fma_peak (in-bounds FMA chains on every SM, best of 5 ~4 ms "
                                    "launches, 2 FLOP per FMA); HBM: MEASURED_PEAKS.json copy bandwidth"}
    peak = peaks["fp32_tflops"] if a.precision == "mixed" else peaks["fp64_tflops"]
    global FP32_PEAK_TFLOPS
    FP32_PEAK_TFLOPS = peaks["fp32_tflops"]
    ctx_args = {"barrier": barrier}

    # ---- the headline: workload 2 (N = 1e5, p = 6, theta_min = 0.5) in the requested precision
    cfgd = workload_config(a)
    d = diskgen.make_disk(a.n, a.seed + rank)
    t = time_disk(a, ncorp, torch, ctx_args, d, a.n, a.p, a.theta, a.precision, a.steps, a.warmup,
                  min(a.steps, 10), local, stream, flush)
    head = summarize(a, t, a.n, a.steps, world, dist, hbm, peak, a.p)
    roofline = near_roofline(t, peak, a.precision, eval_traffic(a.n, a.p, a.theta, a.precision, leaf_size_of(a, a.n, a.p)))

    extra = {}
    if not a.headline_only:
        # ---- the same disk in the other precision (FP64 is the paper's arithmetic; workload 2 names both)
        other = "fp64" if a.precision == "mixed" else "mixed"
        opeak = peaks["fp64_tflops"] if other == "fp64" else peaks["fp32_tflops"]
        osteps = max(5, a.steps // 10)
        t2 = time_disk(a, ncorp, torch, ctx_args, d, a.n, a.p, a.theta, other, osteps, 3, min(osteps, 5),
                       local, stream, flush)
        extra[other] = {"config": workload_config(a, precision=other), **summarize(a, t2, a.n, osteps, world, dist,
                                                                                     hbm, opeak, a.p),
                        "roofline": near_roofline(t2, opeak, other, None)}
        # ---- workload 3: N = 1e6 (seed 3), p = 4, theta_min = 0.6, mixed, 100 steps
        n3 = 1_000_000
        d3 = diskgen.make_disk(n3, 3 + rank)
        t3 = time_disk(a, ncorp, torch, ctx_args, d3, n3, 4, 0.6, "mixed", a.steps3, 3, 5, local, stream, flush)
        extra["config3"] = {"config": workload_config(a, n=n3, seed=3, p=4, theta=0.6, precision="mixed"),
                            **summarize(a, t3, n3, a.steps3, world, dist, hbm, peaks["fp32_tflops"], 4),
                            "roofline": near_roofline(t3, peaks["fp32_tflops"], "mixed",
                                                      eval_traffic(n3, 4, 0.6, "mixed", leaf_size_of(a, n3, 4)))}
        # ---- workload 4: 64 disks of mixed size in one batch, 50 steps replayed from one graph
        extra["config4"] = time_ensemble(a, ncorp, torch, dist, world, rank, stream, a.steps4, 3)
    clocks = sampler.stop()
    # ---- accuracy of the headline disk's mutual accelerations against direct summation (rank 0)
    accuracy = {}
    if rank == 0:
        accuracy[a.precision] = measure_accuracy(ncorp, d, a.n, a.p, a.theta, a.precision, local, stream)
        if not a.headline_only:
            other = "fp64" if a.precision == "mixed" else "mixed"
            accuracy[other] = measure_accuracy(ncorp, d, a.n, a.p, a.theta, other, local, stream)

    # ---- end to end through the C ABI with pinned host buffers: every step
    # copies the state in (positions, velocities, masses, radii), runs the step
    # from it and copies the new state and the colliding pairs out.
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_MIXED if a.precision == "mixed" else ncorp.NCORP_FP64
    cfg.leaf_size = cfgd["leaf_size"]
    cfg.n_cs, cfg.n_cc_pre, cfg.n_cc_post = cfgd["gravity_thresholds"]
    cfg.resolve_f = a.resolve_f
    ctx = ncorp.ncorp_init(cfg, a.n, local, stream.cuda_stream)
    hp = torch.tensor(d["pos"]).pin_memory()
    hv = torch.tensor(d["vel"]).pin_memory()
    hm = torch.tensor(d["mass"]).pin_memory()
    hR = torch.tensor(d["radius"]).pin_memory()
    hpairs = torch.empty((1 << 16, 2), dtype=torch.int64).pin_memory()
    e2e_steps = max(3, min(a.steps, 10))
    ncorp.ncorp_step(ctx, hp, hv, hm, hR, a.n, a.p, a.theta, a.dt)
    barrier()
    t0 = time.perf_counter()
    npairs = 0
    for _ in range(e2e_steps):
        ncorp.ncorp_reset(ctx)
        ncorp.ncorp_step(ctx, hp, hv, hm, hR, a.n, a.p, a.theta, a.dt)
        npairs += ncorp.ncorp_collisions(ctx, hpairs, hpairs.shape[0])
    barrier()
    e2e_s = slowest_rank(dist, time.perf_counter() - t0, world)
    e2e = {"value": round(replica_throughput(a.n, e2e_steps, world, e2e_s), 1), "unit": UNIT,
           "h2d_bytes_per_step": a.n * (24 + 24 + 8 + 8),
           "d2h_bytes_per_step": a.n * (24 + 24) + 16 * (npairs // e2e_steps),
           "note": "state uploaded from pinned host memory every step (so the step also recomputes the "
                   "acceleration of the uploaded state), new state and pairs read back"}
    ncorp.ncorp_free(ctx)

    out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": max(a.warmup, 3), "ms_per_step": head["ms_per_step"],
           "p50_step_ms": head["p50_step_ms"], "p99_step_ms": head["p99_step_ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64 (mixed)" if a.precision == "mixed" else "f64",
           "data": "synthetic (seeded moonlet disk shaped like the paper's)", "config": cfgd,
           "gpu_launches": head["gpu_launches"], "graph_steps": head["graph_steps"],
           "colliding_pairs_per_step": head["colliding_pairs_per_step"],
           "tree_stats_last_step": head["tree_stats_last_step"],
           "stage_ms_per_step": head["stage_ms_per_step"], "stage_note": head["stage_note"],
           "clocks": clocks, "e2e": e2e, "roofline": roofline, "peaks": peaks,
           "stage_roofline": head["stage_roofline"], "accuracy": accuracy,
           "stage_roofline_note": "per stage of one step against the measured HBM copy bandwidth or the measured "
                                  "FMA peak of the stage's precision; at N = 1e5 the working set (~20 MB) stays "
                                  "in L2, and walk/descend are latency-bound chains",
           **extra}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(a, cfgd, d)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------- oracle
def oracle_params(cfgd, a):
    import oracle
    return oracle.params(p=a.p, theta=a.theta, leaf_size=cfgd["leaf_size"],
                         gravity_thresholds=tuple(cfgd["gravity_thresholds"]),
                         collision_thresholds=tuple(cfgd["collision_thresholds"]), resolve_f=a.resolve_f)


def time_oracle_steps(a, cfgd, d, nsteps):
    """Wall time of nsteps oracle SBAB1 steps (acceleration of the start state computed untimed)."""
    import oracle
    P = oracle_params(cfgd, a)
    acc0, _ = oracle.falcon_accel(P, d["pos"], d["mass"])
    acc0 = acc0 + oracle.external_accel(P, d["pos"])
    t0 = time.perf_counter()
    oracle.kdk(P, d["pos"], d["vel"], d["mass"], d["radius"], a.dt, nsteps, acc0=acc0)
    return time.perf_counter() - t0


def _oracle_step_worker(args):
    """One oracle SBAB1 step of a disk from the generator (runs in a spawned process)."""
    n, seed, p, theta, dt, leaf, grav, col = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2310_20374_gb300 import diskgen
    d = diskgen.make_disk(n, seed)
    P = oracle.params(p=p, theta=theta, leaf_size=leaf, gravity_thresholds=tuple(grav), collision_thresholds=tuple(col))
    acc0, _ = oracle.falcon_accel(P, d["pos"], d["mass"])
    acc0 = acc0 + oracle.external_accel(P, d["pos"])
    t0 = time.perf_counter()
    oracle.kdk(P, d["pos"], d["vel"], d["mass"], d["radius"], dt, 1, acc0=acc0)
    return time.perf_counter() - t0


def cpu_baseline(a, cfgd, d):
    """The oracle as it stands on this host: one SBAB1 step of the same disk on one core, and one step of an
    independent disk per core at once (the all-core figure: disks one per core, one oracle process each)."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    secs = time_oracle_steps(a, cfgd, d, 1)
    cores = host_cores()
    ncores = int(cores.get("nproc") or 1)
    job = [(a.n, a.seed + 1000 + k, a.p, a.theta, a.dt, cfgd["leaf_size"], cfgd["gravity_thresholds"],
            cfgd["collision_thresholds"]) for k in range(ncores)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(ncores) as pool:
        per = pool.map(_oracle_step_worker, job)
    wall = time.perf_counter() - t0
    all_core = a.n * ncores / max(per)
    return {"value": round(a.n / secs, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 SBAB1 step of the same {a.n}-moonlet disk (falcON p={a.p} + tree collision search), "
                      f"plain C FP64 oracle, single thread; acceleration of the start state computed outside "
                      f"the timing", "seconds": round(secs, 3),
            "all_cores": {"value": round(all_core, 1), "unit": UNIT, "cores": ncores,
                          "sample": f"{ncores} independent {a.n}-moonlet disks, one oracle process per core, one "
                                    f"step each at once; value = moonlet-steps / the slowest process's step time",
                          "slowest_s": round(max(per), 3), "fastest_s": round(min(per), 3),
                          "wall_s_with_setup": round(wall, 2)},
            "host": cores}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2310_20374_gb300 import diskgen
    import oracle
    oracle.build()
    # bounded sample: a disk small enough that warmup + steps end within ~2 minutes
    per_particle_s = 6e-5
    n = int(min(a.n, max(2000, 120.0 / (per_particle_s * (a.steps + max(a.warmup, 3) + 1)))))
    cfgd = workload_config(a, n=n, precision="fp64 (the plain-C oracle)")
    d = diskgen.make_disk(n, a.seed)
    import copy
    b = copy.copy(a)
    b.n = n
    time_oracle_steps(b, cfgd, d, max(a.warmup, 3))
    secs = time_oracle_steps(b, cfgd, d, a.steps)
    value = n * a.steps / secs
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
           "steps": a.steps, "warmup": max(a.warmup, 3), "ms_per_step": round(1e3 * secs / a.steps, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded moonlet disk shaped like the paper's)", "config": cfgd,
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{a.steps} SBAB1 steps of a {n}-moonlet disk from the same generator "
                                      f"(the workload's {a.n}-moonlet disk scaled down to keep the run within "
                                      f"minutes)", "host": host_cores()},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------- batches
def ensemble_sizes(k, lo, hi, seed):
    """k disk sizes log-uniform in [lo, hi] (seeded)."""
    u = np.random.default_rng(seed).random(k)
    return np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo))).astype(np.int64)


def batch_common(a):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2310_20374_gb300 import ncorp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build()
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_MIXED if a.precision == "mixed" else ncorp.NCORP_FP64
    return torch, dist, ncorp, cfg, rank, world, local


def time_ensemble(a, ncorp, torch, dist, world, rank, stream, steps, warmup):
    """Workload 4: 64 disks per GPU, N log-uniform in [1e3, 2e5] (sizes seeded 100 + rank, disk k seeded
    100 + 64 rank + k), p = 6, theta_min = 0.5, mixed, dt = 1e-3, advanced together by ncorp_batch_run: every
    disk in one forest, one launch per stage, the run of `steps` steps replayed from one CUDA graph."""
    from paper_2310_20374_gb300 import diskgen
    cfg = ncorp.ncorp_config_default()
    cfg.precision = ncorp.NCORP_MIXED
    p, theta, dt = 6, 0.5, 1e-3
    sizes = ensemble_sizes(64, 1e3, 2e5, 100 + rank)
    b = ncorp.ncorp_batch_create(cfg, 0, stream.cuda_stream)
    try:
        for k, n in enumerate(sizes):
            d = diskgen.make_disk(int(n), 100 + 64 * rank + k)
            args = [torch.tensor(d[f], device="cuda") for f in ("pos", "vel", "mass", "radius")]
            ncorp.ncorp_batch_add_disk(b, *args, int(n), p, theta, dt)
        total = int(sizes.sum())
        ncorp.ncorp_batch_run(b, warmup)
        ncorp.ncorp_batch_run(b, steps)   # captures the graph of this run length
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ncorp.ncorp_batch_run(b, steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        info = ncorp.ncorp_batch_info(b)
        t_max = slowest_rank(dist, ms, world)
        # end to end: another run, then every disk's state read back to pinned host memory
        hp = [torch.empty((int(n), 3), dtype=torch.float64).pin_memory() for n in sizes]
        hv = [torch.empty((int(n), 3), dtype=torch.float64).pin_memory() for n in sizes]
        t0 = time.perf_counter()
        ncorp.ncorp_batch_run(b, steps)
        for k in range(len(sizes)):
            ncorp.ncorp_batch_get_state(b, k, hp[k], hv[k])
        e2e_s = slowest_rank(dist, time.perf_counter() - t0, world)
    finally:
        ncorp.ncorp_batch_free(b)
    value = replica_throughput(total, steps, world, t_max * 1e-3)
    return {"value": round(value, 1), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": round(t_max / steps, 4),
            "config": {"workload": f"64 disks per GPU, N log-uniform in [1e3, 2e5] (total {total} moonlets), "
                                   f"falcON p={p} theta_min={theta}, {steps} SBAB1 steps dt={dt} with collision "
                                   f"search, mixed precision, one ncorp_batch_run (one forest: one launch per "
                                   f"stage over all disks, the run replayed from one CUDA graph)",
                       "moonlets_per_gpu": total, "disks_per_gpu": 64, "leaf_size": info["leaf_size"],
                       "leaf_size_chosen_by": "the batch's autotuner (timed candidates around the default "
                                              f"{leaf_size_for(p)} for p = {p})" if info["tuned"] else "default",
                       "gravity_thresholds": list(thresholds_for(p)),
                       "l2": "inputs larger than L2 (about 1 kB of state and tree per moonlet)",
                       "parallelism": "replicas (one batch of 64 disks per GPU)"},
            "gpu_launches": info["launches"], "forests": info["forests"],
            "e2e": {"value": round(replica_throughput(total, steps, world, e2e_s), 1), "unit": UNIT,
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(48 * total / steps),
                    "note": "host wall time of ncorp_batch_run plus reading every disk's state back to pinned "
                            "host memory once per run (per-step bytes averaged)"}}


def run_ensemble(a):
    """Workload 4 alone (see time_ensemble); value = moonlet-steps of all disks / time."""
    torch, dist, ncorp, cfg, rank, world, local = batch_common(a)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(physical_gpu_index(local))
    r = time_ensemble(a, ncorp, torch, dist, world, rank, stream, a.steps, max(a.warmup, 3))
    clocks = sampler.stop()
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": max(a.warmup, 3), "ms_per_step": r["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
           "data": "synthetic (seeded moonlet disks shaped like the paper's)", "config": r["config"],
           "gpu_launches": r["gpu_launches"], "clocks": clocks, "e2e": r["e2e"]}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_serving(a):
    """Serving (continuous batching): disks arrive as a Poisson stream (rate r per s over the window), N
    log-uniform in [1e3, 1e6], p uniform in {3, 4, 6}, theta_min = 0.5, each integrated for 100 steps; the loop
    of paper_2310_20374_gb300.serving admits arrived requests in order while the batch's memory budget allows
    and advances every resident disk by up to --tick-steps steps per ncorp_batch_run.  The run lasts the
    arrival window: admission stops at its end (requests still queued then are reported as not admitted), and
    the disks already admitted are integrated to the end of their steps."""
    torch, dist, ncorp, cfg, rank, world, local = batch_common(a)
    from paper_2310_20374_gb300 import diskgen, serving
    reqs = serving.poisson_requests(a.serve_rate, a.serve_seconds, 1e3, 1e6, (3, 4, 6), 100, seed=500 + rank)
    # inputs are generated before the clock starts (they stand in for requests already in host memory); a
    # long window reuses the disks of its first --serve-pool requests (request k starts from disk k mod pool,
    # with that disk's N), so the host holds a bounded number of initial states
    pool = len(reqs) if a.serve_pool <= 0 else min(len(reqs), a.serve_pool)
    disks = [diskgen.make_disk(r.n, 700 + 1000 * rank + k) for k, r in enumerate(reqs[:pool])]
    for k, r in enumerate(reqs):
        r.disk = disks[k % pool]
        r.n = len(r.disk["pos"])
    stream = torch.cuda.current_stream()
    free_b, _ = torch.cuda.mem_get_info()
    budget = int(a.serve_budget * free_b)
    b = ncorp.ncorp_batch_create(cfg, budget, stream.cuda_stream)   # admission: a fraction of free HBM
    log = open(a.serve_log, "a") if a.serve_log else None

    def progress(state):
        log.write(json.dumps(state) + "\n")
        log.flush()

    sampler = ClockSampler(physical_gpu_index(local))
    try:
        # each finished disk's state goes back to host memory (what a client receives)
        backend = serving.BatchBackend(ncorp, b, a.theta, a.dt)
        st = serving.serve(backend, reqs, tick_steps=a.tick_steps,
                           on_done=lambda r: (np.empty((r.n, 3)), np.empty((r.n, 3))),
                           progress=progress if log else None, max_wall=a.serve_seconds)
    finally:
        clocks = sampler.stop()
        ncorp.ncorp_batch_free(b)
        if log:
            log.close()
    offered = sum(r.n for r in reqs) * 100 / a.serve_seconds
    served_n = sum(r.n for r in reqs if r.done is not None)
    value = slowest_rank(dist, st["throughput"], world) if world > 1 else st["throughput"]
    out = {"metric": METRIC, "value": round(value * (world if world > 1 else 1), 1), "unit": UNIT, "n_gpus": world,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64 (mixed)" if a.precision == "mixed" else "f64",
           "data": "synthetic (seeded moonlet disks shaped like the paper's)",
           "config": {"workload": f"serving: Poisson arrivals at {a.serve_rate}/s for {a.serve_seconds} s "
                                  f"({len(reqs)} disks, {pool} distinct initial states), N log-uniform in "
                                  f"[1e3, 1e6], p in {{3,4,6}}, "
                                  f"theta_min={a.theta}, 100 SBAB1 steps each, dt={a.dt}, {a.precision} precision, "
                                  f"up to {a.tick_steps} steps per tick",
                      "requests": st["requests"], "served": st["served"],
                      "not_admitted": st["requests"] - st["served"], "moonlet_steps": st["moonlet_steps"],
                      "parallelism": "replicas (one serving loop per GPU)"},
           "latency": {
               "step_ms_p50": st["step_ms_p50"], "step_ms_p99": st["step_ms_p99"],
               "tick_ms_p50": st["tick_ms_p50"], "tick_ms_p99": st["tick_ms_p99"],
               "request_s_p50": st["request_s_p50"], "request_s_p99": st["request_s_p99"],
               "admission_wait_s_p50": st["admission_wait_s_p50"], "admission_wait_s_p99": st["admission_wait_s_p99"],
               "note": "host wall times: step = one tick (one ncorp_batch_run of k steps over every resident disk) "
                       "/ k, one sample per disk and step; request = arrival to last step, admission wait included; "
                       "request and admission figures cover the requests admitted within the window"},
           "peak_batch_bytes": getattr(backend, "peak_bytes", None),
           "peak_resident_moonlets": getattr(backend, "peak_moonlets", None),
           "hbm_budget_bytes": budget,
           "concurrent_disks_mean": round(st["concurrent_disks_mean"], 2),
           "concurrent_disks_max": st["concurrent_disks_max"],
           "busy_throughput": round(st["busy_throughput"], 1),
           "wall_s": round(st["wall_s"], 2), "offered_moonlet_steps_per_s": round(offered, 1),
           "clocks": clocks,
           "e2e": {"value": round(value, 1), "unit": UNIT,
                   # every served disk's state in (x, v, m, R: 64 B per moonlet) and out (x, v: 48 B per moonlet),
                   # over the batch steps of the run
                   "h2d_bytes_per_step": round(64 * served_n / max(st["batch_steps"], 1)),
                   "d2h_bytes_per_step": round(48 * served_n / max(st["batch_steps"], 1)),
                   "note": "the serving throughput is end to end: host arrays in, each disk's state back to host "
                           "memory when it finishes; bytes per step = all requests' bytes / batch steps "
                           "(ncorp_batch_run steps over every resident disk)"}}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_standard(a):
    """Force evaluation of one disk by the standard tree code (ncorp_accel_standard) and, on the same disk
    and context settings, by falcON (ncorp_accel): moonlet accelerations per second of each, inputs resident
    in HBM, L2 flushed before every evaluation."""
    torch, dist, ncorp, cfg, rank, world, local = batch_common(a)
    from paper_2310_20374_gb300 import diskgen
    stream = torch.cuda.current_stream()
    d = diskgen.make_disk(a.n, a.seed + rank)
    ctx = ncorp.ncorp_init(cfg, a.n, local, stream.cuda_stream)
    pos = torch.tensor(d["pos"], device="cuda")
    m = torch.tensor(d["mass"], device="cuda")
    acc = torch.empty_like(pos)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn):
        for _ in range(max(a.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(a.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return slowest_rank(dist, total, world), ncorp.ncorp_stats(ctx)

    sampler = ClockSampler(physical_gpu_index(local))
    ms_std, st_std = timed(lambda: ncorp.ncorp_accel_standard(ctx, pos, m, a.n, a.p, a.theta, acc))
    ms_fal, st_fal = timed(lambda: ncorp.ncorp_accel(ctx, pos, m, a.n, a.p, a.theta, acc))
    clocks = sampler.stop()
    ncorp.ncorp_free(ctx)
    unit = "moonlet accelerations/s"
    value = replica_throughput(a.n, a.steps, world, ms_std * 1e-3)
    out = {"metric": "moonlet accelerations/s, standard tree code (Algorithm StandardTree) vs falcON",
           "value": round(value, 1), "unit": unit, "n_gpus": world, "steps": a.steps, "warmup": max(a.warmup, 3),
           "ms_per_step": round(ms_std / a.steps, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64 (mixed)" if a.precision == "mixed" else "f64",
           "data": "synthetic (seeded moonlet disk shaped like the paper's)",
           "config": {"workload": f"1 disk x {a.n} moonlets per GPU (seed {a.seed}+rank), p={a.p} theta_min={a.theta}, "
                                  f"N_cb,pre={cfg.n_cb_pre} N_cb,post={cfg.n_cb_post}, one force evaluation per step "
                                  f"(tree build, climb, multipoles, walk, evaluation), {a.precision} precision",
                      "l2": "flushed by a 256 MiB device write before every timed evaluation",
                      "parallelism": "replicas (one independent disk per GPU)"},
           "standard_stats": {k: st_std[k] for k in ("cells", "leaves", "m2l", "p2p_pairs", "p2p_interactions")},
           "falcon": {"value": round(replica_throughput(a.n, a.steps, world, ms_fal * 1e-3), 1), "unit": unit,
                      "ms_per_eval": round(ms_fal / a.steps, 4),
                      "stats": {k: st_fal[k] for k in ("m2l", "p2p_pairs", "p2p_interactions")}},
           "falcon_speedup": round(ms_std / ms_fal, 2),
           "gpu_launches": st_std["launches"] * a.steps, "clocks": clocks}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.thresholds:
        THRESHOLDS_OVERRIDE[a.p] = [int(v) for v in a.thresholds.split(",")]
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "ensemble":
        run_ensemble(a)
    elif a.workload == "serving":
        run_serving(a)
    elif a.workload == "standard":
        run_standard(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
