#!/usr/bin/env python
"""Benchmark: MI pose evaluations per second on the LiDAR-shaped 120k-point pair.

One step is one pass of the whole hot path on one scan pair: build A's reference state
(voxelize A, symbols, bbox, prefix counts), then a coarse-to-fine lattice search of B
(6 levels x 4,096 poses; each level: pose rounding, transform + voxelize + accumulate,
symbols + joint histogram, overlap + MI, argmax).  `value` counts MI pose evaluations
per second with both scans already in device memory; `e2e` is the same through the C
ABI from pinned host buffers (copies inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it runs under torchrun, one independent pair per rank (weak scaling, no
collective on the data path).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scangen  # noqa: E402

METRIC = "MI pose evals/s on 120k-pt pair; served alignment p50/p99 ms vs plain loop"
UNIT = "pose-evals/s"
LEVELS = 6
COUNTS = (8, 8, 2, 2, 2, 8)
RANGE = np.array([2.0, 2.0, 0.25, math.radians(1.0), math.radians(1.0), math.radians(5.0)])
# Algorithmic ALU work per (point, pose) in 32-bit lane operations: transform, voxel key,
# dz and bounds, with the 9-operation rotation (OPS_MAP) and with the rotation amortised
# across the translations that share it (OPS_MAP_AMORTISED).  Shared-memory atomics: three
# per occupied voxel of a pose (n, S1, S2).
OPS_MAP = 24
OPS_MAP_AMORTISED = 15
ATOMICS_PER_VOXEL = 3


def workload_config(pair, levels):
    X, Y, Z = pair.grid.dims
    return {
        "workload": "lidar-120k: 64-beam ray-cast urban pair, grid 160x160x16 @ 0.5 m, z-variance 16 symbols, "
                    f"set_reference + {levels}-level lattice search of 4,096 poses per level",
        "points_A": int(pair.xyzA.shape[0]),
        "points_B": int(pair.xyzB.shape[0]),
        "grid": f"{X}x{Y}x{Z}@{pair.grid.res_m}m",
        "poses_per_level": int(np.prod(COUNTS)),
        "levels": levels,
        "lattice": "x".join(str(c) for c in COUNTS),
        "l2": "flushed between steps (256 MiB write)",
        "parallelism": "replicas (one independent pair per GPU)",
    }


# --------------------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self, t_begin=None, t_end=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if t_begin is not None and not (t_begin - 0.05 <= ts <= t_end + 0.05):
                    continue
            except ValueError:
                pass
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return None


def code_digest(path):
    """sha256 of a source file's code: `//` comments, trailing blanks and empty lines
    removed (a comment-only edit leaves the kernel, and its profile, unchanged)."""
    lines = []
    with open(path, encoding="utf-8") as f:
        for line in f:
            i = line.find("//")
            line = (line[:i] if i >= 0 else line).rstrip()
            if line:
                lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def committed_traffic():
    """Per-launch DRAM bytes of the eval kernel from the committed ncu summary, if it was
    taken on the current kernel code (else None)."""
    path = os.path.join(ROOT, "profiles", "eval_pair_kernel_lidar120k.md")
    src = os.path.join(ROOT, "paper_1709_06948_gb300", "csrc", "eval.cu")
    try:
        text = open(path).read()
        digest = code_digest(src)
    except Exception:
        return None
    m_sha = re.search(r"eval\.cu code sha256[^:]*:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != digest:
        return None
    return float(m_b.group(1))


def host_cpu():
    """Host CPU model and core count (for the CPU baseline)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "nproc": os.cpu_count()}


def measure_peaks(align, gpu_id, reps=5):
    """Measured throughput peaks of this GPU (align_microbench), with the SM clock sampled
    while they run."""
    import torch
    buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    t0 = time.time()
    r = {}
    for k, name in align.MICROBENCH_KINDS.items():
        for _ in range(3):  # repeat the set so the sampler sees every kind under load
            rate, ms, ops = align.align_microbench(k, buf, reps=reps)
            if name not in r or rate > r[name]["per_s"]:
                r[name] = {"per_s": rate, "ms": ms, "ops": ops}
    t1 = time.time()
    clocks = sampler.stop(t0, t1)
    del buf
    alu = max(r["fp32 ffma lane-ops"]["per_s"], r["int32 add/xor lane-ops"]["per_s"])
    return {"alu_lane_ops_per_s": alu, "keymix_lane_ops_per_s": r["voxel-map mix lane-ops"]["per_s"],
            "smem_red_random_per_s": r["shared red.add (random words)"]["per_s"],
            "smem_atom_random_per_s": r["shared atom.add (random words)"]["per_s"],
            "l2_atomic_per_s": r["L2 atomic add (random words)"]["per_s"],
            "all": {k: v["per_s"] for k, v in r.items()}, "clocks": clocks,
            "how": f"align_microbench, fastest of {reps} runs x 3 rounds, 2 x 1,024-thread CTAs per SM, "
                   "CUDA events"}


# --------------------------------------------------------------------------------------
# CPU oracle (reference arm and the cpu_baseline leg)
# --------------------------------------------------------------------------------------
def oracle_rate(pair, n_poses, nthreads):
    import oracle
    G = oracle.Grid(pair.grid.origin, pair.grid.res_m, pair.grid.dims, pair.grid.feature, pair.grid.count_levels,
                    pair.grid.var_levels)
    symA, boxA = G.reference(pair.xyzA)
    etas = oracle.lattice(np.zeros(6), RANGE, COUNTS)[:n_poses]
    poses = G.round_pose(etas)
    t0 = time.perf_counter()
    G.eval_mi(symA, boxA, pair.xyzB, poses, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return n_poses / dt, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    pair = scangen.lidar_pair()
    cores = oracle.host_cores()
    sample = 4096
    for _ in range(args.warmup):
        oracle_rate(pair, sample, cores)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(pair, sample, cores)
        times.append(dt)
    total = sum(times)
    value = sample * args.steps / total
    desc = (f"all {sample} level-0 lattice poses of the 120k-point pair per step (one of the 6 levels of a "
            f"search step), oracle (dense per-pose arrays, FP64 MI) on {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(pair, LEVELS),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------------------
# batched pairs (many pairs in one captured launch sequence) and served requests
# --------------------------------------------------------------------------------------
BATCH_PAIRS = 64
SERVE_REQUESTS = 400
SERVE_RATES_HZ = (80.0, 120.0, 150.0, 200.0)
SERVE_RANGE = np.array([3.0, 3.0, 0.5, math.radians(2.0), math.radians(2.0), math.radians(10.0)])
SERVE_RES = (0.25, 0.5, 0.75, 1.0)
SERVE_SLOTS = 3


def run_batched(align, steps):
    """64 pairs (20k-130k points, 0.25/0.5/1 m grids), each with its own 4,096-pose lattice,
    in one launch sequence (graph replay, tuned kernel shape); against one align_eval_mi
    launch per pair on the same inputs."""
    pairs = scangen.batched_pairs(BATCH_PAIRS)
    grids, items = [], []
    for p in pairs:
        g = align.align_create_grid(p.grid.origin, p.grid.res_m, p.grid.dims, p.grid.feature,
                                    p.grid.count_levels, p.grid.var_levels)
        align.align_set_reference(g, p.xyzA)
        grids.append(g)
        items.append((g, p.xyzB, scangen.lidar_poses()))
    b = align.align_batch_create()
    first = align.align_eval_batch(b, items, graph=True, tune=True)  # tunes, captures
    align.align_eval_batch(b, items, graph=True)
    dev_us, wall = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        res = align.align_eval_batch(b, items, graph=True)
        wall.append(time.perf_counter() - t0)
        dev_us.append(align.align_batch_stats(b)["last_us"])
    same = all(np.array_equal(a[0], r[0]) and a[1] == r[1] for a, r in zip(first, res))
    # plain loop: one launch per pair (same inputs, host poses)
    for g, B, etas in items[:2]:
        align.align_eval_mi(g, B, eta6=etas)
    loop = []
    loop_reps = max(1, min(steps, 3))
    for g in grids:
        align.align_profile(g, 1)
    for _ in range(loop_reps):
        t0 = time.perf_counter()
        single = [align.align_eval_mi(g, B, eta6=etas)[:2] for g, B, etas in items]
        loop.append(time.perf_counter() - t0)
    loop_dev_ms = 0.0  # eval + compose kernels, CUDA events per launch
    for g in grids:
        ev_ms, comp_ms, _ = align.align_profile(g, 2)
        align.align_profile(g, 0)
        loop_dev_ms += ev_ms + comp_ms
    loop_dev_ms /= loop_reps
    same = same and all(np.array_equal(a[0], r[0]) and a[1] == r[1] for a, r in zip(single, res))
    P = sum(len(e) for _, _, e in items)
    st = align.align_batch_stats(b)
    dev_s = statistics.median(dev_us) / 1e6
    out = {"workload": f"{BATCH_PAIRS} pairs, points log-uniform 20k-130k, grids 0.25/0.5/1 m cycled "
                       "(320x320x32, 160x160x16, 80x80x8), z-variance 16 symbols, 4,096 lattice poses each, "
                       "one launch sequence replayed as a CUDA graph",
           "points": [int(p.xyzB.shape[0]) for p in pairs][:8] + ["..."],
           "poses_per_launch": P,
           "pose_evals_per_s_device": P / dev_s,
           "ms_per_launch_device": dev_s * 1e3,
           "pose_evals_per_s_wall": P / statistics.median(wall),
           "ms_per_call_wall": statistics.median(wall) * 1e3,
           "plain_loop_pose_evals_per_s_wall": P / statistics.median(loop),
           "plain_loop_ms_wall": statistics.median(loop) * 1e3,
           "plain_loop_eval_compose_ms_device": loop_dev_ms,
           "speedup_vs_plain_loop_wall": statistics.median(loop) / statistics.median(wall),
           "tuned_shape": st["shape"], "table_slots": st["table_slots"], "graph_replays": st["graph_replays"],
           "graph_captures": st["graph_captures"], "tuner_trials": st["tuner_trials"],
           "results_identical_to_plain_loop": bool(same)}
    b.close()
    for g in grids:
        g.close()
    return out


def run_refine(align, pair, L, T_search):
    """Nelder-Mead refinement (Algorithm 1's optimiser) of the search result: 64 simplices
    from starts scattered around it, 40 iterations each, batched evaluations."""
    rng = np.random.default_rng(scangen.SEED_BASE + 6)
    S, iters = 64, 40
    starts = T_search[None, :] + rng.normal(0, 1, (S, 6)) * np.array([0.3, 0.3, 0.05, 0.004, 0.004, 0.01])
    step = np.array([0.3, 0.3, 0.1, 0.005, 0.005, 0.02])
    align.align_refine_nm(L, pair.xyzB, starts[:4], step=step, max_iter=2)  # warm-up
    t0 = time.perf_counter()
    T, mi, it = align.align_refine_nm(L, pair.xyzB, starts, step=step, max_iter=iters)
    dt = time.perf_counter() - t0
    k = int(np.argmax(mi))
    return {"workload": f"{S} simplices x {iters} iterations on the 120k-point pair, started around the "
                        "lattice-search result (step 0.3 m / 0.1 m / 0.005 rad / 0.02 rad)",
            "ms": dt * 1e3, "best_mi": float(mi[k]),
            "best_T": [float(x) for x in T[k]],
            "xy_error_m": float(np.hypot(T[k][0] - pair.T[0], T[k][1] - pair.T[1])),
            "note": "each iteration evaluates the reflections, then expansions/contractions, then shrinks of "
                    "all simplices in one batched evaluation each"}


def run_large(align, steps):
    """128-beam pair (~260k points), 400x400x40 grid at 0.2 m (6.4M voxels), joint count x
    z-variance feature (57 symbols), one 32,768-pose lattice per launch."""
    import torch
    pair = scangen.large_pair()
    spec = pair.grid
    L = align.align_create_grid(spec.origin, spec.res_m, spec.dims, spec.feature, spec.count_levels,
                                spec.var_levels)
    align.align_set_reference(L, pair.xyzA)
    etas = scangen.large_poses()
    P = len(etas)
    B = torch.from_numpy(pair.xyzB).cuda()
    # warm-up: the grid learns its key partitions and which way of sweeping fits (pose pairs,
    # one pose per CTA, one pose per 2-CTA cluster); stop once that stays the same
    prev, learned = None, []
    for _ in range(8):
        align.align_eval_mi(L, B, eta6=etas)
        st = align.align_eval_stats(L)
        cur = (st["sweep"], st["passes"])
        learned.append(cur)
        if cur == prev:
            break
        prev = cur
    torch.cuda.synchronize()
    align.align_profile(L, 1)
    wall = []
    for _ in range(steps):
        t0 = time.perf_counter()
        mi, am, _ = align.align_eval_mi(L, B, eta6=etas)
        wall.append(time.perf_counter() - t0)
    ev_ms, comp_ms, n = align.align_profile(L, 2)
    align.align_profile(L, 0)
    st = align.align_eval_stats(L)
    out = {"poses": P, "points": int(pair.xyzB.shape[0]),
           "workload": f"large: {pair.xyzB.shape[0]}-point 128-beam pair, grid 400x400x40 @ 0.2 m (6.4M voxels), "
                       f"joint count x z-variance 57 symbols, {P} lattice poses per launch (+-10 m, +-30 deg yaw)",
           "pose_evals_per_s_wall": P / statistics.median(wall),
           "ms_per_launch_wall": statistics.median(wall) * 1e3,
           "eval_kernel_ms": ev_ms / max(n, 1), "key_partitions": st["passes"],
           "sweep": align.SWEEP_KINDS.get(st["sweep"], st["sweep"]),
           "warmup_sweep_and_partitions": [[align.SWEEP_KINDS.get(k, k), p] for k, p in learned],
           "argmax_eta": [float(x) for x in etas[am]], "T_true": [float(x) for x in pair.T], "mi_max": float(mi[am])}
    L.close()
    return out


def _serve_requests(rng, scenes, refs, n):
    reqs = []
    for _ in range(n):
        r = int(rng.integers(len(refs)))
        n_pts = int(round(math.exp(rng.uniform(math.log(10000), math.log(130000)))))
        B = scangen.subsample(scenes[refs[r][0]].xyzB, n_pts, rng)
        err_r, err_a = 3.0 * math.sqrt(rng.uniform()), rng.uniform(-math.pi, math.pi)
        init = scenes[refs[r][0]].T + np.array([err_r * math.cos(err_a), err_r * math.sin(err_a), 0.0, 0.0, 0.0,
                                                math.radians(rng.uniform(-10.0, 10.0))])
        reqs.append((r, B, init))
    return reqs


def run_serving(align, slots=SERVE_SLOTS, rates=SERVE_RATES_HZ):
    """Poisson arrivals of alignment requests against 16 resident references, at several
    rates: the continuous-batching server and the plain loop (one request at a time, one
    align_search each, first come first served), both driven by the same arrival times in
    real time; latency = completion - arrival."""
    import threading
    rng = np.random.default_rng(scangen.SEED_BASE + 5)
    scenes = [scangen.lidar_pair(seed=scangen.SEED_BASE + 200 + k, az_step_deg=0.15) for k in range(4)]
    refs = [(k, res) for k in range(4) for res in SERVE_RES]  # 16 references
    srv = align.align_server_create(96 << 30, slots)
    ids, grids = [], []
    for k, res in refs:
        spec = scangen.lidar_grid(res)
        ids.append(align.align_server_add_reference(srv, scenes[k].xyzA, spec.origin, spec.res_m, spec.dims,
                                                    spec.feature, spec.count_levels, spec.var_levels))
        g = align.align_create_grid(spec.origin, spec.res_m, spec.dims, spec.feature, spec.count_levels,
                                    spec.var_levels)
        align.align_set_reference(g, scenes[k].xyzA)
        grids.append(g)
    reqs = _serve_requests(rng, scenes, refs, SERVE_REQUESTS)
    # warm-up (kernels, allocations) on both paths
    for r, B, init in reqs[:8]:
        align.align_wait(srv, align.align_submit(srv, ids[r], B, init, SERVE_RANGE, levels=LEVELS, counts=COUNTS))
        align.align_search(grids[r], B, init, SERVE_RANGE, levels=LEVELS, counts=COUNTS)
    out = {"workload": f"{SERVE_REQUESTS} requests per rate, Poisson arrivals, 10k-130k points, 16 resident "
                       "references (4 scenes x grids 0.25/0.5/0.75/1 m), init error <= 3 m / 10 deg yaw, ranges "
                       "+-3 m xy, +-0.5 m z, +-2 deg roll/pitch, +-10 deg yaw, 6 levels x 4,096 poses",
           "slots": slots, "rates": []}
    plain_T = None
    for k, rate in enumerate(rates):
        arrivals = scangen.poisson_arrivals(rate, SERVE_REQUESTS, seed=scangen.SEED_BASE + 4 + k)
        # server: a client thread submits at the arrival times
        tickets = [None] * len(reqs)
        wall0 = time.perf_counter()
        t0 = align.align_server_now(srv)

        def client():
            for i, (r, B, init) in enumerate(reqs):
                delay = arrivals[i] - (time.perf_counter() - wall0)
                if delay > 0:
                    time.sleep(delay)
                tickets[i] = align.align_submit(srv, ids[r], B, init, SERVE_RANGE, levels=LEVELS, counts=COUNTS)

        th = threading.Thread(target=client)
        st0 = align.align_server_stats(srv)
        th.start()
        th.join()
        res = [align.align_wait(srv, t) for t in tickets]
        st = align.align_server_stats(srv)
        lat = np.array([x["t_done"] - x["t_submit"] for x in res])
        span = max(x["t_done"] for x in res) - (t0 + arrivals[0])
        # plain loop: FIFO, one request at a time, driven by the same arrivals in real time
        wall0 = time.perf_counter()
        plat, got = [], []
        for i, (r, B, init) in enumerate(reqs):
            delay = arrivals[i] - (time.perf_counter() - wall0)
            if delay > 0:
                time.sleep(delay)
            T, mi, _ = align.align_search(grids[r], B, init, SERVE_RANGE, levels=LEVELS, counts=COUNTS)
            plat.append(time.perf_counter() - wall0 - arrivals[i])
            got.append((T, mi))
        pspan = time.perf_counter() - wall0 - arrivals[0]
        plat = np.array(plat)
        same = all(x["T"].tolist() == T.tolist() and x["mi"] == mi for x, (T, mi) in zip(res, got))
        plain_T = got
        out["rates"].append({
            "arrival_rate_hz": rate,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "requests_per_s": len(res) / span,
            "plain_loop_p50_ms": float(np.percentile(plat, 50) * 1e3),
            "plain_loop_p99_ms": float(np.percentile(plat, 99) * 1e3),
            "plain_loop_requests_per_s": len(reqs) / pspan,
            "steps": st["steps"] - st0["steps"], "max_active": st["max_active"],
            "results_identical_to_plain_loop": bool(same)})
    st = align.align_server_stats(srv)
    out["peak_bytes"] = st["bytes_peak"]
    err = [float(np.hypot(*(T[:2] - scenes[refs[q[0]][0]].T[:2]))) for (T, _), q in zip(plain_T, reqs)]
    out["median_xy_error_m"] = float(np.median(err))
    out["latency_basis"] = ("completion minus arrival, measured; both paths see the same Poisson arrival times in "
                            "real time (the plain loop waits for the next arrival when idle)")
    srv.close()
    for g in grids:
        g.close()
    return out


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_1709_06948_gb300 import align

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    pair = scangen.lidar_pair(seed=scangen.SEED_BASE + 2 + rank)
    spec = pair.grid
    stream = torch.cuda.current_stream()
    L = align.align_create_grid(spec.origin, spec.res_m, spec.dims, spec.feature, spec.count_levels,
                                spec.var_levels, stream=stream)
    A = torch.from_numpy(pair.xyzA).cuda()
    B = torch.from_numpy(pair.xyzB).cuda()
    init = np.zeros(6)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    P = int(np.prod(COUNTS)) if args.mode == "search" else args.poses
    etas_eval = scangen.lidar_poses()[:P] if args.mode == "eval" else None
    poses_dev = torch.from_numpy(align.align_round_poses(spec.origin, etas_eval)).cuda() if args.mode == "eval" else None
    mi_dev = torch.empty(max(P, 1), dtype=torch.float32, device="cuda")
    am_dev = torch.empty(1, dtype=torch.int64, device="cuda")

    def step():
        align.align_set_reference(L, A)
        if args.mode == "eval":
            align.align_eval_mi(L, B, poses12=poses_dev, out=(mi_dev, am_dev, None))
            return None, None, None
        return align.align_search(L, B, init, RANGE, levels=LEVELS)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    # in-grid point count of B at the lattice centre (for the accumulation op count)
    ident = align.align_round_poses(spec.origin, np.zeros((1, 6)))[0]
    acc, _ = align.align_accumulate(L, pair.xyzB, ident)
    occ = int(np.count_nonzero(acc[:, 0]))
    del acc

    dev_props = torch.cuda.get_device_properties(local)
    gpu_id = None
    uuid = getattr(dev_props, "uuid", None)
    if uuid is not None:
        u = str(uuid)
        gpu_id = u if u.startswith("GPU-") else "GPU-" + u
    sampler = ClockSampler(gpu_id)
    launches0 = align.align_eval_stats(L)["kernel_launches"]
    align.align_profile(L, 1)
    sampler.start()
    time.sleep(0.5)  # let nvidia-smi start sampling
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_begin = time.time()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        T, mi, _ = step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_end = time.time()
    clocks = sampler.stop(t_begin, t_end)
    prof = align.align_profile(L, 2)
    align.align_profile(L, 0)
    launches = align.align_eval_stats(L)["kernel_launches"] - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    evals_per_step = P * LEVELS if args.mode == "search" else P
    value = ws * evals_per_step * args.steps / (total_ms / 1000.0)

    # ---- end to end through the C ABI from pinned host buffers ----
    A_pin = torch.from_numpy(pair.xyzA).pin_memory()
    B_pin = torch.from_numpy(pair.xyzB).pin_memory()
    A_h, B_h = A_pin.numpy(), B_pin.numpy()
    e2e_steps = max(1, min(args.steps, 50)) if args.mode == "search" else 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_s = 0.0
    for _ in range(e2e_steps):
        flush.zero_()  # the same cold L2 as the device-timed steps; not timed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        align.align_set_reference(L, A_h)
        align.align_search(L, B_h, init, RANGE, levels=LEVELS)  # returns T on the host: synchronised
        e2e_s += time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = ws * evals_per_step * e2e_steps / e2e_s if e2e_steps else None
    h2d = (pair.xyzA.shape[0] + pair.xyzB.shape[0]) * 12 + LEVELS * P * 48
    d2h = 24 + LEVELS * (8 + 12 + 4)

    # ---- measured peaks (micro-benchmarks on this GPU, clocks sampled while they run) ----
    peaks = measure_peaks(align, gpu_id) if not args.no_peaks else None

    # ---- roofline of the dominant kernel (eval) ----
    eval_ms = prof[0] / max(prof[2], 1)
    nB = pair.xyzB.shape[0]
    ops_per_launch = P * nB * OPS_MAP
    achieved = ops_per_launch / (eval_ms / 1000.0) / 1e12
    achieved_am = P * nB * OPS_MAP_AMORTISED / (eval_ms / 1000.0) / 1e12
    traffic = committed_traffic()
    if peaks is not None:
        peak = peaks["alu_lane_ops_per_s"] / 1e12
        basis = (f"measured: fastest of FP32 FFMA and INT32 add/xor issue micro-benchmarks on this GPU at "
                 f"{peaks['clocks']['sm_mhz']} MHz median SM clock (of measured peak)")
    else:
        peak = dev_props.multi_processor_count * 128 * 2070.0e6 / 1e12
        basis = "derived: SMs x 128 lanes x 2,070 MHz (of derived peak; micro-benchmarks skipped)"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "eval_pair_kernel (pose pairs; eval_kernel for single poses)",
                "eval_kernel_ms": eval_ms,
                "ops_per_launch": ops_per_launch,
                "ops_basis": f"{OPS_MAP} lane-ops per (point, pose) x {nB} points x {P} poses",
                "achieved_amortised": achieved_am, "frac_amortised": achieved_am / peak,
                "amortised_basis": f"{OPS_MAP_AMORTISED} lane-ops per (point, pose): the rotation shared by the "
                                   "translations of a lattice (the kernel reads pre-rotated copies)",
                "peak_basis": basis,
                "kernel_share_of_step": (prof[0] / total_ms) if total_ms > 0 else None}
    if peaks is not None:
        atom = P * occ * ATOMICS_PER_VOXEL / (eval_ms / 1000.0)
        roofline["shared_atomics"] = {
            "achieved_per_s": atom, "peak_per_s": peaks["smem_red_random_per_s"],
            "frac": atom / peaks["smem_red_random_per_s"],
            "basis": f"{ATOMICS_PER_VOXEL} atomics per occupied voxel x {occ} occupied voxels (lattice centre) x "
                     f"{P} poses; peak: shared red.add on random words (measured)"}
        roofline["mix_peak"] = {"lane_ops_per_s": peaks["keymix_lane_ops_per_s"],
                                "frac": achieved * 1e12 / peaks["keymix_lane_ops_per_s"],
                                "basis": "the voxel map's own instruction mix (with float-to-int conversions) "
                                         "as a micro-benchmark"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+i32", "data": "synthetic", "config": workload_config(pair, LEVELS), "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches), "clocks": clocks,
            "result_check": ({"T": [float(x) for x in T], "T_true": [float(x) for x in pair.T], "mi": mi}
                             if args.mode == "search" else {"argmax": int(am_dev.item()), "mi_max": float(mi_dev.max())})}
    if peaks is not None:
        line["peaks"] = peaks
    if args.mode == "eval":
        line["config"]["workload"] = (f"lidar-120k eval: set_reference + one align_eval_mi of {P} lattice poses "
                                      "(device-resident inputs and outputs)")
        line["config"]["poses_per_level"] = P
        line["config"]["levels"] = 1
        line["e2e"] = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.mode == "search":
        import oracle
        cores = oracle.host_cores()
        n_all, n_one = 4096, 2048
        rate, dt = oracle_rate(pair, n_all, cores)
        rate1, dt1 = oracle_rate(pair, n_one, 1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n_all} level-0 lattice poses (of 4,096) on the same pair, "
                                          f"{dt:.1f} s wall on {cores} threads (MI evaluations only)",
                                "one_core": {"value": rate1, "unit": UNIT, "cores": 1,
                                             "sample": f"the first {n_one} of those poses on 1 thread, "
                                                       f"{dt1:.1f} s wall"},
                                "host": host_cpu()}
    if rank == 0 and ws == 1 and args.mode == "search" and not args.no_refine:
        line["refine"] = run_refine(align, pair, L, np.array(T, dtype=np.float64))
    L.close()
    if rank == 0 and ws == 1 and args.mode == "search":
        if not args.no_batched:
            line["batched"] = run_batched(align, max(3, min(args.steps, 10)))
        if not args.no_serving:
            line["serving"] = run_serving(align, args.serve_slots)
        if not args.no_large:
            line["large"] = run_large(align, 2)
            # the same operation count over the same peak as the headline's roofline
            lg = line["large"]
            ops = lg["poses"] * lg["points"] * OPS_MAP
            lg["roofline"] = {"bound": "alu", "achieved": ops / (lg["eval_kernel_ms"] / 1000.0) / 1e12,
                              "peak": peak, "unit": "Tops/s",
                              "frac": ops / (lg["eval_kernel_ms"] / 1000.0) / 1e12 / peak,
                              "ops_basis": f"{OPS_MAP} lane-ops per (point, pose) x {lg['points']} points x "
                                           f"{lg['poses']} poses, eval kernels (exact path included)"}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------------------
# synthetic stand-ins for the paper's accuracy experiments (Figs. 4-5) and cost surfaces
# (Fig. 6); not part of the default run
# --------------------------------------------------------------------------------------
ACC_T_ERRORS = (1.0, 3.0, 5.0, 7.0, 9.0)
ACC_YAW_ERRORS = (2.0, 5.0, 10.0, 15.0, 20.0)
PAPER_SIMPLEX = np.array([8.0, 8.0, 1.0, 0.1, 0.1, 0.8])  # Sec. IV


def _rot_err(a, b):
    """Angle (rad) of R(a)^T R(b)."""
    Ra, Rb = scangen.rot_zyx(a), scangen.rot_zyx(b)
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return float(np.arccos(np.clip(c, -1.0, 1.0)))


def run_accuracy(args):
    """Final alignment error against the initial error, for the count (MI-N) and z-variance
    (MI-VARZ) features at 1 m voxels: Nelder-Mead from the identity with the paper's simplex
    (Algorithm 1), and lattice search + Nelder-Mead.  Pairs: 64-beam ray-cast scans with the
    true offset of the given size in a random direction."""
    from paper_1709_06948_gb300 import align
    import torch
    torch.cuda.set_device(0)
    n_pairs = args.pairs
    feats = {"MI-N": dict(feature=0, count_levels=7, var_levels=1), "MI-VARZ": dict(feature=1, count_levels=1,
                                                                                      var_levels=15)}
    rng = np.random.default_rng(scangen.SEED_BASE + 7)
    results = {}
    for kind, errors in (("translation_m", ACC_T_ERRORS), ("yaw_deg", ACC_YAW_ERRORS)):
        for e in errors:
            for k in range(n_pairs):
                a = rng.uniform(-math.pi, math.pi)
                if kind == "translation_m":
                    T = np.array([e * math.cos(a), e * math.sin(a), rng.uniform(-0.1, 0.1), 0.0, 0.0,
                                  math.radians(rng.uniform(-3, 3))])
                else:
                    r = rng.uniform(0, 2)
                    T = np.array([r * math.cos(a), r * math.sin(a), 0.0, 0.0, 0.0,
                                  math.radians(e) * (1 if rng.uniform() < 0.5 else -1)])
                pair = scangen.lidar_pair(seed=scangen.SEED_BASE + 1000 + 37 * k + int(10 * e), T=T)
                for fname, fk in feats.items():
                    spec = scangen.lidar_grid(1.0)
                    L = align.align_create_grid(spec.origin, spec.res_m, spec.dims, fk["feature"], fk["count_levels"],
                                                fk["var_levels"])
                    align.align_set_reference(L, pair.xyzA)
                    Tn, _, _ = align.align_refine_nm(L, pair.xyzB, np.zeros((1, 6)), step=PAPER_SIMPLEX, max_iter=150)
                    rngs = np.array([10.0, 10.0, 0.5, math.radians(2.0), math.radians(2.0), math.radians(25.0)])
                    Ts, _, _ = align.align_search(L, pair.xyzB, np.zeros(6), rngs, levels=5,
                                                  counts=(12, 12, 2, 2, 2, 12))
                    Tl, _, _ = align.align_refine_nm(L, pair.xyzB, Ts[None, :],
                                                     step=np.array([0.5, 0.5, 0.2, 0.01, 0.01, 0.03]), max_iter=60)
                    for meth, Tf in (("nm_paper_simplex", Tn[0]), ("lattice_then_nm", Tl[0])):
                        key = f"{fname}/{meth}/{kind}={e:g}"
                        r = results.setdefault(key, {"t_err": [], "r_err": []})
                        r["t_err"].append(float(np.linalg.norm(Tf[:3] - T[:3])))
                        r["r_err"].append(_rot_err(Tf, T))
                    L.close()
    summary = {k: {"mean_translation_error_m": float(np.mean(v["t_err"])),
                   "mean_rotation_error_rad": float(np.mean(v["r_err"])),
                   "success_rate_t_lt_0.5m": float(np.mean(np.array(v["t_err"]) < 0.5)), "pairs": len(v["t_err"])}
               for k, v in results.items()}
    print(json.dumps({"mode": "accuracy", "data": "synthetic (64-beam ray-cast pairs; the paper's Ford/KITTI data "
                                                  "are not available)", "grid": "80x80x8 @ 1 m",
                      "results": summary}))
    return 0


def run_surface(args):
    """MI over (t_x, t_y) on a 0.25 m grid within +-8 m of the truth, and over heading within
    +-30 deg at 0.5 deg, other parameters at the truth: the peak's offset from the truth and
    the number of strict local maxima (8-neighbourhood) of the 2-D surface."""
    from paper_1709_06948_gb300 import align
    import torch
    torch.cuda.set_device(0)
    pair = scangen.lidar_pair()
    out = {}
    for fname, feat in (("MI-N", (0, 7, 1)), ("MI-VARZ", (1, 1, 15))):
        spec = scangen.lidar_grid(1.0)
        L = align.align_create_grid(spec.origin, spec.res_m, spec.dims, *feat)
        align.align_set_reference(L, pair.xyzA)
        g = np.arange(-8.0, 8.0001, 0.25)
        etas = np.repeat(pair.T[None, :], len(g) * len(g), 0)
        etas[:, 0] = pair.T[0] + np.repeat(g, len(g))
        etas[:, 1] = pair.T[1] + np.tile(g, len(g))
        mi, am, _ = align.align_eval_mi(L, pair.xyzB, eta6=etas)
        S = mi.reshape(len(g), len(g))
        inner = S[1:-1, 1:-1]
        nb = np.stack([S[1 + dy:S.shape[0] - 1 + dy, 1 + dx:S.shape[1] - 1 + dx]
                       for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dy, dx) != (0, 0)])
        n_max = int(np.sum(np.all(inner > nb, axis=0)))
        h = np.arange(-30.0, 30.0001, 0.5)
        eh = np.repeat(pair.T[None, :], len(h), 0)
        eh[:, 5] = pair.T[5] + np.radians(h)
        mh, amh, _ = align.align_eval_mi(L, pair.xyzB, eta6=eh)
        out[fname] = {"xy_peak_offset_m": [float(etas[am][0] - pair.T[0]), float(etas[am][1] - pair.T[1])],
                      "xy_strict_local_maxima": n_max, "xy_grid": f"{len(g)}x{len(g)} at 0.25 m",
                      "heading_peak_offset_deg": float(h[amh]),
                      "heading_strict_local_maxima": int(np.sum((mh[1:-1] > mh[:-2]) & (mh[1:-1] > mh[2:])))}
        if args.surface_out:
            np.save(f"{args.surface_out}_{fname}_xy.npy", S)
            np.save(f"{args.surface_out}_{fname}_heading.npy", mh)
        L.close()
    print(json.dumps({"mode": "surface", "data": "synthetic 64-beam pair, grid 80x80x8 @ 1 m", "results": out}))
    return 0


SWEEP_WORKLOADS = ("lidar0.5", "lidar0.25", "large")


def run_sweeps(args):
    """Each way of sweeping poses (align_set_sweep kinds 0-2, kind 0 with the spill queues
    off, and the automatic choice) on 4,096 lattice poses of three grids: the 120k-point
    LiDAR pair at 0.5 m and 0.25 m (z-variance) and the large pair (260k points, 0.2 m, joint
    feature; every 8th pose of its 32,768-pose lattice).  Per kind: key partitions learned, eval-kernel time per launch
    (CUDA events, median over --steps launches after the partitions settle).  One JSON line."""
    import torch
    from paper_1709_06948_gb300 import align
    torch.cuda.set_device(0)
    names = [w for w in args.sweep_workloads.split(",") if w]
    bad = [w for w in names if w not in SWEEP_WORKLOADS]
    if bad:
        raise SystemExit(f"unknown workloads {bad}; choose from {SWEEP_WORKLOADS}")
    kinds = [k for k in args.sweep_kinds.split(",") if k]  # a kind, or "0nospill": one pose per CTA
    # sweeping B once per key partition instead of queueing the later partitions' runs
    res = []
    for name in names:
        if name == "large":
            pair = scangen.large_pair()
            spec, etas = pair.grid, scangen.large_poses()[::8]
        else:
            pair = scangen.lidar_pair()
            spec, etas = scangen.lidar_grid(float(name[5:])), scangen.lidar_poses()
        B = torch.from_numpy(pair.xyzB).cuda()
        row = {"workload": name, "points": int(pair.xyzB.shape[0]), "dims": list(spec.dims), "poses": len(etas)}
        ref_mi = None
        for kname in kinds:
            kind = int(kname.replace("nospill", ""))
            L = align.align_create_grid(spec.origin, spec.res_m, spec.dims, spec.feature, spec.count_levels,
                                        spec.var_levels)
            align.align_set_reference(L, pair.xyzA)
            align.align_set_sweep(L, kind)
            align.align_set_spill(L, "nospill" not in kname)
            prev = None
            for _ in range(8):  # until the kind and its partition count stay the same
                mi, am, _ = align.align_eval_mi(L, B, eta6=etas)
                st = align.align_eval_stats(L)
                cur = (st["sweep"], st["passes"])
                if cur == prev:
                    break
                prev = cur
            if ref_mi is None:
                ref_mi = mi
            times = []
            for _ in range(max(1, args.steps)):
                align.align_profile(L, 1)
                align.align_eval_mi(L, B, eta6=etas)
                ev_ms, _, n = align.align_profile(L, 2)
                times.append(ev_ms / max(n, 1))
            align.align_profile(L, 0)
            st = align.align_eval_stats(L)
            row[f"kind{kname}"] = {"sweep": align.SWEEP_KINDS.get(st["sweep"], st["sweep"]),
                                  "key_partitions": st["passes"],
                                  "eval_kernel_ms": round(statistics.median(times), 4),
                                  "same_mi_as_first_kind": bool(np.array_equal(mi, ref_mi))}
            L.close()
        res.append(row)
    print(json.dumps({"mode": "sweeps", "gpu": torch.cuda.get_device_name(0), "results": res}))
    return 0


def run_dense(args):
    """The 128-beam large scan (258k points; every 8th pose of its lattice: 4,096) on coarse
    240 m square z-variance grids at 1 m and 0.5 m, whose near-sensor voxels hold thousands of
    points: per call of align_eval_mi on one grid, the eval-kernel time (CUDA events, exact
    path included), the sweep kind, key partitions, table slots (the layout) and the poses
    the exact path finished, for the automatic choice and single poses.  One JSON line."""
    import torch
    from paper_1709_06948_gb300 import align
    torch.cuda.set_device(0)
    big = scangen.large_pair()
    etas = scangen.large_poses()[::8]
    B = torch.from_numpy(big.xyzB).cuda()
    out = []
    for res in (1.0, 0.5):
        n = int(round(240 / res))
        kw = dict(origin=(-120.0, -120.0, -5.0), res_m=res, dims=(n, n, int(round(20 / res))), feature=1,
                  count_levels=1, var_levels=15)
        for kind in (-1, 0):
            L = align.align_create_grid(**kw)
            align.align_set_reference(L, big.xyzA)
            align.align_set_sweep(L, kind)
            calls = []
            for _ in range(max(5, args.steps)):
                align.align_profile(L, 1)
                align.align_eval_mi(L, B, eta6=etas)
                ev, _, cnt = align.align_profile(L, 2)
                st = align.align_eval_stats(L)
                calls.append({"eval_ms": round(ev / max(cnt, 1), 3), "sweep": align.SWEEP_KINDS.get(st["sweep"]),
                              "key_partitions": st["passes"], "table_slots": st["table_slots"],
                              "exact_path_poses": int(len(align.align_eval_redo_poses(L)))})
            align.align_profile(L, 0)
            out.append({"res_m": res, "dims": kw["dims"], "kind": kind, "calls": calls})
            L.close()
    print(json.dumps({"mode": "dense", "gpu": torch.cuda.get_device_name(0), "points": int(big.xyzB.shape[0]),
                      "poses": len(etas), "results": out}))
    return 0


def run_peaks(args):
    """The measured peaks alone (one JSON line)."""
    import torch
    from paper_1709_06948_gb300 import align
    torch.cuda.set_device(0)
    props = torch.cuda.get_device_properties(0)
    uuid = getattr(props, "uuid", None)
    gpu_id = None if uuid is None else (str(uuid) if str(uuid).startswith("GPU-") else "GPU-" + str(uuid))
    print(json.dumps({"mode": "peaks", "gpu": props.name, "sms": props.multi_processor_count,
                      "peaks": measure_peaks(align, gpu_id)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="search",
                    choices=["search", "eval", "accuracy", "surface", "peaks", "sweeps", "dense"],
                    help="search: reference build + 6-level search per step (default); "
                         "eval: reference build + one align_eval_mi of --poses poses per step; "
                         "accuracy: final error vs initial error (synthetic Figs. 4-5); "
                         "surface: MI cost surfaces around the truth (synthetic Fig. 6); "
                         "peaks: the throughput micro-benchmarks alone; "
                         "sweeps: eval-kernel time of each way of sweeping poses on three grids; "
                         "dense: a dense 128-beam scan on coarse grids, per call (layout and partitions learned)")
    ap.add_argument("--sweep-workloads", default=",".join(SWEEP_WORKLOADS), help="sweeps mode: workloads")
    ap.add_argument("--sweep-kinds", default="-1,0,0nospill,1,2",
                    help="sweeps mode: align_set_sweep kinds (0nospill: kind 0 with align_set_spill off)")
    ap.add_argument("--pairs", type=int, default=4, help="accuracy mode: pairs per initial error")
    ap.add_argument("--surface-out", default=None, help="surface mode: prefix of .npy files for the surfaces")
    ap.add_argument("--poses", type=int, default=4096)
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-pair batched leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-requests leg")
    ap.add_argument("--no-refine", action="store_true", help="skip the Nelder-Mead refinement leg")
    ap.add_argument("--no-large", action="store_true", help="skip the large-grid leg")
    ap.add_argument("--serve-slots", type=int, default=SERVE_SLOTS, help="request slots of the served leg")
    ap.add_argument("--no-peaks", action="store_true", help="skip the peak micro-benchmarks")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "accuracy":
        return run_accuracy(args)
    if args.mode == "surface":
        return run_surface(args)
    if args.mode == "peaks":
        return run_peaks(args)
    if args.mode == "sweeps":
        return run_sweeps(args)
    if args.mode == "dense":
        return run_dense(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
