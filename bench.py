#!/usr/bin/env python3
"""DSES registration benchmark on B300.

One step = one full registration (Algorithm 2: every rotation of the grid
votes, counts inliers, is scored, and the argmin is returned). The default
workload is the robot-pose-like problem, the largest single-GPU
configuration: a 20,000-point target (a ~0.3 m assembly of primitives), a
5,000-point depth-view source with 30% clutter, the N_side 32 Hopf grid
(2,359,296 rotations) plus Euler boxes (7^3, 0.3125 deg) around the best 32
candidates, a 3 mm translation lattice over +-5 cm, the Huber metric read
from the target's 128^3 FP32 distance grid. --workload modelnet_like runs the
ModelNet-shaped problem (294,912 rotations, 717 x 1,024 points, truncated
L2) in the same form; the other workloads print their own lines.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]

Under torchrun every rank registers its own problem of the same shape (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rotation-candidates x source-points / s"
UNIT = "rot*pts/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# recipe unit counts: 148 SMs x 128 FP32 lanes at the 2032 MHz maximum SM clock
ALU_PEAK_OPS = 148 * 128 * 2032e6
# algorithmic work of the rotation pass: per (rotation, source point, target
# point) pair 3 FP32 operations and one shared-memory histogram increment; per
# (rotation, source point) 15 FP32 operations (the rotation R x_i)
OPS_PER_PAIR = 4
OPS_PER_ROT_SRC = 15
# DRAM bytes (read + write) of one vote_kernel launch per workload, from an
# ncu capture of the current kernel on the same problem at N_side 4 (None: no
# capture of the current kernel): a launch reads its inputs (KB) once, so the
# figure does not grow with the rotations and is used unscaled.
VOTE_DRAM_BYTES = {"robot_like": None, "modelnet_like": 269056}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: 3 robot-like, 10 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--hopf-n", type=int, default=0,
                    help="grid N_side (0: the workload's own, 32 robot-like / 16 ModelNet-shaped; smaller for profiling)")
    ap.add_argument("--points-per-thread", type=int, default=0, help="vote launch shape (0: library default)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["robot_like", "modelnet_like", "batched", "serving", "robot_local", "quality",
                                           "sweep", "tiny"],
                    default="robot_like",
                    help="robot_like (default) / modelnet_like: the benchmark line; the others print their own")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--quality-count", type=int, default=64, help="quality: number of problems")
    ap.add_argument("--rotated-frame", action="store_true", help="quality: both clouds in a rotated frame")
    ap.add_argument("--refine-iterations", type=int, default=3, help="quality: translation refinement steps")
    ap.add_argument("--refine-top-k", type=int, default=16, help="quality: Euler-box second pass around the best k")
    ap.add_argument("--refine-K", type=int, default=3, help="quality: Euler-box half-size of the second pass")
    ap.add_argument("--refine-delta-deg", type=float, default=1.0, help="quality: Euler-box step (degrees)")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: arrival window (s)")
    ap.add_argument("--queue-cap", type=int, default=64, help="serving: requests waiting before arrivals are refused")
    ap.add_argument("--seq-sample", type=int, default=400, help="serving: admitted requests re-run as blocking calls")
    ap.add_argument("--serve-iter-pairs", type=float, default=0, help="serving: pair votes per iteration (0: library default)")
    ap.add_argument("--split", choices=["problems", "rotations"], default="problems",
                    help="robot_like / modelnet_like under torchrun: one problem per rank (weak scaling) or one "
                         "problem's rotations sharded over the ranks (strong scaling)")
    return ap.parse_args()


def dist_setup(ngpu_flag):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.f = None
        self.path = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w", prefix="clocks", suffix=".csv", delete=False)
            self.path = self.f.name
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            if self.f is not None:
                self.f.close()
                os.unlink(self.path)
                self.f = None
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def workload(name, seed, hopf_n=0):
    """(problem, target grid cap, rotations per registration) of a benchmark line's workload."""
    from paper_2502_00115_b300 import synth

    if name == "robot_like":
        p = synth.robot_like_problem(seed, hopf_n=hopf_n or 32)
        return p, p.grid_cap, p.n_rotations
    p = synth.modelnet_like_problem(seed, hopf_n=hopf_n or 16)
    return p, 2 * p.tau, 72 * p.hopf_n**3


def gpu_params(capi, p):
    return capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau, huber_h=p.huber_h,
                            t_half=p.t_half, nn_mode="grid", refine_top_k=p.refine_top_k, refine_K=p.refine_K,
                            refine_delta_r=p.refine_delta_r)


def config_dict(name, p):
    n1 = 72 * p.hopf_n**3
    box = math.floor((p.t_center[0] + p.t_half[0]) / p.delta_t) - math.ceil((p.t_center[0] - p.t_half[0]) / p.delta_t) + 1
    c = {"workload": f"{name}_single_problem", "target_points": int(len(p.Y)), "source_points": int(len(p.X)),
         "rotations": int(p.n_rotations), "rotation_grid": f"hopf N_side={p.hopf_n} ({n1})", "metric": p.metric,
         "tau": p.tau, "epsilon": p.epsilon, "delta_t": p.delta_t,
         "translation_box": f"+-{p.t_half[0]} per axis ({box}^3 lattice)", "distance_grid": "128^3 fp32",
         "l2": "flushed between steps (512 MB write)"}
    if p.refine_top_k:
        c["second_pass"] = (f"Euler boxes (2K+1)^3, K={p.refine_K}, {math.degrees(p.refine_delta_r):.4g} deg, "
                            f"around the best {p.refine_top_k}")
    if name == "robot_like":
        c["huber_h"] = p.huber_h
        c["source"] = "3,500 visible-surface points (sigma 1 mm) + 1,500 clutter points (30%)"
    return c


# ---------------------------------------------------------------------------
# multi-rank aggregation (one process per GPU; each rank registers its own
# problem, so ranks exchange only their timings)


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise max of per-rank timing values (identity on one rank)."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(world_size, steps, units_per_step, total_ms):
    """Whole-job units per second: every rank processed `steps` steps of
    `units_per_step` units, and the job took the slowest rank's time."""
    return world_size * steps * units_per_step / (total_ms / 1000.0)


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)


def oracle_sample(p, target_s, threads):
    """Time the FP64 oracle (Algorithm 2 over an even-stride sample of the
    first-pass grid, every sampled rotation scored on the prebuilt distance
    field); returns a runner, the sample size and the per-rotation time."""
    import oracle

    oracle.build()
    n_all = 72 * p.hopf_n**3
    P = oracle.params_from_problem(p, nn_mode="grid", grid_cap=p.grid_cap or 2 * p.tau, refine_top_k=0)
    field = oracle.Field(p.Y, P.grid_res, P.grid_cap, threads=threads)

    def run(count, offset=0):
        stride = max(1, n_all // count)
        idx = (np.arange(count) * stride + offset) % n_all
        Rs = np.stack([oracle.hopf_rotation(p.hopf_n, int(i)) for i in idx])
        t0 = time.perf_counter()
        oracle.register_field_threads(p.X, p.Y, Rs, P, field, threads)
        return time.perf_counter() - t0

    probe = threads
    dt = run(probe)
    per_rot = dt / probe
    count = int(max(probe, min(n_all, target_s / per_rot)))
    return run, count, per_rot, field


def cpu_baseline(p, target_s):
    threads = os.cpu_count() or 1
    run, count, per_rot, field = oracle_sample(p, target_s, threads)
    dt = run(count, offset=1)
    field.close()
    return {"value": count * len(p.X) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{count} of {72 * p.hopf_n**3} first-pass rotations (even stride) of the same problem, FP64 "
                      f"Algorithm 2 fanned over {threads} threads, every sampled rotation scored, distance field "
                      f"prebuilt (not timed), {dt:.1f} s"}


def reference_arm(args, ws, rank):
    if rank != 0:
        return
    name = args.workload if args.workload in ("robot_like", "modelnet_like") else "robot_like"
    p, cap, n_rot = workload(name, args.seed, args.hopf_n)
    threads = os.cpu_count() or 1
    steps = args.steps or 3
    # each step: a bounded rotation sample sized to ~4 s so K + W steps stay within minutes
    run, count, per_rot, field = oracle_sample(p, 4.0, threads)
    for w in range(args.warmup):
        run(count, offset=w + 1)
    times = [run(count, offset=100 + k) for k in range(steps)]
    field.close()
    tot = sum(times)
    value = steps * count * len(p.X) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(name, p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{count} first-pass rotations per step (even stride, shifted per step) of "
                                       f"{72 * p.hopf_n**3}; distance field prebuilt"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm


def ours(args, ws, rank, local):
    import torch

    from paper_2502_00115_b300 import build, capi

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    if rank == 0 or ws > 1:
        build.build()
    if dist:
        dist.barrier()
    name = args.workload
    steps = args.steps or (3 if name == "robot_like" else 10)
    p, cap, n_rot = workload(name, args.seed + rank, args.hopf_n)
    units = n_rot * len(p.X)
    stream = torch.cuda.Stream()
    ctx = capi.Context(local, stream.cuda_stream)
    tgt = ctx.create_target(p.Y, grid_cap=cap)
    params = gpu_params(capi, p)
    grid = capi.hopf_grid(p.hopf_n)
    Xd = torch.from_numpy(p.X).cuda()
    Xh = torch.from_numpy(p.X).pin_memory()
    torch.cuda.synchronize()
    pb_dev = ctx.problem(tgt, None, grid, params, src_ptr=Xd.data_ptr(), n_src=len(p.X))
    pb_host = ctx.problem(tgt, Xh.numpy(), grid, params)
    pb_host.src = Xh.data_ptr()  # pinned host buffer
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ctx.set_option("record_timing", 1)
    if args.points_per_thread:
        ctx.set_option("points_per_thread", args.points_per_thread)

    for w in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        ctx.register(pb_host if w % 2 else pb_dev)

    # device-resident inputs, CUDA events on the library's stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    pass_ns, count_ns, launches_per_step, votes = [], [], [], []
    results = []
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = ctx.get_option("kernel_launches")
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[k][0].record(stream)
        r = ctx.register(pb_dev)
        ev[k][1].record(stream)
        results.append(capi.result_dict(r))
        pass_ns.append(ctx.get_option("last_pass_ns"))
        count_ns.append(ctx.get_option("last_count_ns"))
        launches_per_step.append(ctx.get_option("last_pass_launches"))
        votes.append(ctx.get_option("last_votes_total"))
    torch.cuda.synchronize()
    launches = ctx.get_option("kernel_launches") - launches0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)

    # end to end through the public API: pinned host source in, result out
    e2e_s = []
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        ctx.register(pb_host)
        e2e_s.append(time.perf_counter() - t0)
    clk = clocks.stop()
    shapes = {"points_per_thread_mask": ctx.get_option("last_p_mask"),
              "tile_rotations_max": ctx.get_option("last_tile_max"),
              "culled_vote": bool(ctx.get_option("last_vote_sparse")),
              "paired_groups": bool(ctx.get_option("last_vote_paired"))}

    total_ms, e2e_tot = max_over_ranks([total_ms, sum(e2e_s)], dist, device="cuda")
    ctx.close()
    if rank != 0:
        return
    try:
        from paper_2502_00115_b300 import peaks

        pk = peaks.run(local)
    except Exception as e:  # the microbenchmark is auxiliary evidence
        pk = {"error": str(e)}
    value = job_throughput(ws, steps, units, total_ms)
    # the vote kernel (the dominant kernel): its launches per step (first pass
    # and, with a second pass, the Euler boxes) timed with CUDA events on the
    # library's stream; per launch = per step / launches per step
    pass_s = statistics.mean(pass_ns) / 1e9
    n_launch = max(1, int(statistics.mean(launches_per_step)))
    incr = statistics.mean(votes)  # in-box histogram increments per step
    atomic_peak = pk.get("smem_atomic_random_per_s")
    achieved = incr / pass_s
    # ALU work of the windowed formulation: 4 operations per in-box pair (3
    # FP32 and the increment) + 15 FP32 per (rotation, source point) for R x_i
    ops = incr * OPS_PER_PAIR + n_rot * len(p.X) * OPS_PER_ROT_SRC
    dense_pairs = n_rot * len(p.X) * len(p.Y)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps, "warmup": args.warmup,
        "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": config_dict(name, p),
        "registrations_per_s": ws * steps / (total_ms / 1000),
        "latency_ms": {"p50": 1000 * float(np.percentile(e2e_s, 50)), "p99": 1000 * float(np.percentile(e2e_s, 99))},
        "roofline": {
            "bound": "smem_atomic", "kernel": "vote_kernel",
            "achieved": achieved / 1e12, "peak": (atomic_peak / 1e12) if atomic_peak else None,
            "unit": "T increments/s", "frac": (achieved / atomic_peak) if atomic_peak else None,
            "traffic": VOTE_DRAM_BYTES.get(name), "traffic_unit": "DRAM bytes per launch (ncu, N_side 4 capture)",
            "increments_per_launch": incr / n_launch, "launches_per_step": n_launch,
            "kernel_ms_per_launch": 1000 * pass_s / n_launch, "kernel_ms_per_step": 1000 * pass_s,
            "peak_source": "measured in this run: red.shared.add.u32 on random bins of a 46,575-word histogram "
                           "(one CTA of 1,024 threads per SM)",
            "issued_per_s": None},
        "alu_roofline": {
            "bound": "alu", "achieved": ops / pass_s / 1e12, "peak": ALU_PEAK_OPS / 1e12, "unit": "Tops/s",
            "frac": ops / pass_s / ALU_PEAK_OPS, "ops_per_step": ops,
            "peak_source": "recipe unit counts: 148 SMs x 128 lanes x 2032 MHz",
            "frac_of_measured_ffma": (ops / pass_s / pk["ffma_per_s"]) if "ffma_per_s" in pk else None},
        # the fused inlier-count / score kernel: per (rotation, source point) the
        # trilinear distance-grid lookup reads its 8 corners as two 16-byte
        # corner blocks from the L2-resident grid; bound by random L2 gathers
        "score_roofline": {
            "kernel": "count_kernel", "bound": "l2_gather",
            "achieved": n_rot * len(p.X) * 2 / (statistics.mean(count_ns) / 1e9),
            "peak": pk.get("l2_gather_16B_per_s"), "unit": "16-byte gathers/s",
            "frac": (n_rot * len(p.X) * 2 / (statistics.mean(count_ns) / 1e9) / pk["l2_gather_16B_per_s"])
            if "l2_gather_16B_per_s" in pk else None,
            "kernel_ms_per_step": statistics.mean(count_ns) / 1e6,
            "peak_source": "measured in this run: random aligned 16-byte loads from a 32 MB table"},
        "work_per_step": {"in_box_increments": incr, "dense_pairs": dense_pairs,
                          "in_box_fraction_of_dense": incr / dense_pairs},
        "launch_shapes": shapes,
        "peaks_measured": pk,
        "e2e": {"value": job_throughput(ws, steps, units, 1000 * e2e_tot), "unit": UNIT,
                "h2d_bytes_per_step": int(p.X.nbytes),
                "d2h_bytes_per_step": 72},
        "gpu_launches": int(launches),
        "clocks": clk,
        "result": {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in results[-1].items()},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# other configurations: batched problems, served requests


def batched(args, ws, rank, local):
    """64 uneven problems in one persistent launch (autotuned launch shapes) vs
    the same batch with fixed shapes and vs one launch per problem."""
    import torch

    from paper_2502_00115_b300 import build, capi, synth

    torch.cuda.set_device(local)
    build.build()
    probs = synth.batch_problems(args.seed, count=args.batch_count)
    ctx = capi.Context(local)
    targets = [ctx.create_target(p.Y, grid_cap=2 * p.tau) for p in probs]
    pbs = [ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n),
                       capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau,
                                        t_half=p.t_half)) for t, p in zip(targets, probs)]
    units = sum(72 * p.hopf_n**3 * len(p.X) for p in probs)
    pairs = sum(72 * p.hopf_n**3 * len(p.X) * len(p.Y) for p in probs)
    steps = args.steps or 3

    def timed(fn, n):
        ts = []
        for _ in range(n):
            t0 = time.perf_counter()
            out = fn()
            ts.append(time.perf_counter() - t0)
        return statistics.mean(ts), out

    for _ in range(max(1, args.warmup)):  # the first call also tunes every problem-size bucket
        ctx.register_batch(pbs)
    tb, rb = timed(lambda: ctx.register_batch(pbs), steps)
    shapes = {"points_per_thread_mask": ctx.get_option("last_p_mask"),
              "tile_rotations_max": ctx.get_option("last_tile_max")}
    tsq, rs = timed(lambda: [ctx.register(pb) for pb in pbs], max(1, steps // 2))
    ctx.set_option("autotune", 0)
    ctx.register_batch(pbs)
    tfix, rf = timed(lambda: ctx.register_batch(pbs), steps)
    fixed_shapes = {"points_per_thread_mask": ctx.get_option("last_p_mask"),
                    "tile_rotations_max": ctx.get_option("last_tile_max")}
    ctx.set_option("autotune", 1)
    same = all(capi.result_dict(a)["rot_index"] == capi.result_dict(b)["rot_index"] == capi.result_dict(c)["rot_index"]
               for a, b, c in zip(rb, rs, rf))
    ctx.close()
    print(json.dumps({
        "workload": "batched", "metric": METRIC, "value": units / tb, "unit": UNIT, "problems": len(probs),
        "registrations_per_s": len(probs) / tb, "s_per_batch": tb, "pair_votes_per_s": pairs / tb,
        "launch_shapes_autotuned": shapes,
        "fixed_shapes": {"value": units / tfix, "s_per_batch": tfix, "launch_shapes": fixed_shapes},
        "sequential": {"value": units / tsq, "registrations_per_s": len(probs) / tsq, "s_per_batch": tsq},
        "batch_over_sequential": tsq / tb, "autotuned_over_fixed": tfix / tb,
        "steps": steps, "results_equal": same,
        "config": {"targets": f"{min(len(p.Y) for p in probs)}..{max(len(p.Y) for p in probs)} pts",
                   "sources": f"{min(len(p.X) for p in probs)}..{max(len(p.X) for p in probs)} pts",
                   "rotations": f"{min(72 * p.hopf_n**3 for p in probs)}..{max(72 * p.hopf_n**3 for p in probs)}"},
    }), flush=True)


def fcfs_queue(arrivals, service, cap):
    """First-come first-served single server with at most `cap` requests
    waiting (an arrival that finds cap waiting is rejected): (latencies of the
    admitted, number rejected, time the last one finished)."""
    done_at, lat, rejected, free_at = [], [], 0, 0.0
    for a, sv in zip(arrivals, service):
        # requests admitted before a that are still waiting at time a
        started_by = [d - s for d, s in done_at[-(cap + 2):]]
        waiting = sum(1 for st in started_by if st > a)
        if waiting >= cap:
            rejected += 1
            continue
        start = max(a, free_at)
        free_at = start + sv
        done_at.append((free_at, sv))
        lat.append(free_at - a)
    return lat, rejected, free_at


def serving(args, ws, rank, local):
    """Poisson arrivals over resident targets through dses_submit / dses_poll,
    with load shedding at the queue capacity (--queue-cap requests waiting;
    later arrivals are refused with DSES_ERR_QUEUE_FULL and counted), against
    the same requests as sequential blocking calls (a first-come first-served
    queue with the same capacity)."""
    import torch

    from paper_2502_00115_b300 import build, capi, synth

    torch.cuda.set_device(local)
    build.build()
    wl = synth.serving_workload(args.seed, rate=args.rate, duration=args.duration)
    ctx = capi.Context(local)
    ctx.set_option("serve_queue_cap", args.queue_cap)
    if args.serve_iter_pairs:
        ctx.set_option("serve_iter_pairs", int(args.serve_iter_pairs))
    tmap = {}
    for i, Y in enumerate(wl.targets):
        tmap[i] = ctx.create_target(Y, grid_cap=0.1)
    reqs = []
    first_of_kind = {}
    for (t_arr, ti, p) in wl.requests:
        pb = ctx.problem(tmap[ti], p.X, capi.hopf_grid(p.hopf_n),
                         capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau,
                                          t_half=p.t_half))
        reqs.append((t_arr, pb, 72 * p.hopf_n**3 * len(p.X)))
        first_of_kind.setdefault((ti, len(p.X).bit_length()), pb)
    # warm the path outside both measurements: the grid, every target's
    # per-epsilon cell list and per-delta bounds (built on a target's first
    # use), and the autotuned launch shape of every (target, source size)
    # bucket (the serving worker runs no tuning trials)
    for pb in first_of_kind.values():
        ctx.register(pb)
    for key in ("serve_max_active", "serve_busy_ns", "serve_iterations"):
        ctx.set_option(key, 0)
    pending = {}
    lat, admitted = [], []
    rejected = 0
    units = 0
    t0 = time.perf_counter()
    nxt = 0
    while nxt < len(reqs) or pending:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt][0] <= now:
            st, tk = capi.dses_submit(ctx.h, reqs[nxt][1])
            if st == capi.DSES_ERR_QUEUE_FULL:
                rejected += 1
            else:
                assert st == capi.DSES_OK, capi.status_string(st)
                pending[tk] = (t0 + reqs[nxt][0], reqs[nxt][2])
                admitted.append(nxt)
            nxt += 1
        for tk in list(pending):
            st, r = ctx.poll(tk)
            if st != capi.DSES_NOT_READY:
                t_sub, u = pending.pop(tk)
                lat.append(time.perf_counter() - t_sub)
                units += u
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    max_active = ctx.get_option("serve_max_active")
    ctx_max_batch = ctx.get_option("serve_max_batch")
    busy_s = ctx.get_option("serve_busy_ns") / 1e9
    iterations = ctx.get_option("serve_iterations")
    # the same requests as sequential single-problem launches (blocking
    # dses_register one after another): measured service times of the
    # admitted requests (at most --seq-sample of them), and the latencies of a
    # first-come first-served queue with the same arrivals and capacity
    sample = admitted[: args.seq_sample]
    svc = []
    for i in sample:
        t1 = time.perf_counter()
        ctx.register(reqs[i][1])
        svc.append(time.perf_counter() - t1)
    ctx.close()
    arrivals = [r[0] for r in reqs]
    service = [svc[k % len(svc)] for k in range(len(reqs))]  # measured times, cycled over the stream
    # the server holds up to queue_cap waiting requests plus serve_max_batch
    # admitted ones; the queue of blocking calls gets the same room (all but
    # the one in service wait)
    room = args.queue_cap + ctx_max_batch - 1
    seq_lat, seq_rej, seq_end = fcfs_queue(arrivals, service, room)
    print(json.dumps({
        "workload": "serving", "metric": METRIC, "value": units / wall, "unit": UNIT,
        "offered_rate": args.rate, "arrival_window_s": args.duration, "requests_offered": len(reqs),
        "serve_iter_pairs": args.serve_iter_pairs or "library default",
        "admitted": len(admitted), "rejected_queue_full": rejected, "queue_cap": args.queue_cap,
        "registrations_per_s": len(lat) / wall, "max_requests_in_flight": max_active,
        "latency_ms": {"p50": 1000 * float(np.percentile(lat, 50)), "p99": 1000 * float(np.percentile(lat, 99)),
                       "max": 1000 * max(lat)},
        "wall_s": wall, "device_busy_s": busy_s, "iterations": iterations,
        "device_ms_per_registration": 1000 * busy_s / max(1, len(lat)),
        "sequential": {"registrations_per_s": 1.0 / statistics.mean(svc), "service_ms_mean": 1000 * statistics.mean(svc),
                       "service_sample": len(svc), "fcfs_room": room, "fcfs_rejected": seq_rej,
                       "fcfs_latency_ms": {"p50": 1000 * float(np.percentile(seq_lat, 50)),
                                           "p99": 1000 * float(np.percentile(seq_lat, 99))},
                       "fcfs_registrations_per_s": len(seq_lat) / max(seq_end, 1e-9)},
        "data": "synthetic",
    }), flush=True)


def pose_errors(R_est, t_est, R_true, t_true) -> dict:
    """Pose-error measures of Section V-A. Isotropic (Yew & Lee 2020): the
    angle of R_true^T R_est in degrees and ||t_est - t_true||. Mean absolute
    (Wang & Solomon 2019): the mean over the three 'zyx' Euler angles of
    |angle(R_est) - angle(R_true)| in degrees, and the mean over the axes of
    |t_est - t_true|."""
    from scipy.spatial.transform import Rotation

    R_est, R_true = np.asarray(R_est, np.float64), np.asarray(R_true, np.float64)
    c = (np.trace(R_true.T @ R_est) - 1.0) / 2.0
    mie_r = float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))
    mie_t = float(np.linalg.norm(np.asarray(t_est, np.float64) - t_true))
    e_est = Rotation.from_matrix(R_est).as_euler("zyx", degrees=True)
    e_true = Rotation.from_matrix(R_true).as_euler("zyx", degrees=True)
    mae_r = float(np.mean(np.abs(e_est - e_true)))
    mae_t = float(np.mean(np.abs(np.asarray(t_est, np.float64) - t_true)))
    return {"mie_r": mie_r, "mie_t": mie_t, "mae_r": mae_r, "mae_t": mae_t}


def summarise_errors(errs: list[dict]) -> dict:
    """Means of the four measures and the recall (MAE(R) < 1 deg and MAE(t) < 0.1)."""
    out = {k: float(np.mean([e[k] for e in errs])) for k in ("mie_r", "mie_t", "mae_r", "mae_t")}
    out["recall"] = float(np.mean([(e["mae_r"] < 1.0) and (e["mae_t"] < 0.1) for e in errs]))
    return out


def quality(args, ws, rank, local):
    """Pose quality of Section V-A on synthetic ModelNet-shaped problems: Euler
    angles in [-45, 45] deg, translations in [-0.5, 0.5]^3, one registration
    per problem (the Hopf grid, then Euler boxes around the best candidates,
    the local search of Algorithm 2's loops), errors of the voxel-centre
    translation t* and of the sub-voxel refined one."""
    import torch

    from paper_2502_00115_b300 import build, capi, synth

    torch.cuda.set_device(local)
    build.build()
    ctx = capi.Context(local)
    raw, ref, times = [], [], []
    for k in range(args.quality_count):
        p = synth.modelnet_like_problem(args.seed + k, hopf_n=args.hopf_n or 16, max_euler_deg=45.0,
                                        rotated_frame=args.rotated_frame)
        t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
        pr = capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau, t_half=p.t_half,
                              refine_top_k=args.refine_top_k, refine_K=args.refine_K,
                              refine_delta_r=math.radians(args.refine_delta_deg))
        pb = ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), pr)
        t0 = time.perf_counter()
        r = capi.result_dict(ctx.register(pb))
        t1 = time.perf_counter()
        tr, _ = ctx.refine_translation(t, p.X, r["R"], r["t"], p.epsilon, args.refine_iterations)
        times.append((t1 - t0, time.perf_counter() - t1))
        raw.append(pose_errors(r["R"], r["t"], p.R_true, p.t_true))
        ref.append(pose_errors(r["R"], tr, p.R_true, p.t_true))
        ctx.destroy_target(t)
    ctx.close()
    a, b = summarise_errors(raw), summarise_errors(ref)
    print(json.dumps({
        "workload": "quality_modelnet_like", "metric": "recall (MAE(R) < 1 deg and MAE(t) < 0.1)",
        "value": b["recall"], "unit": "fraction", "higher_is_better": True, "problems": args.quality_count,
        "rotated_frame": bool(args.rotated_frame), "rotation_grid": f"hopf N_side={args.hopf_n or 16}",
        "voxel_centre_t": a, "refined_t": b, "refine_iterations": args.refine_iterations,
        "second_pass": {"top_k": args.refine_top_k, "K": args.refine_K, "delta_deg": args.refine_delta_deg},
        "register_s_mean": statistics.mean(x[0] for x in times),
        "refine_ms_mean": 1e3 * statistics.mean(x[1] for x in times), "data": "synthetic",
    }), flush=True)


def sweep(args, ws, rank, local):
    """Registration time against the search range (the compute-time study of
    Section V): rotation range swept at a +-0.2 translation box, translation
    range swept at +-45 deg, on Euler-box grids (step 2.5 deg) centred on the
    identity, ModelNet-shaped clouds, the translation box centred on a 0.1
    rounding of the true translation (a local search around a prior)."""
    import torch

    from paper_2502_00115_b300 import build, capi, synth

    torch.cuda.set_device(local)
    build.build()
    ctx = capi.Context(local)
    ctx.set_option("record_timing", 1)
    step = math.radians(2.5)
    points = [("rotation", deg, 0.2) for deg in (5.0, 10.0, 20.0, 30.0, 45.0)]
    points += [("translation", 45.0, s) for s in (0.05, 0.1, 0.2, 0.4, 0.8)]
    rows = []
    for kind, deg, half in points:
        p = synth.modelnet_like_problem(args.seed, max_euler_deg=deg)
        K = int(round(deg / 2.5))
        t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
        centre = tuple(float(v) for v in np.round(p.t_true, 1))
        pr = capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau, t_center=centre,
                              t_half=(half, half, half))
        pb = ctx.problem(t, p.X, capi.euler_box_grid(np.eye(3), K, step), pr)
        for _ in range(max(1, args.warmup)):
            ctx.register(pb)
        ts = []
        for _ in range(max(1, args.steps)):
            t0 = time.perf_counter()
            r = capi.result_dict(ctx.register(pb))
            ts.append(time.perf_counter() - t0)
        ctx.destroy_target(t)
        e = pose_errors(r["R"], r["t"], p.R_true, p.t_true)
        rows.append({"sweep": kind, "rotation_range_deg": deg, "translation_half": half,
                     "rotations": (2 * K + 1) ** 3, "ms_per_registration": 1e3 * statistics.median(ts),
                     "vote_ms": ctx.get_option("last_pass_ns") / 1e6,
                     "count_ms": ctx.get_option("last_count_ns") / 1e6,
                     "culled_vote": bool(ctx.get_option("last_vote_sparse")),
                     "rotation_error_deg": e["mie_r"], "translation_error": e["mie_t"]})
    ctx.close()
    print(json.dumps({"workload": "search_range_sweep", "metric": "ms per registration", "unit": "ms",
                      "higher_is_better": False, "data": "synthetic", "euler_step_deg": 2.5,
                      "source_points": len(p.X), "target_points": len(p.Y), "points": rows}), flush=True)


def robot_local(args, ws, rank, local):
    """The paper's robot-experiment search ranges (local search of +-5 deg and
    +-1.6 cm around a prior pose) on the synthetic robot-like clouds: Euler box
    of 0.5 deg steps (21^3 rotations) around a prior 2.7 deg and 5.4 mm off
    the true pose, 3 mm lattice."""
    import torch

    from paper_2502_00115_b300 import build, capi, synth

    torch.cuda.set_device(local)
    build.build()
    p = synth.robot_like_problem(args.seed, hopf_n=2, refine_top_k=0)
    ctx = capi.Context(local)
    ctx.set_option("record_timing", 1)
    t = ctx.create_target(p.Y, grid_cap=p.grid_cap)
    a, b, c = np.radians([2.0, -1.5, 1.0])
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(c), -math.sin(c)], [0, math.sin(c), math.cos(c)]])
    R0 = np.asarray(p.R_true) @ Rz @ Ry @ Rx
    t0 = tuple(float(v) for v in np.asarray(p.t_true) + np.array([0.004, -0.003, 0.002]))
    K, step = 10, math.radians(0.5)
    pr = capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau, huber_h=p.huber_h,
                          t_center=t0, t_half=(0.016, 0.016, 0.016))
    pb = ctx.problem(t, p.X, capi.euler_box_grid(R0, K, step), pr)
    for _ in range(max(1, args.warmup)):
        ctx.register(pb)
    ts, vote = [], []
    for _ in range(max(1, args.steps)):
        t1 = time.perf_counter()
        r = capi.result_dict(ctx.register(pb))
        ts.append(time.perf_counter() - t1)
        vote.append(ctx.get_option("last_pass_ns") / 1e6)
    modes = {"culled": ctx.get_option("last_vote_sparse"), "paired": ctx.get_option("last_vote_paired")}
    ctx.close()
    n_rot = (2 * K + 1) ** 3
    e = pose_errors(r["R"], r["t"], p.R_true, p.t_true)
    print(json.dumps({
        "workload": "robot_local", "metric": METRIC, "value": n_rot * len(p.X) / statistics.median(ts),
        "unit": UNIT, "ms_per_registration": 1e3 * statistics.median(ts), "vote_ms": statistics.median(vote),
        "rotations": n_rot, "source_points": len(p.X), "target_points": len(p.Y),
        "search": "+-5 deg (Euler box, 0.5 deg) x +-1.6 cm (3 mm lattice)", "vote_modes": modes,
        "rotation_error_deg": e["mie_r"], "translation_error_m": e["mie_t"], "data": "synthetic",
    }), flush=True)


def tiny_cpu_baseline(p, threads):
    """cpu_baseline leg of the tiny workload: the FP64 oracle's whole
    registration of the same problem, single-threaded and on every host core."""
    import oracle

    oracle.build()
    P = oracle.make_params(metric=p.metric, epsilon=float(np.float32(p.epsilon)), tau=float(np.float32(p.tau)),
                           t_half=[float(np.float32(v)) for v in p.t_half], grid_cap=float(np.float32(2 * p.tau)))
    grid = oracle.hopf_grid(p.hopf_n)
    t0 = time.perf_counter()
    oracle.register(p.X, p.Y, grid, P)
    single = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.register_threads(p.X, p.Y, grid, P, threads)
    multi = time.perf_counter() - t0
    return {"value": len(grid) * len(p.X) / multi, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the whole registration ({len(grid)} rotations), distance grid built inside; "
                      f"{multi:.2f} s on {threads} threads, {single:.2f} s on one"}


def tiny(args, ws, rank, local):
    """The tiny configuration (256-point target, 128-point source, 4,608
    rotations) in full on the GPU, beside the oracle's whole registration."""
    import torch

    from paper_2502_00115_b300 import build, capi, synth

    torch.cuda.set_device(local)
    build.build()
    p = synth.tiny_problem(args.seed)
    ctx = capi.Context(local)
    t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    pr = capi.make_params(metric=p.metric, epsilon=p.epsilon, tau=p.tau, t_half=p.t_half)
    pb = ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n), pr)
    for _ in range(max(1, args.warmup)):
        ctx.register(pb)
    ts = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        ctx.register(pb)
        ts.append(time.perf_counter() - t0)
    ctx.close()
    n_rot = 72 * p.hopf_n**3
    gpu_s = statistics.median(ts)
    line = {
        "workload": "tiny", "metric": METRIC, "value": n_rot * len(p.X) / gpu_s, "unit": UNIT,
        "ms_per_registration": 1e3 * gpu_s, "rotations": n_rot, "source_points": len(p.X),
        "target_points": len(p.Y), "data": "synthetic",
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = tiny_cpu_baseline(p, os.cpu_count() or 1)
    print(json.dumps(line), flush=True)


def ours_split(args, ws, rank, local):
    """One registration per step with its rotation grid (and second pass) split
    over the ranks (strong scaling): each rank registers its contiguous ranges
    and the ranks exchange, through an all-gather, only what Algorithm 2
    reduces over all rotations (dses_register_sharded); the timed step covers
    all of it. On one rank this is the whole registration."""
    import torch

    from paper_2502_00115_b300 import build, capi, shard

    torch.cuda.set_device(local)
    import torch.distributed as dist

    if ws > 1:
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    build.build()
    name = args.workload
    p, cap, n_rot = workload(name, args.seed, args.hopf_n)  # the same problem on every rank
    steps = args.steps or (3 if name == "robot_like" else 10)
    stream = torch.cuda.Stream()
    ctx = capi.Context(local, stream.cuda_stream)
    tgt = ctx.create_target(p.Y, grid_cap=cap)
    params = gpu_params(capi, p)
    Xd = torch.from_numpy(p.X).cuda()
    pb = ctx.problem(tgt, None, capi.hopf_grid(p.hopf_n), params, src_ptr=Xd.data_ptr(), n_src=len(p.X))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    solo_gather = capi.make_allgather(lambda mine: [mine])

    def step():
        if ws > 1:
            return shard.register_sharded(ctx, pb)
        return ctx.register_sharded(pb, 0, 1, solo_gather)

    for _ in range(args.warmup):
        step()
    whole = capi.result_dict(ctx.register(pb)) if rank == 0 else None
    times = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        r = step()
        times.append(time.perf_counter() - t0)
    total_ms = max_over_ranks([1000 * sum(times)], dist if ws > 1 else None, device="cuda")[0]
    ctx.close()
    if rank != 0:
        return
    got = capi.result_dict(r)
    line = {
        "workload": f"{name}_split_rotations", "metric": METRIC,
        "value": steps * n_rot * len(p.X) / (total_ms / 1000.0), "unit": UNIT, "n_gpus": ws,
        "steps": steps, "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "strong", "data": "synthetic", "config": config_dict(name, p),
        "timing": "host wall clock per step: every rank's ranges and the exchanges (all-gathers of a few bytes)",
        "equals_whole_registration": bool(got["rot_index"] == whole["rot_index"] and got["cost"] == whole["cost"]),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        reference_arm(args, ws, rank)
        return
    if args.workload == "batched":
        batched(args, ws, rank, local)
    elif args.workload == "serving":
        serving(args, ws, rank, local)
    elif args.workload == "quality":
        quality(args, ws, rank, local)
    elif args.workload == "sweep":
        sweep(args, ws, rank, local)
    elif args.workload == "tiny":
        tiny(args, ws, rank, local)
    elif args.workload == "robot_local":
        robot_local(args, ws, rank, local)
    elif args.split == "rotations":
        ours_split(args, ws, rank, local)
    else:
        ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
