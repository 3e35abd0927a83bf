#!/usr/bin/env python3
"""DSES registration benchmark on B300.

One step = one full registration (Algorithm 2: every rotation of the grid
votes, counts inliers, is scored, and the argmin is returned) of the
ModelNet-shaped synthetic problem: 1,024-point target, 717-point source (70%
half-space crop), 294,912-rotation Hopf grid (N_side 16, ~3.75 degrees),
truncated-L2 metric read from the target's 128^3 FP32 distance grid.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
# DRAM bytes (read + write) of one vote_kernel launch, from an ncu capture of
# the same kernel on this problem at N_side 4: a launch reads its inputs (KB)
# once, so the figure does not grow with the rotations and is used unscaled.
VOTE_DRAM_BYTES = 261376


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--hopf-n", type=int, default=16, help="grid N_side (16 = the benchmark; smaller for profiling)")
    ap.add_argument("--points-per-thread", type=int, default=0, help="vote launch shape (0: library default)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["modelnet_like", "batched", "serving", "robot_like", "robot_local", "quality", "sweep", "tiny"],
                    default="modelnet_like",
                    help="modelnet_like: the benchmark line; batched / serving: the other configurations")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--quality-count", type=int, default=64, help="quality: number of problems")
    ap.add_argument("--rotated-frame", action="store_true", help="quality: both clouds in a rotated frame")
    ap.add_argument("--refine-iterations", type=int, default=3, help="quality: translation refinement steps")
    ap.add_argument("--refine-top-k", type=int, default=16, help="quality: Euler-box second pass around the best k")
    ap.add_argument("--refine-K", type=int, default=3, help="quality: Euler-box half-size of the second pass")
    ap.add_argument("--refine-delta-deg", type=float, default=1.0, help="quality: Euler-box step (degrees)")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: arrival window (s)")
    ap.add_argument("--split", choices=["problems", "rotations"], default="problems",
                    help="modelnet_like under torchrun: one problem per rank (weak scaling) or one problem's "
                         "rotations sharded over the ranks (strong scaling)")
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
        self.path = tempfile.mktemp(prefix="clocks", suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
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


def workload(seed, hopf_n=16):
    from paper_2502_00115_b300 import synth

    return synth.modelnet_like_problem(seed, hopf_n=hopf_n)


def config_dict(p):
    R = 72 * p.hopf_n**3
    return {"workload": "modelnet_like_single_problem", "target_points": int(len(p.Y)),
            "source_points": int(len(p.X)), "rotations": R, "rotation_grid": f"hopf N_side={p.hopf_n}",
            "metric": p.metric, "tau": p.tau, "epsilon": p.epsilon, "delta_t": p.delta_t,
            "translation_box": f"+-{p.t_half[0]} per axis", "distance_grid": "128^3 fp32",
            "l2": "flushed between steps (512 MB write)"}


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
    """Time the FP64 oracle (Algorithm 2 on a rotation subset, prebuilt field)."""
    import oracle

    oracle.build()
    R_all_n = p.hopf_n
    P = oracle.params_from_problem(p, nn_mode="grid", grid_cap=2 * p.tau)
    field = oracle.Field(p.Y, P.grid_res, P.grid_cap)
    n_all = 72 * R_all_n**3

    def run(count, offset=0):
        stride = max(1, n_all // count)
        idx = (np.arange(count) * stride + offset) % n_all
        Rs = np.stack([oracle.hopf_rotation(R_all_n, int(i)) for i in idx])
        t0 = time.perf_counter()
        oracle.register_field_threads(p.X, p.Y, Rs, P, field, threads)
        return time.perf_counter() - t0

    probe = 4 * threads
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
            "sample": f"{count} of {72 * p.hopf_n**3} rotations (even stride) of the same problem, FP64 "
                      f"Algorithm 2 fanned over {threads} threads, distance field prebuilt (not timed), {dt:.1f} s"}


def reference_arm(args, ws, rank):
    if rank != 0:
        return
    p = workload(args.seed, args.hopf_n)
    threads = os.cpu_count() or 1
    # each step: a bounded rotation sample sized to ~4 s so K + W steps stay within minutes
    run, count, per_rot, field = oracle_sample(p, 4.0, threads)
    for w in range(args.warmup):
        run(count, offset=w + 1)
    times = [run(count, offset=100 + k) for k in range(args.steps)]
    field.close()
    tot = sum(times)
    value = args.steps * count * len(p.X) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{count} rotations per step (even stride, shifted per step) of "
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
    p = workload(args.seed + rank, args.hopf_n)
    n_rot = 72 * p.hopf_n**3
    units = n_rot * len(p.X)
    stream = torch.cuda.Stream()
    ctx = capi.Context(local, stream.cuda_stream)
    tgt = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    params = capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau,
                              huber_h=p.huber_h, t_half=p.t_half, nn_mode="grid")
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

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        ctx.register(pb_dev)
        ctx.register(pb_host)

    # device-resident inputs, CUDA events on the library's stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    pass_ns = []
    count_ns = []
    results = []
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = ctx.get_option("kernel_launches")
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[k][0].record(stream)
        r = ctx.register(pb_dev)
        ev[k][1].record(stream)
        results.append(capi.result_dict(r))
        pass_ns.append(ctx.get_option("last_pass_ns"))
        count_ns.append(ctx.get_option("last_count_ns"))
        votes = ctx.get_option("last_votes_total")
    torch.cuda.synchronize()
    launches = ctx.get_option("kernel_launches") - launches0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)

    # end to end through the public API: pinned host source in, result out
    e2e_s = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        ctx.register(pb_host)
        e2e_s.append(time.perf_counter() - t0)
    clk = clocks.stop()

    total_ms, e2e_tot = max_over_ranks([total_ms, sum(e2e_s)], dist, device="cuda")
    ctx.close()
    if rank != 0:
        return
    try:
        from paper_2502_00115_b300 import peaks

        pk = peaks.run(local)
    except Exception as e:  # the microbenchmark is auxiliary evidence
        pk = {"error": str(e)}
    value = job_throughput(ws, args.steps, units, total_ms)
    pass_s = statistics.mean(pass_ns) / 1e9
    M = len(p.Y)
    ops = n_rot * len(p.X) * (M * OPS_PER_PAIR + OPS_PER_ROT_SRC)
    achieved = ops / pass_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": config_dict(p),
        "registrations_per_s": ws * args.steps / (total_ms / 1000),
        "latency_ms": {"p50": 1000 * float(np.percentile(e2e_s, 50)), "p99": 1000 * float(np.percentile(e2e_s, 99))},
        "roofline": {"bound": "alu", "kernel": "vote_kernel", "achieved": achieved / 1e12,
                     "peak": ALU_PEAK_OPS / 1e12, "unit": "Tops/s", "frac": achieved / ALU_PEAK_OPS,
                     "traffic": VOTE_DRAM_BYTES, "traffic_unit": "bytes per launch (ncu, N_side 4 capture)",
                     "kernel_ms": pass_s * 1000,
                     "count_kernel_ms": statistics.mean(count_ns) / 1e6,
                     "peak_source": "recipe unit counts: 148 SMs x 128 lanes x 2032 MHz",
                     "frac_of_measured_ffma": (achieved / pk["ffma_per_s"]) if "ffma_per_s" in pk else None,
                     "ops_per_launch": ops},
        "smem_atomic_roofline": {
            "kernel": "vote_kernel", "achieved": votes / pass_s,
            "peak": pk.get("smem_atomic_random_per_s"), "unit": "increments/s",
            "frac": (votes / pass_s / pk["smem_atomic_random_per_s"]) if "smem_atomic_random_per_s" in pk else None,
            "increments_per_launch": int(votes),
            # the kernel issues one atomic per pair (pairs outside the box add to a sink word)
            "issued_per_s": n_rot * len(p.X) * M / pass_s,
            "issued_frac": (n_rot * len(p.X) * M / pass_s / pk["smem_atomic_random_per_s"])
            if "smem_atomic_random_per_s" in pk else None,
            "peak_source": "measured in this run: red.shared.add on random bins of a 46,575-word histogram"},
        # the fused inlier-count / score kernel: per (rotation, source point) the
        # trilinear distance-grid lookup reads its 8 corners as two 16-byte
        # corner blocks from the L2-resident grid; bound by random L2 gathers
        "score_roofline": {
            "kernel": "count_kernel", "bound": "l2_gather",
            "achieved": n_rot * len(p.X) * 2 / (statistics.mean(count_ns) / 1e9),
            "peak": pk.get("l2_gather_16B_per_s"), "unit": "16-byte gathers/s",
            "frac": (n_rot * len(p.X) * 2 / (statistics.mean(count_ns) / 1e9) / pk["l2_gather_16B_per_s"])
            if "l2_gather_16B_per_s" in pk else None,
            "peak_source": "measured in this run: random aligned 16-byte loads from a 32 MB table"},
        "peaks_measured": pk,
        "e2e": {"value": job_throughput(ws, args.steps, units, 1000 * e2e_tot), "unit": UNIT,
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
    """64 uneven problems in one persistent launch vs one launch per problem."""
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
    for _ in range(max(1, args.warmup)):
        ctx.register_batch(pbs)
    t_batch = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rb = ctx.register_batch(pbs)
        t_batch.append(time.perf_counter() - t0)
    t_seq = []
    for _ in range(max(1, args.steps // 2)):
        t0 = time.perf_counter()
        rs = [ctx.register(pb) for pb in pbs]
        t_seq.append(time.perf_counter() - t0)
    same = all(capi.result_dict(a)["rot_index"] == capi.result_dict(b)["rot_index"] for a, b in zip(rb, rs))
    ctx.close()
    tb, tsq = statistics.mean(t_batch), statistics.mean(t_seq)
    print(json.dumps({
        "workload": "batched", "metric": METRIC, "value": units / tb, "unit": UNIT, "problems": len(probs),
        "registrations_per_s": len(probs) / tb, "sequential": {"value": units / tsq,
                                                                "registrations_per_s": len(probs) / tsq},
        "batch_over_sequential": tsq / tb, "pair_votes_per_s": pairs / tb, "s_per_batch": tb,
        "steps": args.steps, "results_equal_sequential": same,
        "config": {"targets": f"{min(len(p.Y) for p in probs)}..{max(len(p.Y) for p in probs)} pts",
                   "sources": f"{min(len(p.X) for p in probs)}..{max(len(p.X) for p in probs)} pts",
                   "rotations": f"{min(72 * p.hopf_n**3 for p in probs)}..{max(72 * p.hopf_n**3 for p in probs)}"},
    }), flush=True)


def serving(args, ws, rank, local):
    """Poisson arrivals over resident targets through dses_submit / dses_poll."""
    import torch

    from paper_2502_00115_b300 import build, capi, synth

    torch.cuda.set_device(local)
    build.build()
    wl = synth.serving_workload(args.seed, rate=args.rate, duration=args.duration)
    ctx = capi.Context(local)
    tmap = {}
    for i, Y in enumerate(wl.targets):
        tmap[i] = ctx.create_target(Y, grid_cap=0.1)
    reqs = []
    first_of_target = {}
    for (t_arr, ti, p) in wl.requests:
        pb = ctx.problem(tmap[ti], p.X, capi.hopf_grid(p.hopf_n),
                         capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau,
                                          t_half=p.t_half))
        reqs.append((t_arr, pb, 72 * p.hopf_n**3 * len(p.X)))
        first_of_target.setdefault(ti, pb)
    # warm the path outside both measurements: the grid, and every target's
    # per-epsilon cell list and per-delta bounds (built on a target's first use)
    for pb in first_of_target.values():
        ctx.register(pb)
    pending = {}
    lat = []
    units = 0
    t0 = time.perf_counter()
    nxt = 0
    while nxt < len(reqs) or pending:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt][0] <= now:
            pending[ctx.submit(reqs[nxt][1])] = (t0 + reqs[nxt][0], reqs[nxt][2])
            nxt += 1
        for tk in list(pending):
            st, r = ctx.poll(tk)
            if st != capi.DSES_NOT_READY:
                t_sub, u = pending.pop(tk)
                lat.append(time.perf_counter() - t_sub)
                units += u
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    # the same requests as sequential single-problem launches (blocking
    # dses_register one after another): measured service times, and the
    # latencies of a first-come first-served queue with the same arrivals
    svc = []
    for (_, pb, _) in reqs:
        t1 = time.perf_counter()
        ctx.register(pb)
        svc.append(time.perf_counter() - t1)
    ctx.close()
    finish, seq_lat = 0.0, []
    for (t_arr, _, _), sv in zip(reqs, svc):
        finish = max(finish, t_arr) + sv
        seq_lat.append(finish - t_arr)
    print(json.dumps({
        "workload": "serving", "metric": METRIC, "value": units / wall, "unit": UNIT,
        "offered_rate": args.rate, "requests": len(reqs), "registrations_per_s": len(reqs) / wall,
        "latency_ms": {"p50": 1000 * float(np.percentile(lat, 50)), "p99": 1000 * float(np.percentile(lat, 99)),
                       "max": 1000 * max(lat)},
        "wall_s": wall, "arrival_window_s": args.duration,
        "sequential": {"registrations_per_s": len(reqs) / max(finish, sum(svc)),
                       "service_ms_mean": 1000 * statistics.mean(svc),
                       "latency_ms": {"p50": 1000 * float(np.percentile(seq_lat, 50)),
                                      "p99": 1000 * float(np.percentile(seq_lat, 99))}},
    }), flush=True)


def robot(args, ws, rank, local):
    """The robot-pose-like problem: 2.36M-rotation grid plus Euler boxes around the best 32."""
    import torch

    from paper_2502_00115_b300 import build, capi, synth

    torch.cuda.set_device(local)
    build.build()
    p = synth.robot_like_problem(args.seed, hopf_n=args.hopf_n if args.hopf_n != 16 else 32)
    ctx = capi.Context(local)
    ctx.set_option("record_timing", 1)
    if args.points_per_thread:
        ctx.set_option("points_per_thread", args.points_per_thread)
    t = ctx.create_target(p.Y, grid_cap=p.grid_cap)
    pb = ctx.problem(t, p.X, capi.hopf_grid(p.hopf_n),
                     capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau,
                                      huber_h=p.huber_h, t_half=p.t_half, refine_top_k=p.refine_top_k,
                                      refine_K=p.refine_K, refine_delta_r=p.refine_delta_r))
    for _ in range(max(1, args.warmup)):
        ctx.register(pb)
    ts, vote_ms, count_ms = [], [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = ctx.register(pb)
        ts.append(time.perf_counter() - t0)
        vote_ms.append(ctx.get_option("last_pass_ns") / 1e6)
        count_ms.append(ctx.get_option("last_count_ns") / 1e6)
    ctx.close()
    res = capi.result_dict(r)
    ang = float(np.degrees(np.arccos(np.clip((np.trace(res["R"].astype(np.float64).T @ p.R_true) - 1) / 2, -1, 1))))
    n_rot = p.n_rotations
    tm = statistics.mean(ts)
    print(json.dumps({
        "workload": "robot_like", "metric": METRIC, "value": n_rot * len(p.X) / tm, "unit": UNIT,
        "s_per_registration": tm, "vote_ms": statistics.mean(vote_ms), "count_ms": statistics.mean(count_ms),
        "pair_votes_per_s": n_rot * len(p.X) * len(p.Y) / tm, "rotations": n_rot, "source_points": len(p.X),
        "target_points": len(p.Y), "rotation_error_deg": ang,
        "translation_error_m": float(np.linalg.norm(res["t"] - p.t_true)), "result": {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in res.items()},
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
        p = synth.modelnet_like_problem(args.seed + k, hopf_n=args.hopf_n, max_euler_deg=45.0,
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
        "rotated_frame": bool(args.rotated_frame), "rotation_grid": f"hopf N_side={args.hopf_n}",
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
    """One ModelNet-shaped registration per step with its rotation grid split
    over the ranks (strong scaling): each rank registers its contiguous range,
    the ranks all-gather their result structs and combine them; the timed
    step covers both. On one rank this is the whole registration."""
    import torch

    from paper_2502_00115_b300 import build, capi, shard

    torch.cuda.set_device(local)
    import torch.distributed as dist

    if ws > 1:
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    build.build()
    p = workload(args.seed, args.hopf_n)  # the same problem on every rank
    n_rot = 72 * p.hopf_n**3
    stream = torch.cuda.Stream()
    ctx = capi.Context(local, stream.cuda_stream)
    tgt = ctx.create_target(p.Y, grid_cap=2 * p.tau)
    params = capi.make_params(metric=p.metric, epsilon=p.epsilon, delta_t=p.delta_t, tau=p.tau,
                              huber_h=p.huber_h, t_half=p.t_half, nn_mode="grid")
    Xd = torch.from_numpy(p.X).cuda()
    pb = ctx.problem(tgt, None, capi.hopf_grid(p.hopf_n), params, src_ptr=Xd.data_ptr(), n_src=len(p.X))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def step():
        if ws > 1:
            return shard.register_sharded(ctx, pb)
        return capi.combine_results([ctx.register_shard(pb, 0, 1)])

    for _ in range(args.warmup):
        step()
    whole = capi.result_dict(ctx.register(pb)) if rank == 0 else None
    times = []
    for _ in range(args.steps):
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
        "workload": "modelnet_like_split_rotations", "metric": METRIC,
        "value": args.steps * n_rot * len(p.X) / (total_ms / 1000.0), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "data": "synthetic", "config": config_dict(p),
        "timing": "host wall clock per step: every rank's range, the all-gather of result structs and the combine",
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
    elif args.workload == "robot_like":
        robot(args, ws, rank, local)
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
