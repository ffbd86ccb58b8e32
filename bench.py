"""Benchmark of the Walk-on-Interfaces hot path on GB300.

One step = one woi_estimate over the whole workload (every point, every walk,
all M+1 steps of each walk, the u and grad u tallies, the per-point reduction
and the finalize), inputs resident in HBM.  Default workload: 3D nested spheres
(radii 1 / 0.8 / 0.5, sigma 1 / 5 / 0.2), 4096 points uniform in the ball,
1e5 walks per point, M = 6, FP32 walks with FP64 reductions.

Metric: accurate u + grad u estimates per second at the RMS standard error the
estimator reaches with 1e5 walks per point (every path computes the same
estimator, so equal walks mean equal error).  Also reported: walk-steps/s, the
roofline of the walk kernel against the FP32 peak, the end-to-end figure
through the C ABI with host buffers, and the CPU oracle timed on the host.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload 3d-nested|2d-concentric|2d-star-inclusions|6d-nested]
                    [--precision mixed|fp64]

Multi-GPU (torchrun): each rank runs the full workload on its own GPU with its
own walk range (weak scaling, no data-path collective); timing is the max over
ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic FP32 flops per walk-step (FMA = 2) of the walk on circles /
# d-spheres: 11 d + 15 (direction sampling, one transition and the Phi /
# grad Phi tally); 2D circles 30.  Derivation in the design notes.
def alg_flops_per_walk_step(dim: int, ellipsoid: bool = False) -> float:
    # ellipsoids add the two matrix-vector products A z and A (y - c) of the line / ray
    # quadratic: 4 d^2
    return 30.0 if dim == 2 else 11.0 * dim + 15.0 + (4.0 * dim * dim if ellipsoid else 0.0)


# of which the Phi / grad Phi tally at one point: 2D 14, d-spheres 5 d + 8
def alg_tally_flops(dim: int) -> float:
    return 14.0 if dim == 2 else 5.0 * dim + 8.0


# DRAM bytes per launch of the walk kernel from the ncu capture of the
# workload named as key, scaled to one full launch (None once the kernel has
# changed since the counters were taken).
TRAFFIC = {"3d-nested": 312_060}   # ncu dram__bytes_read.sum + dram__bytes_write.sum, full-size launch

WORKLOADS = {
    "3d-nested": dict(points=4096, walks=100_000, M=6),
    "2d-concentric": dict(points=64, walks=10_000, M=4),
    # the star workload shares each schedule among the 32 walks of a warp (Alg. 1's S x W
    # structure): on the star the lanes of a warp then take the same transition
    "2d-star-inclusions": dict(points=16384, walks=100_000, M=4, sched_group=32),
    "6d-nested": dict(points=1024, walks=1_000_000, M=8),
    "3d-ellipsoids": dict(points=4096, walks=100_000, M=5),
    "6d-ellipsoids": dict(points=1024, walks=1_000_000, M=8, sched_group=32),   # same SE as W_g = 1
    "3d-rocks": dict(points=4096, walks=100_000, M=5, sched_group=32),   # warp-shared schedules: the
                                                                       # lanes traverse the same mesh
    "batch": dict(points=None, walks=None, M=None),
}


def make_workload(name):
    from paper_2508_16767_gb300 import workloads as wl
    if name == "3d-nested":
        return wl.nested_3d_problem(), wl.ball_points(4096, 3, 12)
    if name == "2d-concentric":
        return wl.concentric_2d_problem(), wl.concentric_2d_points()
    if name == "2d-star-inclusions":
        p = wl.star_inclusions_problem()
        return p, wl.star_inclusions_points(p, 16384)
    if name == "6d-nested":
        return wl.nested_6d_problem(), wl.ball_points(1024, 6, 14)
    if name == "3d-rocks":
        p = wl.rocks_problem()
        return p, wl.mesh_points(p, WORKLOADS[name]["points"], seed=17)
    if name in ("3d-ellipsoids", "6d-ellipsoids"):
        d = int(name[0])
        p = wl.ellipsoids_problem(d)
        return p, wl.ellipsoid_points(p, WORKLOADS[name]["points"], seed=16)
    raise ValueError(name)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(problem, points, M, W_full, target_s=12.0, sched_group=1, single_core=False):
    """The CPU oracle as it stands on a bounded sample of the workload: all host
    threads, a subset of points and walks sized to ~target_s seconds; returns
    estimates/s at W_full walks per point (time is linear in walks)."""
    from oracle import core
    prep = core.Prepared(problem)
    n_pts, w = 16, 2048
    t0 = time.perf_counter()
    core.estimate(problem, points[:n_pts], w, seed=0, M=M, prepared=prep, sched_group=sched_group)
    t1 = time.perf_counter() - t0
    scale = max(1.0, target_s / max(t1, 1e-3))
    n_pts = int(min(len(points), max(16, n_pts * math.sqrt(scale))))
    w = int(max(2048, 2048 * scale * 16 / n_pts)) // 32 * 32
    w = min(w, W_full)                          # never more than the workload itself
    t0 = time.perf_counter()
    core.estimate(problem, points[:n_pts], w, seed=0, M=M, prepared=prep, sched_group=sched_group)
    t = time.perf_counter() - t0
    est_per_s = n_pts / (t * W_full / w)
    cores = core.threads_used()
    out = {"value": est_per_s, "cores": cores, "kind": "oracle",
           "sample": f"{n_pts} points x {w} walks (of {len(points)} x {W_full}), {t:.1f} s, "
                     f"extrapolated linearly in walks", "seconds": t,
           "walk_steps_per_s": n_pts * w * (M + 1) / t}
    if single_core and cores > 1:
        # the same oracle on one host thread, on a sample sized to ~target_s / 4
        budget = w * n_pts / cores / 4
        w1 = int(min(W_full, max(256, budget))) // 32 * 32
        n1 = int(min(len(points), max(1, round(budget / w1))))
        core.set_threads(1)
        try:
            t0 = time.perf_counter()
            core.estimate(problem, points[:n1], w1, seed=0, M=M, prepared=prep, sched_group=sched_group)
            t1 = time.perf_counter() - t0
        finally:
            core.set_threads(cores)
        out["single_core"] = {"value": n1 / (t1 * W_full / w1), "cores": 1,
                              "sample": f"{n1} points x {w1} walks, {t1:.1f} s"}
    return out


def run_reference(args, workload):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    problem, points = make_workload(workload)
    cfg = WORKLOADS[workload]
    times = []
    for s in range(args.warmup + args.steps):
        r = cpu_oracle_sample(problem, points, cfg["M"], cfg["walks"], target_s=max(2.0, 60.0 / max(args.steps, 1)),
                              sched_group=args.sched_group)
        if s >= args.warmup:
            times.append(r)
    v = float(np.mean([r["value"] for r in times]))
    line = {"impl": "reference", "metric": "accurate u+grad u estimates/s at fixed RMS error", "value": v,
            "unit": "estimates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * cfg["points"] / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "points": len(points), "walks_per_point": cfg["walks"], "M": cfg["M"],
                       "dim": problem["dim"], "precision": "fp64 (CPU oracle)", "sched_group": args.sched_group,
                       "tile_points": 0, "l2": "n/a (host cores)", "parallelism": f"host threads x{times[-1]['cores']}"},
            "cpu_baseline": {"value": v, "unit": "estimates/s", "cores": times[-1]["cores"], "kind": "oracle",
                             "sample": times[-1]["sample"]},
            "e2e": {"value": v, "unit": "estimates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--workload", default="3d-nested", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--walks-per-lane", type=int, default=0)
    ap.add_argument("--sched-group", type=int, default=0, help="walkers per schedule (default: the workload's)")
    ap.add_argument("--points", type=int, default=0, help="use only the first N points (profiling)")
    ap.add_argument("--instances", type=int, default=256, help="batch workload: number of instances")
    ap.add_argument("--tile-points", type=int, default=0, choices=[0, 32],
                    help="32: tiles of 32 points share their walks (Sec. 4.6)")
    ap.add_argument("--no-shared", action="store_true", help="skip the shared-trajectory comparison")
    ap.add_argument("--no-vr", action="store_true", help="skip the variance-reduced comparison")
    args = ap.parse_args()
    if not args.sched_group:
        args.sched_group = WORKLOADS.get(args.workload, {}).get("sched_group", 1) or 1
    if args.impl == "reference":
        return run_reference(args, args.workload)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_16767_gb300 import build
    build.build()
    from paper_2508_16767_gb300 import woi

    if args.workload == "batch":
        return run_batch_bench(args, ws, rank, local)
    cfg = WORKLOADS[args.workload]
    problem, points = make_workload(args.workload)
    if args.points:
        points = np.ascontiguousarray(points[:args.points])
    P, d, Wk, M = len(points), problem["dim"], cfg["walks"], cfg["M"]
    ell = any(srf["kind"] == "ellipsoid" for srf in problem["surfaces"])
    geom = woi.Geometry(problem)
    stream = torch.cuda.Stream()
    xd = torch.from_numpy(points).cuda()
    outs = (torch.empty(P, dtype=torch.float64, device="cuda"), torch.empty(P, d, dtype=torch.float64, device="cuda"),
            torch.empty(P, dtype=torch.float64, device="cuda"), torch.empty(P, d, dtype=torch.float64, device="cuda"))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    opt = dict(M=M, precision=args.precision, sched_group=args.sched_group, block_size=args.block,
               walks_per_lane=args.walks_per_lane, tile_points=args.tile_points)

    def step(timing):
        # each rank runs its own walk range: rank r takes walks [r W, (r + 1) W)
        if ws == 1:
            return woi.woi_estimate(geom, xd, Wk, seed=0, out=outs, stream=stream.cuda_stream, timing=timing, **opt)
        mom = woi.woi_estimate_range(geom, xd, rank * Wk, Wk, seed=0, stream=stream.cuda_stream, timing=timing, **opt)
        return mom

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[k][0].record(stream)
            step(True)
            ev[k][1].record(stream)
            kernel_ms.append(woi.woi_last_kernel_ms(geom))
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) / 1000.0
    if ws > 1:
        tt = torch.tensor([t_total], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_total = float(tt.item())
    ms_per_step = 1000.0 * t_total / args.steps
    value = ws * P / (t_total / args.steps)
    walk_steps = ws * P * Wk * (M + 1)
    wsps = walk_steps / (t_total / args.steps)

    # roofline of the walk kernel: algorithmic FP32 flops per launch / kernel time
    pk, src = peaks()
    props = torch.cuda.get_device_properties(local)
    peak_tflops = props.multi_processor_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    k_ms = float(np.mean(kernel_ms))
    if args.tile_points:
        # one walk per tile of 32 points, tallied at each of them
        n_tiles = -(-P // args.tile_points)
        flops = Wk * (M + 1) * (n_tiles * (alg_flops_per_walk_step(d, ell) - alg_tally_flops(d)) + P * alg_tally_flops(d))
    else:
        flops = P * Wk * (M + 1) * alg_flops_per_walk_step(d, ell)
    achieved = flops / (k_ms / 1000.0) / 1e12
    rms_se = float(torch.sqrt(torch.mean(outs[2] ** 2)).item()) if ws == 1 else None

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if rank == 0:
        hp = torch.from_numpy(points).pin_memory()
        ho = (torch.empty(P, dtype=torch.float64).pin_memory(), torch.empty(P, d, dtype=torch.float64).pin_memory(),
              torch.empty(P, dtype=torch.float64).pin_memory(), torch.empty(P, d, dtype=torch.float64).pin_memory())
        woi.woi_estimate(geom, hp, Wk, seed=0, out=ho, stream=stream.cuda_stream, **opt)
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 3))
        for _ in range(n_e2e):
            woi.woi_estimate(geom, hp, Wk, seed=0, out=ho, stream=stream.cuda_stream, **opt)
        te = (time.perf_counter() - t0) / n_e2e
        e2e = {"value": P / te, "unit": "estimates/s", "h2d_bytes_per_step": P * d * 8,
               "d2h_bytes_per_step": P * (2 + 2 * d) * 8}

    # the plain FP64 one-launch-per-point GPU path on a sample of the points
    # (same estimator, same walks per point, so the same RMS error), for comparison
    fp64 = None
    if rank == 0 and ws == 1 and args.precision == "mixed" and not args.no_fp64_baseline:
        n_s = min(P, 64)
        xs = xd[:n_s].contiguous()
        woi.woi_estimate(geom, xs, Wk, seed=0, stream=stream.cuda_stream, M=M, precision="fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        woi.woi_estimate(geom, xs, Wk, seed=0, stream=stream.cuda_stream, M=M, precision="fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1000.0
        fp64 = {"value": n_s / t64, "unit": "estimates/s", "points_sampled": n_s,
                "speedup_of_mixed": value / (n_s / t64)}

    # the same workload with shared trajectories (Sec. 4.6: tiles of 32 points share
    # their walks), timed like the main steps, for comparison
    shared = None
    if rank == 0 and ws == 1 and args.precision == "mixed" and not args.tile_points and not args.no_shared:
        so = dict(opt, tile_points=32)
        so.pop("walks_per_lane", None)
        so.pop("block_size", None)
        for _ in range(args.warmup):
            woi.woi_estimate(geom, xd, Wk, seed=0, out=outs, stream=stream.cuda_stream, **so)
        sms = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            woi.woi_estimate(geom, xd, Wk, seed=0, out=outs, stream=stream.cuda_stream, timing=True, **so)
            e1.record(stream)
            torch.cuda.synchronize()
            sms.append((e0.elapsed_time(e1), woi.woi_last_kernel_ms(geom)))
        t_s = float(np.mean([a for a, _ in sms])) / 1000.0
        k_s = float(np.mean([b for _, b in sms]))
        n_tiles = -(-P // 32)
        fl = Wk * (M + 1) * (n_tiles * (alg_flops_per_walk_step(d, ell) - alg_tally_flops(d)) + P * alg_tally_flops(d))
        shared = {"value": P / t_s, "unit": "estimates/s", "ms_per_step": 1000.0 * t_s, "tile_points": 32,
                  "walk_steps_per_s": P * Wk * (M + 1) / t_s, "kernel_ms": k_s,
                  "rms_se_u": float(torch.sqrt(torch.mean(outs[2] ** 2)).item()),
                  "roofline_frac": fl / (k_s / 1000.0) / 1e12 / peak_tflops, "speedup_of_per_point": (P / t_s) / value}

    # the variance-reduced variant (Alg. 3; 2D Fourier data, or hemisphere parts of data linear
    # in the unit vector in d >= 3): two chains per walk from the beta >= 0 and beta < 0 parts;
    # at the plain path's RMS error it needs (se_vr / se_plain)^2 of the walks
    vr = None
    vo = dict(opt, variant="vr")
    vr_ok = rank == 0 and ws == 1 and args.precision == "mixed" and not args.tile_points and not args.no_vr
    if vr_ok:
        try:
            woi.woi_estimate(geom, xd, Wk, seed=0, out=outs, stream=stream.cuda_stream, **vo)
        except woi.WoiError as e:
            if e.status != 4:                     # WOI_E_UNSUPPORTED
                raise
            vr_ok = False                          # no closed-form parts for this data
    if vr_ok:
        for _ in range(args.warmup):
            woi.woi_estimate(geom, xd, Wk, seed=0, out=outs, stream=stream.cuda_stream, **vo)
        vms = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            woi.woi_estimate(geom, xd, Wk, seed=0, out=outs, stream=stream.cuda_stream, **vo)
            e1.record(stream)
            torch.cuda.synchronize()
            vms.append(e0.elapsed_time(e1))
        t_v = float(np.mean(vms)) / 1000.0
        se_v = float(torch.sqrt(torch.mean(outs[2] ** 2)).item())
        ratio = (se_v / rms_se) ** 2 if rms_se else None
        vr = {"value": P / t_v, "unit": "estimates/s", "ms_per_step": 1000.0 * t_v, "rms_se_u": se_v,
              "walk_steps_per_s": 2 * P * Wk * (M + 1) / t_v,
              "value_at_plain_rms_error": (P / (t_v * ratio)) if ratio else None,
              "note": "two chains per walk; value_at_plain_rms_error scales the walks by (se_vr / se_plain)^2"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(problem, points, M, Wk, sched_group=args.sched_group, single_core=True)
        cpu = {k: cpu[k] for k in ("value", "cores", "kind", "sample", "single_core") if k in cpu} | {"unit": "estimates/s"}

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": "accurate u+grad u estimates/s at fixed RMS error", "value": value, "unit": "estimates/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "points": P, "walks_per_point": Wk, "M": M, "dim": d,
                       "precision": args.precision, "sched_group": args.sched_group,
                       "tile_points": args.tile_points,
                       "l2": "flushed between steps (512 MiB write outside the step events)",
                       "parallelism": f"replicas x{ws}, disjoint walk ranges"},
            "walk_steps_per_s": wsps, "rms_se_u": rms_se,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / peak_tflops, "traffic": TRAFFIC.get(args.workload),
                         "peak_source": f"FP32: SMs x 128 lanes x 2 x sm_max_mhz ({src})",
                         "kernel_ms": k_ms, "alg_flops_per_walk_step": alg_flops_per_walk_step(d, ell)},
            "cpu_baseline": cpu, "fp64_plain_gpu_path": fp64, "shared_trajectories": shared,
            "variance_reduced": vr, "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": args.steps * (2 if args.precision == "mixed" else P + 1),
        }
        print(json.dumps(line))
    geom.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_batch_bench(args, ws, rank, local):
    """256 heterogeneous 2D / 3D manufactured-solution instances in one batched
    call (one persistent launch per dimension, replayed as a CUDA graph)."""
    import torch
    from paper_2508_16767_gb300 import build, woi
    from paper_2508_16767_gb300 import workloads as wl
    build.build()
    insts = wl.batch_instances(n_inst=args.instances)
    geoms = [woi.Geometry(it["problem"]) for it in insts]
    args_dev = [(g, torch.from_numpy(it["points"]).cuda(), it["n_walks"]) for g, it in zip(geoms, insts)]
    P = sum(len(it["points"]) for it in insts)
    walk_steps = sum(len(it["points"]) * it["n_walks"] * (it["problem"]["M"] + 1) for it in insts)
    stream = torch.cuda.Stream()
    opt = dict(precision=args.precision, sched_group=args.sched_group, block_size=args.block,
               walks_per_lane=args.walks_per_lane)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    for _ in range(args.warmup):
        woi.woi_estimate_batch(args_dev, seed=0, stream=stream.cuda_stream, **opt)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[k][0].record(stream)
            woi.woi_estimate_batch(args_dev, seed=0, stream=stream.cuda_stream, timing=True, **opt)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) / 1000.0 / args.steps
    k_ms = woi.woi_last_kernel_ms(geoms[0])
    # end to end with host arrays
    args_host = [(g, it["points"], it["n_walks"]) for g, it in zip(geoms, insts)]
    t0 = time.perf_counter()
    woi.woi_estimate_batch(args_host, seed=0, **opt)
    te = time.perf_counter() - t0
    # per-instance plain FP64 launches (one per point) on a sample of instances: the same
    # estimator with the same walks, so the same RMS error
    fp64 = None
    if not args.no_fp64_baseline and args.precision == "mixed":
        rs = np.random.default_rng(1)
        pick = rs.choice(len(insts), size=min(8, len(insts)), replace=False)
        n_s = 0
        t64 = 0.0
        for k in pick:
            g, xd, Wk = args_dev[k]
            xs = xd[:64].contiguous()
            woi.woi_estimate(g, xs, Wk, seed=0, stream=stream.cuda_stream, M=insts[k]["problem"]["M"], precision="fp64")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            woi.woi_estimate(g, xs, Wk, seed=0, stream=stream.cuda_stream, M=insts[k]["problem"]["M"], precision="fp64")
            e1.record(stream)
            torch.cuda.synchronize()
            t64 += e0.elapsed_time(e1) / 1000.0
            n_s += len(xs)
        # walk-steps per second of the FP64 path, turned into this batch's estimates/s
        ws64 = sum(min(64, len(insts[k]["points"])) * insts[k]["n_walks"] * (insts[k]["problem"]["M"] + 1)
                   for k in pick) / t64
        fp64 = {"value": P / (walk_steps / ws64), "unit": "estimates/s", "walk_steps_per_s": ws64,
                "instances_sampled": int(len(pick)), "points_sampled": int(n_s),
                "speedup_of_mixed": (P / t) / (P / (walk_steps / ws64))}
    d_avg = float(np.mean([it["problem"]["dim"] for it in insts]))
    flops = sum(len(it["points"]) * it["n_walks"] * (it["problem"]["M"] + 1) * alg_flops_per_walk_step(it["problem"]["dim"])
                for it in insts)
    pk, src = peaks()
    props = torch.cuda.get_device_properties(local)
    peak = props.multi_processor_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = flops / (k_ms / 1000.0) / 1e12
    line = {"metric": "accurate u+grad u estimates/s at fixed RMS error", "value": P / t, "unit": "estimates/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": "batch", "instances": len(insts), "points": P, "walk_steps": walk_steps,
                       "precision": args.precision,
                       "l2": "flushed between steps (512 MiB write outside the step events)"},
            "walk_steps_per_s": walk_steps / t,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, "kernel_ms": k_ms, "peak_source": f"FP32 ({src})"},
            "e2e": {"value": P / te, "unit": "estimates/s",
                    "h2d_bytes_per_step": int(sum(it["points"].size * 8 for it in insts)),
                    "d2h_bytes_per_step": int(sum(len(it["points"]) * (2 + 2 * it["problem"]["dim"]) * 8 for it in insts))},
            "fp64_plain_gpu_path": fp64, "clocks": clk.summary(), "gpu_launches": args.steps * 4}
    if rank == 0:
        print(json.dumps(line))
    for g in geoms:
        g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
