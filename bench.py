"""Benchmark of the Walk-on-Interfaces hot path on GB300.

Default workload (the headline line): a batch of 256 independent 2D / 3D problem
instances (unit disk / ball with 1-64 circular / spherical inclusions, sigma
log-uniform on [0.05, 20], manufactured harmonic data, 16-4096 points and 1e4-1e5
walks per point, M = 4 in 2D and 6 in 3D; about 1.9e5 points and 4e10
walk-steps).  One step = one woi_estimate_batch call over the whole batch: one
persistent FP32 walk kernel per dimension, regenerating work from device queues,
and the batched finalize, replayed as a captured CUDA graph; inputs resident in
HBM.  The same walks are also run by the plain FP64 path (one launch per
evaluation point, the baseline to beat at equal RMS error: the same estimator
over the same walks), through the C ABI with pinned host buffers (e2e), and by
the CPU oracle on a bounded sample of the batch.

Metric: accurate u + grad u estimates per second at the RMS error the estimator
reaches with each instance's walks (every path computes the same estimator over
the same walks, so equal walks mean equal error; the line states that error: the
standard errors per point and the gradient's RMS error against the manufactured
closed form).  Also reported: walk-steps/s, the roofline of the walk kernel
against the FP32 peak, and the other workloads (3D nested spheres, the 2D star
with 32 inclusions plain and variance-reduced, 6D nested spheres, 2D concentric
circles) under "extra_workloads".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload batch|3d-nested|2d-concentric|2d-star-inclusions|6d-nested|...]

Multi-GPU (torchrun): each rank runs the whole workload on its own walk range
(weak scaling); the per-point raw moments are all-reduced over NCCL and
finalized by the library inside the timed step; timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


# Algorithmic FP32 flops per walk-step (FMA = 2) of the walk on circles / d-spheres:
# d-spheres 11 d + 15 -- direction sampling about 6 d (d / 2 Box-Muller pairs or one
# angle and a height), one transition (the chord, ray and uniform candidates share
# the direction: 2 d dot-product terms plus the selected update), and the Phi / grad Phi
# tally 5 d + 8 (difference, squared distance, the inverse power, d gradient terms);
# 2D circles 30 (8 sampling + 14 tally + 8 transition and weights).
def alg_flops_per_walk_step(dim: int, ellipsoid: bool = False) -> float:
    # ellipsoids add the two matrix-vector products A z and A (y - c) of the line / ray
    # quadratic: 4 d^2
    return 30.0 if dim == 2 else 11.0 * dim + 15.0 + (4.0 * dim * dim if ellipsoid else 0.0)


# of which the Phi / grad Phi tally at one point: 2D 14, d-spheres 5 d + 8
def alg_tally_flops(dim: int) -> float:
    return 14.0 if dim == 2 else 5.0 * dim + 8.0


# DRAM bytes per launch of the walk kernel(s) from an ncu capture of the named workload
# (dram__bytes_read.sum + dram__bytes_write.sum), scaled to one full launch; None once
# the kernel has changed since the counters were taken.
TRAFFIC = {"3d-nested": 625_152, "batch": 284_768_768}   # batch: both group launches of one step

# Warp instructions (all pipes, and the XU pipe: transcendentals, conversions) per walk-step of
# the walk kernels, from an ncu capture of the same kernels (sm__inst_executed.sum and
# sm__inst_executed_pipe_xu.sum of a launch divided by the walk-steps it ran), and the XU pipe's
# peak in warp instructions per SM per cycle (from the same capture:
# sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active).  With the live walk-step rate they
# give the fraction of the issue slots (4 warp instructions per SM per cycle) and of the XU pipe
# the kernel uses; None until measured for the current kernel.
INST_PER_STEP = {"batch": {2: {"inst": 7.539, "xu": 0.2010}, 3: {"inst": 9.226, "xu": 0.2062}}}
XU_PEAK_PER_SM_CYCLE = 0.99

WORKLOADS = {
    "batch": dict(points=None, walks=None, M=None),
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
}
EXTRAS = ["3d-nested", "2d-star-inclusions", "6d-nested", "2d-concentric"]
METRIC = "accurate u+grad u estimates/s at fixed RMS error"


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


def fp32_peak_tflops(local):
    """FP32 peak: SMs x 128 lanes x 2 flops (FMA) x the measured maximum SM clock."""
    import torch
    pk, src = peaks()
    props = torch.cuda.get_device_properties(local)
    return props.multi_processor_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12, \
        f"FP32: SMs x 128 lanes x 2 x sm_max_mhz ({src})"


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


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


def accuracy(u, grad, se_u, se_grad, n_walks):
    """How the standard error is spread over the points: median and 90th percentile of the
    relative SE of u (se_u / |u|) and of grad u (max over components of se / |grad u|), the
    RMS SE, and the walks per point a 1 % median relative error of u would need (SE ~ W^-1/2).
    Arrays of one workload, or lists of per-instance arrays (instances of several dimensions)."""
    if isinstance(u, (list, tuple)):
        parts = [(np.asarray(a), np.asarray(b), np.asarray(c), np.asarray(d)) for a, b, c, d in zip(u, grad, se_u, se_grad)]
        u = np.concatenate([p[0] for p in parts])
        se_u = np.concatenate([p[2] for p in parts])
        gn = np.concatenate([np.linalg.norm(p[1], axis=1) for p in parts])
        sg = np.concatenate([np.max(p[3], axis=1) for p in parts])
    else:
        u, se_u = np.asarray(u, dtype=np.float64), np.asarray(se_u, dtype=np.float64)
        gn = np.linalg.norm(np.asarray(grad, dtype=np.float64), axis=1)
        sg = np.max(np.asarray(se_grad, dtype=np.float64), axis=1)
    n_walks = np.broadcast_to(np.asarray(n_walks, dtype=np.float64), u.shape)
    ru = se_u / np.maximum(np.abs(u), 1e-300)
    rg = sg / np.maximum(gn, 1e-300)
    w1 = n_walks * (ru / 0.01) ** 2
    wg = n_walks * (rg / 0.01) ** 2
    return {"rms_se_u": float(np.sqrt(np.mean(se_u ** 2))), "rms_u": float(np.sqrt(np.mean(u ** 2))),
            "median_rel_se_u": float(np.median(ru)), "p90_rel_se_u": float(np.quantile(ru, 0.9)),
            "median_rel_se_grad": float(np.median(rg)), "p90_rel_se_grad": float(np.quantile(rg, 0.9)),
            "walks_for_1pct_median_rel_err_u": float(np.median(w1)),
            "walks_for_1pct_median_rel_err_grad": float(np.median(wg))}


# ---------------------------------------------------------------------------
# CPU oracle samples (reported baseline; the reference arm)
# ---------------------------------------------------------------------------

def cpu_oracle_sample(problem, points, M, W_full, target_s=12.0, sched_group=1, single_core=False):
    """The CPU oracle as it stands on a bounded sample of one workload: all host threads,
    a subset of points and walks sized to ~target_s seconds; returns estimates/s at W_full
    walks per point (the time is linear in walks)."""
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
    cores = core.threads_used()
    out = {"value": n_pts / (t * W_full / w), "unit": "estimates/s", "cores": cores, "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": f"{n_pts} points x {w} walks (of {len(points)} x {W_full}), {t:.1f} s, "
                     f"extrapolated linearly in walks"}
    if single_core and cores > 1:
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
        out["single_core"] = {"value": n1 / (t1 * W_full / w1), "unit": "estimates/s", "cores": 1,
                              "sample": f"{n1} points x {w1} walks, {t1:.1f} s"}
    return out


def cpu_oracle_batch_sample(insts, target_s=12.0, single_core=False):
    """The CPU oracle on a bounded sample of the batch: every 16th instance, a few points
    each, with its own walks scaled down; the time per walk-step of the sample, times the
    batch's walk-steps, gives the oracle's estimates/s on the whole batch."""
    from oracle import core
    pick = list(range(0, len(insts), 16))
    P_all = sum(len(it["points"]) for it in insts)
    steps_all = sum(len(it["points"]) * it["n_walks"] * (it["problem"]["M"] + 1) for it in insts)

    def run(frac, n_pts):
        t, steps = 0.0, 0
        for k in pick:
            it = insts[k]
            prob, M = it["problem"], it["problem"]["M"]
            w = max(32, int(it["n_walks"] * frac) // 32 * 32)
            n = min(n_pts, len(it["points"]))
            prep = core.Prepared(prob)
            t0 = time.perf_counter()
            core.estimate(prob, it["points"][:n], w, seed=0, M=M, prepared=prep, instance=k)
            t += time.perf_counter() - t0
            steps += n * w * (M + 1)
        return t, steps

    t, steps = run(0.01, 4)
    scale = max(1.0, target_s / max(t, 1e-3))
    frac = min(1.0, 0.01 * scale)                      # first more walks, then more points
    n_pts = int(min(4096, max(4, 4 * scale * 0.01 / frac)))
    t, steps = run(frac, n_pts)
    cores = core.threads_used()
    out = {"value": P_all / (t * steps_all / steps), "unit": "estimates/s", "cores": cores, "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": f"{len(pick)} of {len(insts)} instances x up to {n_pts} points x {frac:.3g} of their walks, "
                     f"{t:.1f} s; time per walk-step scaled to the batch's {steps_all:.3e} walk-steps"}
    if single_core and cores > 1:
        core.set_threads(1)
        try:
            t1, s1 = run(frac / max(4.0, cores / 4.0), 4)
        finally:
            core.set_threads(cores)
        out["single_core"] = {"value": P_all / (t1 * steps_all / s1), "unit": "estimates/s", "cores": 1,
                              "sample": f"{len(pick)} instances x 4 points x {frac / max(4.0, cores / 4.0):.3g} of "
                                        f"their walks, {t1:.1f} s"}
    return out


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores, on a bounded
    sample of the same workload, in the same metric."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2508_16767_gb300 import workloads as wl
    target = max(2.0, 60.0 / max(args.steps + args.warmup, 1))
    times = []
    if args.workload == "batch":
        insts = wl.batch_instances(n_inst=args.instances)
        P = sum(len(it["points"]) for it in insts)
        cfg = {"workload": "batch", "instances": len(insts), "points": P,
               "walk_steps": int(sum(len(it["points"]) * it["n_walks"] * (it["problem"]["M"] + 1) for it in insts))}
        for s in range(args.warmup + args.steps):
            r = cpu_oracle_batch_sample(insts, target_s=target)
            if s >= args.warmup:
                times.append(r)
    else:
        problem, points = make_workload(args.workload)
        w = WORKLOADS[args.workload]
        P = len(points)
        cfg = {"workload": args.workload, "points": P, "walks_per_point": w["walks"], "M": w["M"],
               "dim": problem["dim"], "sched_group": args.sched_group}
        for s in range(args.warmup + args.steps):
            r = cpu_oracle_sample(problem, points, w["M"], w["walks"], target_s=target, sched_group=args.sched_group)
            if s >= args.warmup:
                times.append(r)
    v = float(np.mean([r["value"] for r in times]))
    cfg.update(precision="fp64 (CPU oracle)", l2="n/a (host cores)", parallelism=f"host threads x{times[-1]['cores']}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "estimates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * P / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "estimates/s", "cores": times[-1]["cores"], "kind": "oracle",
                             "cpu_model": times[-1]["cpu_model"], "sample": times[-1]["sample"]},
            "e2e": {"value": v, "unit": "estimates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# one instance (the single-workload line and the extra workloads)
# ---------------------------------------------------------------------------

def measure_single(name, args, local, steps, warmup, extras=True):
    """Times woi_estimate over a whole single-instance workload (inputs in HBM, L2 flushed
    between steps) and returns the measurements of one workload."""
    import torch
    from paper_2508_16767_gb300 import woi
    cfg = WORKLOADS[name]
    problem, points = make_workload(name)
    if args.points:
        points = np.ascontiguousarray(points[:args.points])
    P, d, Wk, M = len(points), problem["dim"], cfg["walks"], cfg["M"]
    sg = args.sched_group or cfg.get("sched_group", 1)
    ws, rank, _ = dist_env()
    ell = any(srf["kind"] == "ellipsoid" for srf in problem["surfaces"])
    geom = woi.Geometry(problem)
    stream = torch.cuda.Stream()
    xd = torch.from_numpy(points).cuda()
    outs = tuple(torch.empty(shape, dtype=torch.float64, device="cuda") for shape in ((P,), (P, d), (P,), (P, d)))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    opt = dict(M=M, precision=args.precision, sched_group=sg, block_size=args.block,
               walks_per_lane=args.walks_per_lane, tile_points=args.tile_points)

    def step(timing, o=opt):
        if ws == 1:
            return woi.woi_estimate(geom, xd, Wk, seed=0, out=outs, stream=stream.cuda_stream, timing=timing, **o)
        # rank r runs the walks [r W, (r + 1) W) of every point; the moments of all ranks are summed
        # (NCCL) and finalized by the library: one estimate with ws W walks per point
        from paper_2508_16767_gb300 import parallel
        mom = woi.woi_estimate_range(geom, xd, rank * Wk, Wk, seed=0, stream=stream.cuda_stream, timing=timing, **o)
        with torch.cuda.stream(stream):
            parallel.allreduce_moments(mom)
        return woi.woi_finalize_moments(mom, ws * Wk, sg, out=outs, stream=stream.cuda_stream)

    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kernel_ms = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[k][0].record(stream)
            step(True)
            ev[k][1].record(stream)
            kernel_ms.append(woi.woi_last_kernel_ms(geom))
        torch.cuda.synchronize()
    t_step = sum(a.elapsed_time(b) for a, b in ev) / 1000.0 / steps
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())
    k_ms = float(np.mean(kernel_ms))
    peak, peak_src = fp32_peak_tflops(local)
    if args.tile_points:
        n_tiles = -(-P // args.tile_points)
        flops = Wk * (M + 1) * (n_tiles * (alg_flops_per_walk_step(d, ell) - alg_tally_flops(d)) + P * alg_tally_flops(d))
    else:
        flops = P * Wk * (M + 1) * alg_flops_per_walk_step(d, ell)
    achieved = flops / (k_ms / 1000.0) / 1e12
    res = {"value": ws * P / t_step, "unit": "estimates/s", "ms_per_step": 1000.0 * t_step,
           "walk_steps_per_s": ws * P * Wk * (M + 1) / t_step,
           "config": {"workload": name, "points": P, "walks_per_point": Wk, "M": M, "dim": d,
                      "precision": args.precision, "sched_group": sg, "tile_points": args.tile_points},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "traffic": TRAFFIC.get(name), "peak_source": peak_src, "kernel_ms": k_ms,
                        "alg_flops_per_walk_step": alg_flops_per_walk_step(d, ell)},
           "clocks": clk.summary(), "gpu_launches": steps * (2 if args.precision == "mixed" else P + 1)}
    res["accuracy"] = accuracy(outs[0].cpu().numpy(), outs[1].cpu().numpy(), outs[2].cpu().numpy(),
                               outs[3].cpu().numpy(), ws * Wk)
    if not extras or rank != 0 or ws != 1 or args.precision != "mixed" or args.tile_points or args.no_vr:
        geom.close()
        return res, problem, points

    # the variance-reduced variant (Alg. 3): two chains per walk; at the plain path's RMS error
    # it needs (se_vr / se_plain)^2 of the walks
    vo = dict(opt, variant="vr")
    try:
        step(False, vo)
        vr_ok = True
    except woi.WoiError as e:
        if e.status != 4:                     # WOI_E_UNSUPPORTED
            raise
        vr_ok = False
    if vr_ok:
        vms = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(False, vo)
            e1.record(stream)
            torch.cuda.synchronize()
            vms.append(e0.elapsed_time(e1))
        t_v = float(np.mean(vms)) / 1000.0
        acc_v = accuracy(outs[0].cpu().numpy(), outs[1].cpu().numpy(), outs[2].cpu().numpy(), outs[3].cpu().numpy(), Wk)
        ratio = (acc_v["rms_se_u"] / res["accuracy"]["rms_se_u"]) ** 2
        res["variance_reduced"] = {"value": P / t_v, "unit": "estimates/s", "ms_per_step": 1000.0 * t_v,
                                   "value_at_plain_rms_error": P / (t_v * ratio), "accuracy": acc_v,
                                   "note": "two chains per walk; value_at_plain_rms_error scales the walks by "
                                           "(se_vr / se_plain)^2"}
    # shared trajectories (Sec. 4.6: tiles of 32 points share their walks) on the nested spheres
    if name in ("3d-nested", "6d-nested"):
        so = dict(opt, tile_points=32, block_size=0, walks_per_lane=0)
        step(False, so)
        sms = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(True, so)
            e1.record(stream)
            torch.cuda.synchronize()
            sms.append((e0.elapsed_time(e1), woi.woi_last_kernel_ms(geom)))
        t_s = float(np.mean([a for a, _ in sms])) / 1000.0
        k_s = float(np.mean([b for _, b in sms]))
        n_tiles = -(-P // 32)
        fl = Wk * (M + 1) * (n_tiles * (alg_flops_per_walk_step(d, ell) - alg_tally_flops(d)) + P * alg_tally_flops(d))
        res["shared_trajectories"] = {
            "value": P / t_s, "unit": "estimates/s", "ms_per_step": 1000.0 * t_s, "tile_points": 32, "kernel_ms": k_s,
            "roofline_frac": fl / (k_s / 1000.0) / 1e12 / peak,
            "accuracy": accuracy(outs[0].cpu().numpy(), outs[1].cpu().numpy(), outs[2].cpu().numpy(),
                                 outs[3].cpu().numpy(), Wk),
            "note": "each tile's 32 points share one walk stream: the SE of every point is its own, the errors "
                    "of points in a tile are correlated"}
    geom.close()
    return res, problem, points


def run_single_line(args, ws, rank, local):
    import torch
    from paper_2508_16767_gb300 import woi
    res, problem, points = measure_single(args.workload, args, local, args.steps, args.warmup)
    P, d = len(points), problem["dim"]
    cfg = WORKLOADS[args.workload]
    line = None
    if rank == 0:
        e2e = None
        if ws == 1:
            # end to end through the C ABI with pinned host buffers, copies inside the timed region
            geom = woi.Geometry(problem)
            stream = torch.cuda.Stream()
            opt = dict(M=cfg["M"], precision=args.precision, sched_group=res["config"]["sched_group"],
                       tile_points=args.tile_points)
            hp = torch.from_numpy(points).pin_memory()
            ho = tuple(torch.empty(s, dtype=torch.float64).pin_memory() for s in ((P,), (P, d), (P,), (P, d)))
            woi.woi_estimate(geom, hp, cfg["walks"], seed=0, out=ho, stream=stream.cuda_stream, **opt)
            n_e2e = 3
            t0 = time.perf_counter()
            for _ in range(n_e2e):
                woi.woi_estimate(geom, hp, cfg["walks"], seed=0, out=ho, stream=stream.cuda_stream, **opt)
            te = (time.perf_counter() - t0) / n_e2e
            geom.close()
            e2e = {"value": P / te, "unit": "estimates/s", "h2d_bytes_per_step": P * d * 8,
                   "d2h_bytes_per_step": P * (2 + 2 * d) * 8, "calls": n_e2e}
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = cpu_oracle_sample(problem, points, cfg["M"], cfg["walks"], sched_group=res["config"]["sched_group"],
                                    single_core=True)
        line = {"metric": METRIC, "value": res["value"], "unit": "estimates/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": dict(res["config"], l2="flushed between steps (512 MiB write outside the step events)",
                               parallelism=f"replicas x{ws}, disjoint walk ranges, moments all-reduced"),
                "walk_steps_per_s": res["walk_steps_per_s"], "accuracy": res["accuracy"], "roofline": res["roofline"],
                "cpu_baseline": cpu, "variance_reduced": res.get("variance_reduced"),
                "shared_trajectories": res.get("shared_trajectories"), "e2e": e2e,
                "clocks": res["clocks"], "gpu_launches": res["gpu_launches"]}
    return line


# ---------------------------------------------------------------------------
# the batch (headline)
# ---------------------------------------------------------------------------

def run_batch_line(args, ws, rank, local):
    """256 heterogeneous 2D / 3D manufactured-solution instances in one batched call (one
    persistent launch per dimension, replayed as a CUDA graph)."""
    import torch
    from paper_2508_16767_gb300 import woi
    from paper_2508_16767_gb300 import workloads as wl
    insts = wl.batch_instances(n_inst=args.instances)
    geoms = [woi.Geometry(it["problem"]) for it in insts]
    stream = torch.cuda.Stream()
    dev = [(g, torch.from_numpy(it["points"]).cuda(), it["n_walks"]) for g, it in zip(geoms, insts)]
    P = sum(len(it["points"]) for it in insts)
    walk_steps = sum(len(it["points"]) * it["n_walks"] * (it["problem"]["M"] + 1) for it in insts)
    opt = dict(precision=args.precision, sched_group=args.sched_group or 1, block_size=args.block,
               walks_per_lane=args.walks_per_lane)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)

    # outputs allocated once, outside the timed steps
    dev_out = [tuple(torch.empty(s, dtype=torch.float64, device="cuda") for s in
                     ((len(it["points"]),), (len(it["points"]), it["problem"]["dim"]), (len(it["points"]),),
                      (len(it["points"]), it["problem"]["dim"]))) for it in insts]

    def step(timing=False):
        if ws == 1:
            return woi.woi_estimate_batch(dev, seed=0, stream=stream.cuda_stream, timing=timing, out=dev_out, **opt)
        # rank r: walks [r W_k, (r + 1) W_k) of every instance; moments all-reduced, finalized
        from paper_2508_16767_gb300 import parallel
        res = []
        for k, (g, xd, w) in enumerate(dev):
            mom = woi.woi_estimate_range(g, xd, rank * w, w, seed=0, stream=stream.cuda_stream,
                                         M=insts[k]["problem"]["M"], **opt)
            with torch.cuda.stream(stream):
                parallel.allreduce_moments(mom)
            res.append(woi.woi_finalize_moments(mom, ws * w, opt["sched_group"], stream=stream.cuda_stream))
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[k][0].record(stream)
            out = step(timing=ws == 1)
            ev[k][1].record(stream)
            if ws == 1:
                kernel_ms.append(woi.woi_last_kernel_ms(geoms[0]))
        torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) / 1000.0 / args.steps
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    if rank != 0:
        for g in geoms:
            g.close()
        return None
    W_pt = np.concatenate([np.full(len(it["points"]), ws * it["n_walks"]) for it in insts])

    def gather(res):
        f = lambda key: [r[key].cpu().numpy() if hasattr(r[key], "cpu") else r[key] for r in res]
        return f("u"), f("grad"), f("se_u"), f("se_grad")

    def grad_rms_err(res):
        """RMS over points of |grad u - grad u_h| (u_h the manufactured solution; grad u has
        no additive constant), per dimension, and its ratio to the RMS SE of grad u."""
        out = {}
        for dim in (2, 3):
            err, se = [], []
            for it, r in zip(insts, res):
                if it["problem"]["dim"] != dim:
                    continue
                g = r["grad"].cpu().numpy() if hasattr(r["grad"], "cpu") else r["grad"]
                s = r["se_grad"].cpu().numpy() if hasattr(r["se_grad"], "cpu") else r["se_grad"]
                _, gh = wl.eval_poly(it["problem"]["u_h"], it["points"])
                err.append(np.sum((g - gh) ** 2, axis=1))
                se.append(np.sum(s ** 2, axis=1))
            e, s = np.concatenate(err), np.concatenate(se)
            out[f"{dim}d"] = {"rms_err_grad": float(np.sqrt(np.mean(e))), "rms_se_grad": float(np.sqrt(np.mean(s)))}
        return out

    acc = accuracy(*gather(out), W_pt)
    acc["closed_form"] = grad_rms_err(out)
    k_ms = float(np.mean(kernel_ms)) if kernel_ms else None
    peak, peak_src = fp32_peak_tflops(local)
    flops = sum(len(it["points"]) * it["n_walks"] * (it["problem"]["M"] + 1) * alg_flops_per_walk_step(it["problem"]["dim"])
                for it in insts)
    roof = None
    clocks = clk.summary()
    if k_ms:
        achieved = flops / (k_ms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TRAFFIC.get("batch"), "kernel_ms": k_ms, "peak_source": peak_src,
                "alg_flops": "sum over instances of points x walks x (M+1) x (30 in 2D, 11 d + 15 in 3D)"}
        ips = INST_PER_STEP["batch"]
        if all(ips.get(d) for d in (2, 3)):
            steps_d = {d: sum(len(it["points"]) * it["n_walks"] * (it["problem"]["M"] + 1) for it in insts
                              if it["problem"]["dim"] == d) for d in (2, 3)}
            sms = torch.cuda.get_device_properties(local).multi_processor_count
            mhz = (clocks or {}).get("sm_mhz") or peaks()[0].get("sm_max_mhz", 2070.0)
            cycles = k_ms / 1000.0 * mhz * 1e6
            inst = sum(ips[d]["inst"] * steps_d[d] for d in (2, 3))
            xu = sum(ips[d]["xu"] * steps_d[d] for d in (2, 3))
            roof["issue_frac"] = inst / (sms * 4 * cycles)
            roof["xu_frac"] = xu / (sms * XU_PEAK_PER_SM_CYCLE * cycles) if XU_PEAK_PER_SM_CYCLE else None
            roof["inst_per_walk_step"] = {f"{d}d": ips[d]["inst"] for d in (2, 3)}
            roof["issue_note"] = ("warp instructions per walk-step from ncu (sm__inst_executed.sum), times the live "
                                  "walk-step rate, over 4 issue slots per SM per cycle at the sampled SM clock")
    line = {"metric": METRIC, "value": ws * P / t, "unit": "estimates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": "batch", "instances": len(insts), "points": P, "walk_steps": int(walk_steps),
                       "walks_per_point": "log-uniform 1e4..1e5 per instance", "M": "4 (2D) / 6 (3D)",
                       "precision": args.precision,
                       "l2": "flushed between steps (512 MiB write outside the step events)",
                       "parallelism": f"replicas x{ws}, disjoint walk ranges, moments all-reduced"},
            "walk_steps_per_s": ws * walk_steps / t, "accuracy": acc, "roofline": roof,
            "clocks": clocks, "gpu_launches": args.steps * (4 if ws == 1 else 2 * len(insts))}
    if ws == 1:
        # end to end: pinned host inputs and outputs, host<->device copies inside the timed region
        hp = [torch.from_numpy(it["points"]).pin_memory() for it in insts]
        ho = [tuple(torch.empty(s, dtype=torch.float64).pin_memory() for s in
                    ((len(it["points"]),), (len(it["points"]), it["problem"]["dim"]), (len(it["points"]),),
                     (len(it["points"]), it["problem"]["dim"]))) for it in insts]
        host = [(g, x, it["n_walks"]) for g, x, it in zip(geoms, hp, insts)]
        woi.woi_estimate_batch(host, seed=0, out=ho, **opt)
        n_e2e = 3
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            woi.woi_estimate_batch(host, seed=0, out=ho, **opt)
        te = (time.perf_counter() - t0) / n_e2e
        line["e2e"] = {"value": P / te, "unit": "estimates/s",
                       "h2d_bytes_per_step": int(sum(it["points"].size * 8 for it in insts)),
                       "d2h_bytes_per_step": int(sum(len(it["points"]) * (2 + 2 * it["problem"]["dim"]) * 8
                                                     for it in insts)), "calls": n_e2e}
    if ws == 1 and args.precision == "mixed" and not args.no_fp64_baseline:
        # the plain FP64 path over the whole batch: instance by instance, one launch per point,
        # the same walks -- so the same estimator and the same error; timed once
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r64 = woi.woi_estimate_batch(dev, seed=0, stream=stream.cuda_stream, precision="fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1000.0
        acc64 = accuracy(*gather(r64), W_pt)
        u32 = np.concatenate(gather(out)[0])
        u64, se64 = np.concatenate(gather(r64)[0]), np.concatenate(gather(r64)[2])
        line["fp64_plain_gpu_path"] = {
            "value": P / t64, "unit": "estimates/s", "ms_per_step": 1000.0 * t64, "launches": P + len(insts),
            "measured": "whole batch, same walks (one timed call)",
            "rms_se_u": acc64["rms_se_u"], "closed_form": grad_rms_err(r64),
            "max_diff_u_in_se": float(np.max(np.abs(u32 - u64) / np.maximum(se64, 1e-300))),
            "speedup_of_mixed": (P / t) / (P / t64)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_batch_sample(insts, single_core=True)
    for g in geoms:
        g.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--workload", default="batch", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads (extra_workloads)")
    ap.add_argument("--no-vr", action="store_true", help="skip the variance-reduced comparison")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--walks-per-lane", type=int, default=0)
    ap.add_argument("--sched-group", type=int, default=0, help="walkers per schedule (default: the workload's)")
    ap.add_argument("--points", type=int, default=0, help="use only the first N points (profiling)")
    ap.add_argument("--instances", type=int, default=256, help="batch workload: number of instances")
    ap.add_argument("--tile-points", type=int, default=0, choices=[0, 32],
                    help="32: tiles of 32 points share their walks (Sec. 4.6)")
    args = ap.parse_args()
    if args.impl == "reference":
        if not args.sched_group:
            args.sched_group = WORKLOADS.get(args.workload, {}).get("sched_group", 1) or 1
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_16767_gb300 import build
    build.build()

    if args.workload == "batch":
        line = run_batch_line(args, ws, rank, local)
    else:
        line = run_single_line(args, ws, rank, local)
    if line is not None and ws == 1 and not args.no_extras and args.workload == "batch":
        # the other workloads, each over its whole size (1 warm-up, 3 timed steps)
        extra = {}
        for name in EXTRAS:
            res, _, _ = measure_single(name, args, local, steps=3, warmup=1)
            res.pop("clocks", None)
            extra[name] = res
        line["extra_workloads"] = extra
    if line is not None and rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
