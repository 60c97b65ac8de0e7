#!/usr/bin/env python
"""Benchmark of the VP-LBM hot path on GB300.

Workload: NACA 0012 at Re 1000 on a 2048 x 1024 FP32 lattice (chord 200),
the five angles 0, 5, 10, 15, 20 degrees as five resident lattices.  One
benchmark step advances every lattice by one time step: the fused
collide-penalize-stream kernel with the MEM force and the SIM force (849
points) of that step.  Metric: million lattice-node updates per second
(MLUPS) over all lattices and ranks.  The five lattices hold 5 x 151 MB of
populations, more than the 129 MB L2, and are stepped in turn as one batch
(vplbm_batch_step: each lattice replays its own CUDA graphs of up to 32
steps on a stream of its own).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs the five lattices on its own GPU (weak
scaling; no collective on the data path).  --impl reference times the FP64
CPU oracle on the host cores on the same workload (one lattice-step per
benchmark step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ANGLES = (0.0, 5.0, 10.0, 15.0, 20.0)
NX, NY = 2048, 1024
# populations read once and written once per node: 9 x 4 B + 9 x 4 B for FP32 storage,
# 9 x 2 B + 9 x 2 B for the 16-bit offset forms
BYTES_PER_LUP = {"f32": 72, "f16": 36, "bf16": 36, "f16sr": 36, "bf16sr": 36}
STORAGE_NAME = {"f32": "float", "f16": "__half", "bf16": "__nv_bfloat16", "f16sr": "__half",
                "bf16sr": "__nv_bfloat16"}
# the arithmetic of the step: FP32, with the 16-bit forms storing FP16 / BF16
# offsets and colliding in FP32 (force sums FP64 in every form)
DTYPE_NAME = {"f32": "f32", "f16": "f16-storage/f32-compute", "bf16": "bf16-storage/f32-compute",
              "f16sr": "f16-storage-stochastic/f32-compute",
              "bf16sr": "bf16-storage-stochastic/f32-compute"}
# the bulk kernel of each storage form (the special kernel runs beside it)
BULK_NAME = {"f32": "bulk32x2_kernel", "f16": "bulk16_kernel<__half>",
             "bf16": "bulk16_kernel<__nv_bfloat16>", "f16sr": "bulk16_kernel<__half, sr>",
             "bf16sr": "bulk16_kernel<__nv_bfloat16, sr>"}
PROFILE = os.path.join(ROOT, "profiles", "step_kernel_naca2048_f32.md")
KERNEL_SOURCES = ("paper_2110_00967_gb300/csrc/step.cu",
                  "paper_2110_00967_gb300/csrc/vplbm_internal.cuh",
                  "paper_2110_00967_gb300/csrc/api.cu")
METRIC = "VP-LBM MLUPS"
CHUNK = 32  # the longest step graph of a lattice
E2E_RUNS = 3  # end-to-end solves timed; the median is reported
HISTORY = 64  # force-history ring of each lattice
def workload_name(dtype: str) -> str:
    return f"naca0012-re1000-2048x1024-{dtype}-alpha0,5,10,15,20"


def config_block(dtype: str = "f32", extra=None):
    mb = 151 if dtype == "f32" else 75
    c = {"workload": workload_name(dtype), "grid": [NX, NY], "instances": len(ANGLES),
         "chord": 200, "reynolds": 1000, "tau_plus": 0.53, "collision": "trt-lambda-1/6",
         "storage": "f32" if dtype == "f32" else f"{dtype} offsets from feq(1, u_in)",
         "forces_per_step": ["mem", "sim-849"],
         "l2": f"inputs larger than L2: 5 lattices x {mb} MB ping-pong, stepped side by side"
               + (" (ncu range replay: DRAM traffic 151.9 MB per lattice step, 151.0 algorithmic)"
                  if dtype == "f32" else "")}
    if extra:
        c.update(extra)
    return c


def kernel_sources_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(dtype: str = "f32"):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source (FP32 storage only)."""
    if dtype != "f32":
        return None
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_sources_hash():
        return None
    return float(m.group(1))


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
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
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# multi-rank plumbing (also exercised with gloo on CPU by the tests)
# ---------------------------------------------------------------------------
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_instance(alpha: float):
    import oracle as o
    from paper_2110_00967_gb300 import workloads as W
    w = W.naca(alpha, dtype="f64")
    cfg = o.make_config(w.nx, w.ny, bc=(o.BC_INLET, o.BC_OUTLET, o.BC_SYMMETRY, o.BC_SYMMETRY),
                        collision=o.TRT, tau_plus=w.tau_plus, lambda_trt=w.lambda_trt,
                        eta=w.eta, u_in=w.u_in)
    body = o.make_body(o.BODY_NACA, length=w.body.length, thickness=w.body.thickness,
                       xg=w.body.x_c, yg=w.body.y_c, theta=w.body.angle,
                       pivot_frac=w.body.pivot_chord_frac)
    chi = o.raster(body, w.nx, w.ny)
    f = o.init(cfg, body, chi)
    return cfg, body, chi, f, o.sim_points(body)


def time_oracle(steps: int, warmup: int):
    """Oracle steps (collision, MEM, SIM, streaming) of the 10-degree lattice."""
    import oracle as o
    cores = o.set_threads(os.cpu_count() or 1)
    cfg, body, chi, f, pts = oracle_instance(10.0)
    if warmup:
        o.run(cfg, body, f, chi, warmup, sim_pts=pts, histories=False)
    t0 = time.perf_counter()
    o.run(cfg, body, f, chi, steps, sim_pts=pts, histories=False)
    dt = time.perf_counter() - t0
    return NX * NY * steps / dt / 1e6, dt, cores


def cpu_baseline_block(budget_s: float = 12.0):
    import oracle as o
    cores = o.set_threads(os.cpu_count() or 1)
    cfg, body, chi, f, pts = oracle_instance(10.0)
    t0 = time.perf_counter()
    o.run(cfg, body, f, chi, 1, sim_pts=pts, histories=False)
    one = time.perf_counter() - t0
    n = int(max(1, min(200, budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.run(cfg, body, f, chi, n, sim_pts=pts, histories=False)
    dt = time.perf_counter() - t0
    return {"value": round(NX * NY * n / dt / 1e6, 3), "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "sample": f"{n} steps of the 10-degree 2048x1024 lattice (FP64 C oracle, "
                      f"{cores} OpenMP threads), {dt:.1f} s"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2110_00967_gb300 import vplbm as V
    from paper_2110_00967_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    works = [W.naca(a, dtype=args.dtype) for a in ANGLES]
    lats = [V.Lattice(V.config_of(w, history_len=HISTORY), device=dev) for w in works]
    for w, lat in zip(works, lats):
        lat.set_body(V.body_of(w))
    # the five lattices advance in lockstep, each replaying its own step graphs
    batch = V.Batch(lats, stream=stream)
    # the bulk kernel's launch form per size class (one class here), timed
    # with the five lattices side by side, before the warm-up
    variants = batch.autotune(64) if not args.no_tune else [lat.bulk_variant for lat in lats]
    # the step graphs of a run of args.steps steps, captured before the timed
    # region (one graph per lattice for up to 32 steps)
    batch.prepare(args.steps)
    # the clock sampler starts before the warm-up, so that the warm-up steps,
    # not an idle wait, lead into the timed region
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    batch.step(args.warmup)
    torch.cuda.synchronize()

    # device-timed region: every lattice advances args.steps steps
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = batch.launches
    barrier(world)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.start()
    start.record(stream)
    batch.step(args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.stop()
    clk = clocks.stop() if clocks else None
    barrier(world)
    launches = batch.launches - l0
    elapsed_ms = reduce_max(start.elapsed_time(end), world, dev)
    lattice_step_ms = elapsed_ms / (args.steps * len(lats))
    for lat in lats:
        lat.check()

    # end-to-end through the public API with host buffers, as a solve runs:
    # place the bodies (geometry and body state up), step, and read every
    # step's forces back (MEM, SIM and the volume integral, 32 steps at a
    # time, queued into pinned host memory behind each run of steps); one
    # synchronisation at the end.  At least 1024 steps, so that placing the
    # bodies weighs as it does in a solve of many steps.
    e2e_steps = max(1024, -(-args.steps // CHUNK) * CHUNK)
    n_chunks = e2e_steps // CHUNK
    pinned = torch.empty((len(lats), n_chunks, CHUNK, 9), dtype=torch.float64, pin_memory=True)
    rows = pinned.numpy()
    # the median of E2E_RUNS such solves (wall-clock time is exposed to the
    # host's own jitter, which one short run can catch)
    e2e_runs = []
    for _ in range(E2E_RUNS):
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for w, lat in zip(works, lats):
            lat.set_body(V.body_of(w))
        for c in range(n_chunks):
            batch.step(CHUNK)
            for i, lat in enumerate(lats):
                V.vplbm_force_history_async(lat.ctx, CHUNK, rows[i, c].ctypes.data)
        torch.cuda.synchronize()
        e2e_runs.append(reduce_max(time.perf_counter() - t0, world, dev))
        assert np.isfinite(rows[:, :, :, :3]).all() and np.isfinite(rows[:, :, :, 3:6]).all()
    e2e_dt = sorted(e2e_runs)[len(e2e_runs) // 2]
    # host -> device per lattice and set_body: the body state and the force region (two
    # buffers each, 152 and 24 bytes) and the 849 SIM points (72 bytes each)
    h2d = len(lats) * (2 * 152 + 2 * 24 + 849 * 72) / e2e_steps
    # device -> host per lattice and step: one history row (9 doubles)
    d2h = len(lats) * 9 * 8
    batch.close()

    nodes = NX * NY * len(lats)
    value = world * nodes * args.steps / (elapsed_ms / 1e3) / 1e6
    e2e_value = world * nodes * e2e_steps / e2e_dt / 1e6
    peak, peak_kind = measured_hbm_peak()
    bpl = BYTES_PER_LUP[args.dtype]
    achieved = bpl * NX * NY / (lattice_step_ms / 1e3) / 1e9
    traffic = profiled_traffic(args.dtype)
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[args.dtype],
        "data": "synthetic",
        "config": config_block(args.dtype, {"parallelism": f"replicas{world}",
                                            "bulk_variant": variants}),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": f"one lattice step: {BULK_NAME[args.dtype]} with "
                               f"special_kernel<{STORAGE_NAME[args.dtype]}> beside it, timed over "
                               "the region",
                     "kernel_avg_us": round(lattice_step_ms * 1e3, 3),
                     "bytes_per_lup": bpl, "peak_kind": peak_kind},
        "e2e": {"value": round(e2e_value, 1), "unit": "MLUPS",
                "h2d_bytes_per_step": round(h2d, 1), "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "runs": E2E_RUNS, "statistic": "median",
                "all_mlups": [round(world * nodes * e2e_steps / t / 1e6, 1) for t in e2e_runs]},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_block()
    return line


def run_sedimentation(args, rank, world, local_rank, paper=False):
    """The sedimentation box (400 x 1600 FP32, disk D = 50, rho_s/rho = 1.03,
    rigid body driven by MEM in one run and by SIM in the other), or with
    `paper` the paper's own channel (1560 x 104, D = 26, zero-velocity inlet
    above, free outlet below; the four density ratios, each driven by MEM and
    by SIM: eight lattices), released at rest and stepped warmup + steps
    times; the timed region covers the last `steps` steps of every run.
    Reports the trajectories' end states (and, for the paper's channel, the
    particle Reynolds numbers beside the paper's terminal values)."""
    import torch
    from paper_2110_00967_gb300 import vplbm as V
    from paper_2110_00967_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    if paper:
        works = [W.sedimentation_paper(r, e) for r in W.RHO_R_PAPER for e in ("mem", "sim")]
    else:
        works = [W.sedimentation(e) for e in ("mem", "sim")]
    lats = [V.Lattice(V.config_of(w), device=dev) for w in works]
    for w, lat in zip(works, lats):
        lat.set_body(V.body_of(w))
    batch = V.Batch(lats, stream=stream)
    batch.prepare(args.steps)
    batch.step(args.warmup)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = batch.launches
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    if args.profile_range:
        torch.cuda.profiler.start()
    start.record(stream)
    batch.step(args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.stop()
    clk = clocks.stop() if clocks else None
    barrier(world)
    elapsed_ms = reduce_max(start.elapsed_time(end), world, dev)
    nodes = works[0].nx * works[0].ny * len(lats)
    traj = {}
    nu = (works[0].tau_plus - 0.5) / 3.0
    for w, lat in zip(works, lats):
        lat.check()
        x, y, th, ux, uy, om = lat.get_body()
        fall_u = ux if paper else -uy  # the fall runs along +x in the paper's channel
        rec = {"x": x, "y": y, "u_x": ux, "u_y": uy, "omega": om,
               "fall": (x - w.body.x_c) if paper else (w.body.y_c - y),
               "re_particle": abs(fall_u) * w.body.length / nu}
        if paper:
            k = W.RHO_R_PAPER.index(w.body.density_ratio)
            rec["re_paper"] = W.RE_TERMINAL_PAPER[k]
            traj[f"rho{w.body.density_ratio}-{w.body.estimator}"] = rec
        else:
            traj[w.body.estimator] = rec
    bpl = BYTES_PER_LUP["f32"]
    lattice_step_ms = elapsed_ms / (args.steps * len(lats))
    achieved = bpl * nodes / len(lats) / (lattice_step_ms / 1e3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    batch.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": round(world * nodes * args.steps / (elapsed_ms / 1e3) / 1e6, 1),
        "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (f"sedimentation-paper-{works[0].nx}x{works[0].ny}-f32-disk26-"
                                "rho1.0015,1.003,1.01,1.03-mem,sim-inlet0-free-outlet" if paper else
                                "sedimentation-400x1600-f32-disk50-rho1.03-mem,sim"),
                   "grid": [works[0].nx, works[0].ny], "instances": len(lats), "tau_plus": 0.6,
                   "gravity": max(abs(g) for g in works[0].body.gravity),
                   "rigid_update": "fp64 every step", "parallelism": f"replicas{world}",
                   **({"physical_time_s": (args.warmup + args.steps) * W.sedimentation_paper_dt()}
                      if paper else {})},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "one lattice step (bulk + special with rigid update and "
                               "re-rasterisation), timed over the region",
                     "kernel_avg_us": round(lattice_step_ms * 1e3, 3), "bytes_per_lup": bpl,
                     "peak_kind": peak_kind},
        "trajectory_after_steps": args.warmup + args.steps,
        "trajectory": traj,
        "gpu_launches": batch.launches - l0,
        "clocks": clk,
    }


def run_serving(args, rank, world, local_rank):
    """A seeded mix of NACA 0012 solves served to convergence (continuous
    batching under a memory budget).  Poisson arrivals at 4 / (mean
    single-instance solve time), the solve time measured first: one 1024 x 512
    request at 10 degrees in FP32, alone, run window by window to convergence
    and scaled to the mix's mean grid size; the same arrival rate for every
    storage form and for the one-at-a-time comparison.  `value` counts
    converged solves only; requests stopped at the step cap are reported
    apart."""
    import torch
    from paper_2110_00967_gb300 import serve as S
    from paper_2110_00967_gb300 import vplbm as V
    from paper_2110_00967_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    backend = S.GpuBackend(args.dtype, device=dev, tune_trials=args.tune_trials)
    # calibration: the single-instance FP32 solve time of a mid-size request
    cal = S.Server(S.GpuBackend("f32", device=dev), memory_bytes=args.memory_gb << 30,
                   window=1000, tol=1e-4, cap=args.cap, max_active=1)
    torch.cuda.synchronize()
    t = time.perf_counter()
    (cal_res,) = cal.run([W.Request(-1, 0.0, 10.0, 1024, 512)])
    torch.cuda.synchronize()
    t_cal = time.perf_counter() - t
    mean_nodes = sum(nx * ny for nx, ny in W.SERVING_GRIDS) / len(W.SERVING_GRIDS)
    solve_s = t_cal * mean_nodes / (1024 * 512)
    rate = 4.0 / solve_s
    # launch forms per grid size, tuned once at server start (outside the
    # served time): together in one batch of the mix's sizes, or each size
    # alone when it first arrives
    t = time.perf_counter()
    if args.tune_trials > 0 and args.tune_mode == "mix":
        backend.tune_mix(W.SERVING_GRIDS)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t
    reqs = W.serving_requests(args.requests, rate=rate)
    srv = S.Server(backend, memory_bytes=args.memory_gb << 30, window=1000, tol=1e-4,
                   cap=args.cap, max_active=args.max_active)
    barrier(world)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    elapsed = reduce_max(time.perf_counter() - t0, world, torch.device("cuda", local_rank))
    node_steps = sum(r.nx * r.ny * r.steps for r in res)
    summ = S.summary(res, elapsed, node_steps)
    if rank != 0:
        return None
    return {
        "metric": "solves/s", "value": round(world * summ["solves_per_s"], 4), "unit": "solves/s",
        "n_gpus": world, "steps": args.cap, "warmup": 1, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[args.dtype], "data": "synthetic",
        "config": {"workload": f"naca0012-serving-{args.requests}req-seed2110-{args.dtype}",
                   "grids": [list(g) for g in W.SERVING_GRIDS], "alpha_deg": [0, 20],
                   "arrival_rate_per_s": round(rate, 4),
                   "calibration": {"request": "1024x512 alpha 10 f32 alone",
                                   "steps": cal_res.steps, "converged": cal_res.converged,
                                   "seconds": round(t_cal, 4),
                                   "mean_solve_s_estimate": round(solve_s, 4)},
                   "window": 1000, "tol": 1e-4,
                   "cap_steps": args.cap, "memory_budget_gb": args.memory_gb,
                   "max_active": args.max_active or "memory-bound",
                   "bulk_forms": ({f"{k[0]}x{k[1]}": v for k, v in sorted(backend.forms.items())}
                                  if args.tune_trials else "default"),
                   "tuning": (f"{args.tune_mode}, {args.tune_trials} timed steps per form, "
                              f"{tune_s:.2f} s at server start" if args.tune_trials and
                              args.tune_mode == "mix" else
                              f"{args.tune_mode}, {args.tune_trials} timed steps per form, "
                              "inside the served time" if args.tune_trials else "none"),
                   "parallelism": f"replicas{world}"},
        "p50_s": round(summ["p50_s"], 4), "p99_s": round(summ["p99_s"], 4),
        "latency": "arrival to converged Cd/Cl, converged requests only",
        "completed_per_s": round(world * summ["completed_per_s"], 4),
        "p50_all_s": round(summ["p50_all_s"], 4), "p99_all_s": round(summ["p99_all_s"], 4),
        "converged": summ["converged"], "capped": summ["capped"],
        "rejected": summ["rejected"], "aggregate_mlups": round(world * summ["mlups"], 1),
        "aggregate_gbs": round(world * summ["mlups"] * BYTES_PER_LUP[args.dtype] / 1e3, 1),
        "elapsed_s": round(elapsed, 3),
    }


def run_naca_large(args, rank, world, local_rank):
    """One 8192 x 4096 NACA 0012 lattice (C = 800, Re 1000: tau+ = 0.62; 2.4 GB
    of FP32 populations, 1.2 GB in 16-bit storage), far larger than L2: the
    bandwidth of a single lattice's step without the help of neighbouring
    lattices running beside it.  Graph-replayed steps timed with events."""
    import torch
    from paper_2110_00967_gb300 import vplbm as V
    from paper_2110_00967_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    w = W.naca(10.0, dtype=args.dtype, nx=8192, ny=4096, tau_plus=0.62)
    lat = V.Lattice(V.config_of(w), device=dev, stream=stream)
    lat.set_body(V.body_of(w))
    variant = lat.autotune(32)
    lat.step(args.warmup)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = lat.launches
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    start.record(stream)
    lat.step(args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    barrier(world)
    lat.check()
    elapsed_ms = reduce_max(start.elapsed_time(end), world, dev)
    nodes = w.nx * w.ny
    bpl = BYTES_PER_LUP[args.dtype]
    step_ms = elapsed_ms / args.steps
    achieved = bpl * nodes / (step_ms / 1e3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": round(world * nodes * args.steps / (elapsed_ms / 1e3) / 1e6, 1),
        "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(step_ms, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAME[args.dtype], "data": "synthetic",
        "config": {"workload": f"naca0012-8192x4096-{args.dtype}-alpha10", "grid": [w.nx, w.ny],
                   "instances": 1, "chord": 800, "reynolds": 1000, "tau_plus": 0.62,
                   "storage": args.dtype, "bulk_variant": [variant],
                   "l2": f"inputs larger than L2: {2 * bpl * nodes / 2 / 1e9:.1f} GB ping-pong",
                   "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "one lattice step (bulk + special), timed over the region",
                     "kernel_avg_us": round(step_ms * 1e3, 3), "bytes_per_lup": bpl,
                     "peak_kind": peak_kind},
        "gpu_launches": lat.launches - l0,
        "clocks": clk,
    }


def run_disk(args, rank, world, local_rank):
    """The 256 x 128 FP64 disk channel (BGK tau 0.65, Re 20, MEM and SIM every
    step), 2000 steps from rest graph-replayed, timed whole; the FP64 oracle's
    run of the same 2000 steps is timed on the host cores beside it.  The
    lattice (4.7 MB) lives in L2 and the step is latency-bound: report the
    time per step."""
    import torch
    from paper_2110_00967_gb300 import vplbm as V
    from paper_2110_00967_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    w = W.disk_channel()
    lat = V.Lattice(V.config_of(w), device=dev)
    times = []
    for rep in range(args.warmup + 1):  # warm-up solves, then the timed one
        lat.set_body(V.body_of(w))
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        lat.step(w.steps)
        end.record(stream)
        torch.cuda.synchronize()
        times.append(start.elapsed_time(end))
    lat.check()
    ms = reduce_max(times[-1], world, dev)
    fx = lat.force_mem()[0]
    cd = 2 * fx / (0.05 ** 2 * 20.0)
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(world * w.nx * w.ny * w.steps / (ms / 1e3) / 1e6, 1),
        "unit": "MLUPS", "n_gpus": world, "steps": w.steps, "warmup": args.warmup,
        "ms_per_step": round(ms / w.steps, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "disk-channel-256x128-f64-re20-bgk", "grid": [w.nx, w.ny],
                   "steps_per_solve": w.steps, "forces_per_step": ["mem", "sim"],
                   "l2": "L2-resident (4.7 MB): latency-bound, reported per step",
                   "parallelism": f"replicas{world}"},
        "us_per_step": round(ms * 1e3 / w.steps, 3),
        "cd_mem_final": cd,
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle as o
        cfg = o.make_config(w.nx, w.ny, bc=(o.BC_INLET, o.BC_OUTLET, o.BC_PERIODIC,
                                            o.BC_PERIODIC),
                            collision=o.BGK, tau_plus=w.tau_plus, eta=w.eta, u_in=w.u_in)
        body = o.make_body(o.BODY_DISK, length=w.body.length, xg=w.body.x_c, yg=w.body.y_c)
        chi = o.raster(body, w.nx, w.ny)
        f = o.init(cfg, body, chi)
        pts = o.sim_points(body)
        cores = o.set_threads(0)
        t0 = time.perf_counter()
        o.run(cfg, body, f, chi, w.steps, sim_pts=pts, histories=False)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(w.nx * w.ny * w.steps / dt / 1e6, 3),
                                "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                "sample": f"the whole {w.steps}-step solve, {dt:.2f} s"}
    return line


SIM_VARIANTS = ((107, 0), (213, 0), (425, 0), (849, 0), (1697, 0), (3393, 0), (849, 1), (3393, 1))


def run_naca_paper(args, rank, world, local_rank, sim_variants=False):
    """The paper's own NACA 0012 case (C = 278, U0 = 0.0599, tau 0.55, 3614 x
    1946 FP32) at ten angles from 0 to 28 degrees as one batch; reports the
    MLUPS of the timed steps, the Cd/Cl means over them (MEM and SIM) and the
    spread of Cl and Cd over the last (up to 50,000) of them.
    With `sim_variants`, the same case at 12 degrees once per SIM variant
    (point counts 107 .. 3393, stress copied or extrapolated to first order):
    the body is fixed, so every lattice carries the same flow and only the
    SIM estimate differs."""
    import dataclasses

    import torch
    from paper_2110_00967_gb300 import vplbm as V
    from paper_2110_00967_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    if sim_variants:
        base = W.naca_paper(12.0, dtype=args.dtype)
        works = [base.with_(body=dataclasses.replace(base.body, n_sim_points=n))
                 for n, _ in SIM_VARIANTS]
        lats = [V.Lattice(V.config_of(w, sim_order=order, max_sim_points=4096), device=dev)
                for w, (_, order) in zip(works, SIM_VARIANTS)]
    else:
        works = [W.naca_paper(a, dtype=args.dtype) for a in W.PAPER_ANGLES]
        lats = [V.Lattice(V.config_of(w, history_len=min(args.steps, 50_000)), device=dev)
                for w in works]
    for w, lat in zip(works, lats):
        lat.set_body(V.body_of(w))
    batch = V.Batch(lats, stream=stream)
    batch.step(args.warmup)
    for lat in lats:
        lat.reset_sums()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = batch.launches
    barrier(world)
    torch.cuda.synchronize()
    start.record(stream)
    batch.step(args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    elapsed_ms = reduce_max(start.elapsed_time(end), world, dev)
    q = 0.5 * 0.0599 ** 2 * 278.0
    coeffs = {}
    for k, (w, lat) in enumerate(zip(works, lats)):
        lat.check()
        sums, n = lat.sums()
        key = (f"n{SIM_VARIANTS[k][0]}-order{SIM_VARIANTS[k][1]}" if sim_variants
               else f"{w.body.angle_deg:g}")
        coeffs[key] = {
            "cd_mem": sums[0] / n[0] / q, "cl_mem": sums[1] / n[0] / q,
            "cd_sim": sums[3] / n[1] / q, "cl_sim": sums[4] / n[1] / q}
        if not sim_variants:
            # unsteadiness over the last steps of the window (up to 50,000): the
            # standard deviation and range of Cl and Cd per estimator
            m = min(args.steps, 50_000)
            for est, name in ((V.MEM, "mem"), (V.SIM, "sim")):
                h = lat.history(est, m)
                coeffs[key][f"cl_{name}_std"] = float(h[:, 1].std() / q)
                coeffs[key][f"cd_{name}_std"] = float(h[:, 0].std() / q)
                coeffs[key][f"cl_{name}_range"] = [float(h[:, 1].min() / q), float(h[:, 1].max() / q)]
    if sim_variants:
        ref = coeffs["n3393-order0"]
        for c in coeffs.values():
            c["rel_to_n3393_order0"] = [(c["cd_sim"] - ref["cd_sim"]) / abs(ref["cd_sim"]),
                                        (c["cl_sim"] - ref["cl_sim"]) / abs(ref["cl_sim"])]
    nodes = works[0].nx * works[0].ny * len(lats)
    bpl = BYTES_PER_LUP[args.dtype]
    lattice_step_ms = elapsed_ms / (args.steps * len(lats))
    achieved = bpl * nodes / len(lats) / (lattice_step_ms / 1e3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    launches = batch.launches - l0
    batch.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": round(world * nodes * args.steps / (elapsed_ms / 1e3) / 1e6, 1),
        "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[args.dtype], "data": "synthetic",
        "config": {"workload": (f"naca0012-paper-3614x1946-{args.dtype}-alpha12-sim-variants"
                                if sim_variants else
                                f"naca0012-paper-3614x1946-{args.dtype}-alpha0..28-10angles"),
                   "grid": [works[0].nx, works[0].ny], "instances": len(lats), "chord": 278,
                   "u0": 0.0599, "tau_plus": 0.55, "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "one lattice step, timed over the region",
                     "kernel_avg_us": round(lattice_step_ms * 1e3, 3), "bytes_per_lup": bpl,
                     "peak_kind": peak_kind},
        "means_over_steps": [args.warmup + 1, args.warmup + args.steps],
        "coefficients": coeffs,
        "gpu_launches": launches,
    }


def run_reference(args, rank, world):
    if rank != 0:
        return None
    mlups, dt, cores = time_oracle(args.steps, args.warmup)
    return {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(args.dtype, {"reference_sample": "one step of the 10-degree "
                                                                "lattice per benchmark step"}),
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{args.steps} steps of the 10-degree 2048x1024 lattice"},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch form instead of tuning it first (fewer "
                         "launches ahead of a profiled region)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed region with cudaProfilerStart/Stop (for ncu's "
                         "application-range replay, which measures the concurrent kernels "
                         "of the whole region)")
    ap.add_argument("--workload",
                    choices=("naca", "sedimentation", "serving", "disk", "naca-paper",
                             "sedimentation-paper", "sim-variants", "naca-large"),
                    default="naca",
                    help="naca: the five NACA 0012 lattices (the benchmark); sedimentation: "
                         "the 400 x 1600 falling-disk box, MEM and SIM runs; serving: a seeded "
                         "mix of NACA solves run to convergence; disk: the FP64 disk channel; "
                         "naca-paper: the paper's C = 278 NACA grid at its angles; "
                         "sedimentation-paper: the paper's D = 26 channel, four density "
                         "ratios, MEM and SIM (20,280 steps per physical second); sim-variants: "
                         "the paper's NACA case at 12 degrees once per SIM point count and "
                         "order; naca-large: one 8192 x 4096 lattice")
    ap.add_argument("--requests", type=int, default=256, help="serving: number of requests")
    ap.add_argument("--cap", type=int, default=200000, help="serving: step cap per request")
    ap.add_argument("--memory-gb", type=int, default=40, help="serving: device-memory budget")
    ap.add_argument("--tune-trials", type=int, default=16,
                    help="serving: timed steps per launch form in the tuner (0: the default "
                         "form everywhere)")
    ap.add_argument("--tune-mode", choices=("mix", "alone"), default="mix",
                    help="serving: tune the launch forms of the mix's grid sizes together in "
                         "one batch at server start (mix), or each size alone on a scratch "
                         "lattice when it first arrives (alone)")
    ap.add_argument("--max-active", type=int, default=0,
                    help="serving: most requests stepped at once (0: as many as fit; 1: one "
                         "request at a time, the single-instance comparison)")
    ap.add_argument("--dtype", choices=("f32", "f16", "bf16", "f16sr", "bf16sr"), default="f32",
                    help="population storage: FP32, or FP16/BF16 offsets (FP32 collision), "
                         "rounded to nearest or (the sr forms) stochastically")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        from __graft_entry__ import build
        build()
        if args.workload in ("sedimentation", "sedimentation-paper"):
            line = run_sedimentation(args, rank, world, local_rank,
                                     paper=args.workload == "sedimentation-paper")
        elif args.workload == "serving":
            line = run_serving(args, rank, world, local_rank)
        elif args.workload == "disk":
            line = run_disk(args, rank, world, local_rank)
        elif args.workload == "naca-large":
            line = run_naca_large(args, rank, world, local_rank)
        elif args.workload in ("naca-paper", "sim-variants"):
            line = run_naca_paper(args, rank, world, local_rank,
                                  sim_variants=args.workload == "sim-variants")
        else:
            line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
