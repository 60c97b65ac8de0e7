"""Serving loop: many NACA 0012 solves at once, each run to a converged Cd/Cl.

Requests (an angle of attack and a grid, arriving over time) are admitted
while their workspaces fit in a device-memory budget, stepped together as one
batch of lattices (`vplbm_batch_*`: each lattice on a stream of its own,
replaying its own step graphs), and retired when converged; the batch is re-formed
whenever its membership changes (continuous batching).  Convergence follows
the time-averaging of Sec. 3.1: the means of Cd = 2F_x/(rho0 U0^2 C) and
Cl = 2F_y/(rho0 U0^2 C) over consecutive windows of `window` steps (from the
device's running force sums) change by less than `tol`, or the request
reaches `cap` steps and is reported unconverged.

The scheduling logic only needs a backend with `make(request)` returning a
lattice (`nbytes`, `sums()`, `reset_sums()`, `close()`) and `batch(lattices)`
returning a batch (`step(n)`, `close()`); `GpuBackend` is the CUDA one.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

U0 = 0.05  # free-stream velocity of the NACA workloads (lattice units)


@dataclass
class Result:
    rid: int
    alpha_deg: float
    nx: int
    ny: int
    arrival: float
    start: float = 0.0
    finish: float = 0.0
    steps: int = 0
    converged: bool = False
    rejected: bool = False
    cd: float = float("nan")      # last window mean, MEM
    cl: float = float("nan")
    cd_sim: float = float("nan")  # last window mean, SIM
    cl_sim: float = float("nan")

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


@dataclass
class _Active:
    req: object
    lat: object
    res: Result
    chord: float
    prev: tuple = field(default=(np.nan, np.nan))


def coefficients(force_sums, counts, chord: float):
    """Window means (Cd, Cl) of MEM and of SIM from the device's running sums
    (F_x, F_y, T of MEM then SIM) and the steps they cover."""
    def cc(fx, fy, n):
        if n <= 0:
            return float("nan"), float("nan")
        q = 0.5 * U0 * U0 * chord  # rho0 = 1
        return fx / n / q, fy / n / q
    return cc(force_sums[0], force_sums[1], counts[0]) + cc(force_sums[3], force_sums[4], counts[1])


class Server:
    def __init__(self, backend, memory_bytes: int, window: int = 1000, tol: float = 1e-4,
                 cap: int = 200_000, max_active: int = 0):
        if window <= 0 or cap <= 0:
            raise ValueError("window and cap must be positive")
        self.backend = backend
        self.memory_bytes = memory_bytes
        self.window = window
        self.tol = tol
        self.cap = cap
        self.max_active = max_active  # 0: no limit beyond memory; 1: one request at a time

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep) -> list:
        """Serves the requests (sorted by arrival time, seconds after the
        start) and returns one Result per request, in request order."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        results = {r.rid: Result(r.rid, r.alpha_deg, r.nx, r.ny, r.arrival) for r in requests}
        active: list[_Active] = []
        used = 0
        batch = None
        t0 = clock()
        while pending or active:
            now = clock() - t0
            changed = False
            # admission: arrived requests, in arrival order, while memory lasts
            while pending and pending[0].arrival <= now:
                req = pending[0]
                need = self.backend.nbytes(req)
                if need > self.memory_bytes:  # can never fit
                    res = results[req.rid]
                    res.rejected = True
                    res.start = res.finish = now
                    pending.pop(0)
                    continue
                if used + need > self.memory_bytes or (
                        self.max_active and len(active) >= self.max_active):
                    break
                pending.pop(0)
                lat = self.backend.make(req)
                used += need
                res = results[req.rid]
                res.start = clock() - t0
                active.append(_Active(req, lat, res, chord=req.nx * 200.0 / 2048.0))
                changed = True
            if not active:
                if pending:
                    sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.05)))
                continue
            if changed or batch is None:
                if batch is not None:
                    batch.close()
                batch = self.backend.batch([a.lat for a in active])
            if hasattr(self.backend, "range_push"):
                self.backend.range_push(f"serve window: {len(active)} requests")
            batch.step(self.window)
            retired = []
            for a in active:
                sums, counts = a.lat.sums()
                a.lat.reset_sums()
                cd, cl, cds, cls = coefficients(sums, counts, a.chord)
                a.res.steps += self.window
                a.res.cd, a.res.cl, a.res.cd_sim, a.res.cl_sim = cd, cl, cds, cls
                done = (abs(cd - a.prev[0]) < self.tol and abs(cl - a.prev[1]) < self.tol)
                a.prev = (cd, cl)
                if done or a.res.steps >= self.cap:
                    a.res.converged = bool(done)
                    a.res.finish = clock() - t0
                    retired.append(a)
            if hasattr(self.backend, "range_pop"):
                self.backend.range_pop()
            if retired:
                for a in retired:
                    active.remove(a)
                    used -= self.backend.nbytes(a.req)
                    a.lat.close()
                batch.close()
                batch = None
        if batch is not None:
            batch.close()
        return [results[r.rid] for r in requests]


def summary(results, elapsed: float, nodes_steps: float) -> dict:
    """Throughput and latency figures of a served mix.  A solve is a request
    whose Cd/Cl converged; requests stopped at the step cap are counted apart
    (with their own throughput), and the latencies are those of the converged
    requests (time from arrival to converged Cd/Cl)."""
    served = [r for r in results if not r.rejected]
    conv = [r for r in served if r.converged]
    lat_c = np.array([r.latency for r in conv]) if conv else np.full(1, np.nan)
    lat_all = np.array([r.latency for r in served]) if served else np.full(1, np.nan)
    per_s = (lambda n: n / elapsed) if elapsed > 0 else (lambda n: 0.0)
    return {
        "solves_per_s": per_s(len(conv)),
        "completed_per_s": per_s(len(served)),
        "p50_s": float(np.percentile(lat_c, 50)),
        "p99_s": float(np.percentile(lat_c, 99)),
        "p50_all_s": float(np.percentile(lat_all, 50)),
        "p99_all_s": float(np.percentile(lat_all, 99)),
        "converged": len(conv),
        "capped": len(served) - len(conv),
        "rejected": sum(r.rejected for r in results),
        "mlups": nodes_steps / elapsed / 1e6 if elapsed > 0 else 0.0,
    }


class GpuBackend:
    """Lattices of the CUDA library for NACA 0012 requests (geometry scaled
    with nx, Re 1000, inlet u = 0.05), in the given storage form."""

    def __init__(self, dtype: str = "f32", device=None, tune_trials: int = 0):
        import torch
        from . import vplbm as V
        from . import workloads as W
        self.V, self.W, self.torch = V, W, torch
        self.dtype = dtype
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = torch.cuda.current_stream(self.device)
        # launch form of the bulk kernel per grid size: the default form
        # (tune_trials 0), or tuned (tune_mix, or once per size on a scratch
        # lattice when a size first arrives)
        self.tune_trials = tune_trials
        self.forms: dict = {}

    def workload(self, req):
        return self.W.naca(req.alpha_deg, dtype=self.dtype, nx=req.nx, ny=req.ny)

    def nbytes(self, req) -> int:
        return self.V.vplbm_workspace_bytes(self.V.config_of(self.workload(req))) + 256

    def tune_mix(self, grids, alpha_deg: float = 10.0) -> dict:
        """Launch forms for the given grid sizes, tuned together: one scratch
        lattice per size stepped as one batch, the batch tuner choosing a
        form per size with the other sizes running beside it, as they do
        when served.  The choices are kept for the requests to come."""
        lats = []
        for nx, ny in grids:
            w = self.W.naca(alpha_deg, dtype=self.dtype, nx=nx, ny=ny)
            lat = self.V.Lattice(self.V.config_of(w), device=self.device, stream=self.stream)
            lat.set_body(self.V.body_of(w))
            lats.append(lat)
        batch = self.V.Batch(lats, stream=self.stream)
        forms = batch.autotune(max(self.tune_trials, 1))
        batch.close()
        for (nx, ny), v, lat in zip(grids, forms, lats):
            self.forms[(nx, ny)] = v
            lat.close()
        return dict(self.forms)

    def form(self, w) -> int:
        """The launch form for the workload's grid size: the tuner's choice on
        a scratch lattice of that size (its steps touch no request)."""
        key = (w.nx, w.ny)
        if key not in self.forms:
            scratch = self.V.Lattice(self.V.config_of(w), device=self.device, stream=self.stream)
            scratch.set_body(self.V.body_of(w))
            self.forms[key] = scratch.autotune(self.tune_trials)
            scratch.close()
        return self.forms[key]

    def make(self, req):
        w = self.workload(req)
        lat = self.V.Lattice(self.V.config_of(w), device=self.device, stream=self.stream)
        lat.set_body(self.V.body_of(w))
        if self.tune_trials > 0:
            lat.bulk_variant = self.form(w)
        lat.reset_sums()
        return lat

    def batch(self, lattices):
        return self.V.Batch(lattices, stream=self.stream)

    # NVTX ranges around each served window, for profiler timelines
    def range_push(self, name: str):
        self.torch.cuda.nvtx.range_push(name)

    def range_pop(self):
        self.torch.cuda.nvtx.range_pop()
