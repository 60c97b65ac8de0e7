"""Writes serving_subset.json: the FP64 oracle's Cd and Cl (MEM and SIM) of
the first eight requests of the seeded serving mix (numpy PCG64 seed 2110,
256 requests, alpha uniform in [0, 20] degrees, grids 512 x 256 .. 2048 x 1024;
the NACA 0012 workload scaled with the grid), each run STEPS steps from the
initial state and averaged over the last WINDOW steps: the time averages of
Sec. 3.1 over the window the serving loop uses.

  python tests/golden/make_serving_subset.py [--threads N]

Only the oracle computes here; the workload module supplies the parameters.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as o  # noqa: E402
from paper_2110_00967_gb300 import workloads as W  # noqa: E402
from tests.helpers import oracle_setup  # noqa: E402

COUNT = 8
STEPS = 3000
WINDOW = 1000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serving_subset.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    cores = o.set_threads(args.threads)
    reqs = W.serving_requests(256)[:COUNT]
    out = {"source": "FP64 oracle (oracle/vplbm_oracle.c), tests/golden/make_serving_subset.py",
           "passage": "Sec. 3.1: time-averaged Cd and Cl from MEM and SIM",
           "mix": "serving_requests(256), seed 2110, first 8", "steps": STEPS,
           "window": [STEPS - WINDOW + 1, STEPS], "requests": []}
    for r in reqs:
        t0 = time.time()
        w = W.naca(r.alpha_deg, dtype="f64", nx=r.nx, ny=r.ny)
        cfg, body, chi, f, pts = oracle_setup(w)
        o.run(cfg, body, f, chi, STEPS - WINDOW, sim_pts=pts, histories=False)
        mh, sh, _, missing = o.run(cfg, body, f, chi, WINDOW, sim_pts=pts)
        assert missing == 0
        q = 0.5 * w.u_in[0] ** 2 * w.body.length
        out["requests"].append({
            "rid": r.rid, "alpha_deg": r.alpha_deg, "nx": r.nx, "ny": r.ny,
            "cd_mem": float(mh[:, 0].mean() / q), "cl_mem": float(mh[:, 1].mean() / q),
            "cd_sim": float(sh[:, 0].mean() / q), "cl_sim": float(sh[:, 1].mean() / q)})
        print(r.rid, r.nx, r.ny, f"{r.alpha_deg:.2f}", f"{time.time() - t0:.0f} s on {cores}",
              flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
