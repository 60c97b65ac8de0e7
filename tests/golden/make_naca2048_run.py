"""Writes naca2048_run.json: the first STEPS steps of the benchmark's NACA 0012
lattice (2048 x 1024, C = 200, Re 1000, TRT, 849 SIM points) at alpha = 20
degrees, where the flow separates, from the FP64 oracle alone.

The file holds the MEM and SIM forces (F_x, F_y, torque) of every EVERY-th
step and, after the last step, rho, u_x and u_y at N_SAMPLE nodes drawn with
numpy's PCG64 (seed SEED) from the whole lattice.

  python tests/golden/make_naca2048_run.py [--threads N]

Only the oracle computes here; the workload module supplies the parameters.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as o  # noqa: E402
from paper_2110_00967_gb300 import workloads as W  # noqa: E402
from tests.helpers import oracle_setup  # noqa: E402

ALPHA = 20.0
STEPS = 4000
EVERY = 10
N_SAMPLE = 2000
SEED = 7
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "naca2048_run.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    cores = o.set_threads(args.threads)
    w = W.naca(ALPHA, dtype="f32", steps=STEPS)
    cfg, body, chi, f, pts = oracle_setup(w)
    t0 = time.time()
    mh, sh, _, missing = o.run(cfg, body, f, chi, STEPS, sim_pts=pts)
    assert missing == 0
    rho, ux, uy = o.fields(cfg, body, chi, f)
    idx = np.random.Generator(np.random.PCG64(SEED)).integers(0, w.nx * w.ny, N_SAMPLE)
    rows = range(EVERY - 1, STEPS, EVERY)
    out = {"source": "FP64 oracle (oracle/vplbm_oracle.c), tests/golden/make_naca2048_run.py",
           "passage": "Sec. 3.1: the NACA 0012 in a uniform stream, MEM (Eq. MMEL) and SIM "
                      "(Eq. defFf) forces",
           "workload": f"naca0012 {w.nx}x{w.ny}, chord 200, u0 0.05, tau+ {w.tau_plus}, TRT "
                       f"Lambda 1/6, eta 1e-6, 849 SIM points, alpha {ALPHA:g}, initial state "
                       "feq(1, u_in)",
           "alpha": ALPHA, "steps": STEPS, "every": EVERY, "seed": SEED,
           "mem": [[float(v) for v in mh[i]] for i in rows],
           "sim": [[float(v) for v in sh[i]] for i in rows],
           "nodes": [int(k) for k in idx],
           "rho": [float(v) for v in rho.ravel()[idx]],
           "ux": [float(v) for v in ux.ravel()[idx]],
           "uy": [float(v) for v in uy.ravel()[idx]]}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(f"{STEPS} steps in {time.time() - t0:.0f} s on {cores} threads")


if __name__ == "__main__":
    main()
