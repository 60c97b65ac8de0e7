"""Writes naca512_means.json: time-averaged force coefficients of the NACA 0012
workload on the 512 x 256 lattice (C = 50, U0 = 0.05, tau+ = 0.53, TRT,
Lambda = 1/6, 849 SIM points) at alpha = 0, 5, 10, 15, 20 degrees, from the
FP64 oracle alone.

The quantity is the one Sec. 3.1 reports: Cd = 2 F_x / (rho0 U0^2 C) and
Cl = 2 F_y / (rho0 U0^2 C) averaged in time, for the momentum exchange force
(Eq. MMEL) and the stress integration force (Eq. defFf).  Each run starts from
the initial state feq(1, u_in) and takes STEPS steps; the means cover the last
WINDOW steps.  Besides the means the file holds, per estimator and angle, the
means of the ten consecutive 1000-step blocks of that window and the standard
deviation of the per-step coefficients over it, from which a test can judge how
much of a difference between two runs is the phase of a shedding cycle.

  python tests/golden/make_naca512_means.py [--threads N]

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

ANGLES = (0.0, 5.0, 10.0, 15.0, 20.0)
NX, NY = 512, 256
STEPS = 30_000
WINDOW = 10_000
BLOCK = 1_000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "naca512_means.json")


def coefficients(hist, chord, u0):
    q = 0.5 * u0 * u0 * chord  # rho0 = 1
    return hist[:, 0] / q, hist[:, 1] / q


def one_angle(alpha):
    w = W.naca(alpha, dtype="f64", nx=NX, ny=NY)
    cfg, body, chi, f, pts = oracle_setup(w)
    o.run(cfg, body, f, chi, STEPS - WINDOW, sim_pts=pts, histories=False)
    mh, sh, _, missing = o.run(cfg, body, f, chi, WINDOW, sim_pts=pts)
    assert missing == 0
    rec = {}
    for name, h in (("mem", mh), ("sim", sh)):
        cd, cl = coefficients(h, w.body.length, w.u_in[0])
        for key, c in (("cd", cd), ("cl", cl)):
            rec[f"{key}_{name}"] = float(c.mean())
            rec[f"{key}_{name}_blocks"] = [float(b) for b in c.reshape(-1, BLOCK).mean(axis=1)]
            rec[f"{key}_{name}_std"] = float(c.std())
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    cores = o.set_threads(args.threads)
    out = {"source": "FP64 oracle (oracle/vplbm_oracle.c), tests/golden/make_naca512_means.py",
           "passage": "Sec. 3.1: time-averaged Cd and Cl of the NACA 0012 from MEM and SIM",
           "workload": f"naca0012 {NX}x{NY}, chord {NX * 200 / 2048:g}, u0 0.05, tau+ 0.53, "
                       "TRT Lambda 1/6, eta 1e-6, 849 SIM points, initial state feq(1, u_in)",
           "steps": STEPS, "window": [STEPS - WINDOW + 1, STEPS], "block": BLOCK,
           "angles": {}}
    for a in ANGLES:
        t0 = time.time()
        out["angles"][f"{a:g}"] = one_angle(a)
        print(f"alpha {a:g}: {time.time() - t0:.0f} s on {cores} threads", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
