"""Writes sedimentation_trajectory.json: the first STEPS steps of the disk
falling in the closed 400 x 1600 box (D = 50, rho_s/rho = 1.03, TRT tau = 0.6,
released at rest 0.75 D from the left wall and 4 D below the top), driven by
the momentum exchange force (Eq. MMEL) or by the stress integration force
(Eq. defFf), from the FP64 oracle alone.

The rigid body follows Eqs. dep1 / theta2 (Sec. 3.2) with the trapezoidal
update of the oracle; chi is re-rasterised every step.  The file holds, every
EVERY steps, the body state (x_c, y_c, theta, u, v, omega) after that step and
the force (F_x, F_y, torque) of that step.

  python tests/golden/make_sedimentation_trajectory.py [--threads N]

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

STEPS = 10_000
EVERY = 100
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sedimentation_trajectory.json")


def one_case(estimator):
    w = W.sedimentation(estimator, steps=STEPS)
    cfg, body, chi, f, pts = oracle_setup(w)
    mh, sh, bh, missing = o.run(cfg, body, f, chi, STEPS,
                                estimator=o.SIM if estimator == "sim" else o.MEM, sim_pts=pts)
    assert missing == 0
    force = sh if estimator == "sim" else mh
    rows = range(EVERY - 1, STEPS, EVERY)
    return {"body": [[float(v) for v in bh[i]] for i in rows],
            "force": [[float(v) for v in force[i]] for i in rows]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    cores = o.set_threads(args.threads)
    out = {"source": "FP64 oracle (oracle/vplbm_oracle.c), "
                     "tests/golden/make_sedimentation_trajectory.py",
           "passage": "Sec. 3.2: a disk settling under gravity, Eqs. dep1 and theta2, "
                      "driven by MEM (Eq. MMEL) or SIM (Eq. defFf)",
           "workload": "closed 400x1600 box, disk D 50, rho_s/rho 1.03, TRT tau 0.6, "
                       "released at rest 0.75 D from the left wall and 4 D below the top",
           "steps": STEPS, "every": EVERY,
           "layout": "body rows (x_c, y_c, theta, u, v, omega) after steps every, 2 every, ...; "
                     "force rows (F_x, F_y, torque) of those steps",
           "cases": {}}
    for est in ("mem", "sim"):
        t0 = time.time()
        out["cases"][est] = one_case(est)
        print(f"{est}: {time.time() - t0:.0f} s on {cores} threads", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
