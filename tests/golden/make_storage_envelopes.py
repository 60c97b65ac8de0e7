"""Writes storage_envelopes.json: how far the FP64 oracle moves from itself in
1000 steps when the populations it stores are rounded, after every step, to
the library's storage formats (FP32, FP16, BF16 offsets h = f - feq(1, u_ref),
round to nearest even).  This is the error the storage precision alone
causes, carried through the method's own dynamics (Secs. 2.2 and 3.1); the
GPU tests hold the library's reduced-precision runs to a stated multiple of
it.  The storage rounding is the only change to the oracle's step: every
operation of the step itself stays FP64.

Cases: the NACA 0012 workload on the 512 x 256 lattice at 0 and 10 degrees,
offsets from the free-stream equilibrium (u_ref = u_in) and from the lattice
weights (u_ref = 0).  Per case and format: the field errors (L-inf error over
L-inf of the unrounded oracle's field, for rho - 1, u_x, u_y) and the force
errors (largest of |F_x|, |F_y| error over the largest of the unrounded
oracle's |F_x|, |F_y|, for MEM and SIM) after 1000 steps.

  python tests/golden/make_storage_envelopes.py [--threads N]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as o  # noqa: E402
from paper_2110_00967_gb300 import workloads as W  # noqa: E402
from tests.helpers import oracle_setup  # noqa: E402

STEPS = 1000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "storage_envelopes.json")
CASES = {"naca0-512": 0.0, "naca10-512": 10.0}
OFFSETS = {"free-stream": (0.05, 0.0), "weights": (0.0, 0.0)}


def round_to(h, fmt):
    """Round-to-nearest-even of FP64 values to the storage format."""
    if fmt == "f32":
        return h.astype(np.float32).astype(np.float64)
    if fmt == "f16":
        return h.astype(np.float16).astype(np.float64)
    m, e = np.frexp(h)  # bfloat16: 8 significant bits, FP32's exponent range
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    o.set_threads(args.threads)
    out = {"source": "FP64 oracle with its stored offsets rounded each step, "
                     "tests/golden/make_storage_envelopes.py",
           "passage": "Secs. 2.2 and 3.1 (the NACA workload); the storage formats are the "
                      "library's, not the paper's",
           "steps": STEPS, "cases": {}}
    for name, alpha in CASES.items():
        w = W.naca(alpha, dtype="f64", nx=512, ny=256, steps=STEPS)
        cfg, body, chi, f_ref, pts = oracle_setup(w)
        f0 = f_ref.copy()
        mh, sh, _, _ = o.run(cfg, body, f_ref, chi, STEPS, sim_pts=pts)
        r0, x0, y0 = o.fields(cfg, body, chi, f_ref)
        for oname, u_ref in OFFSETS.items():
            E = o.feq(1.0, u_ref[0], u_ref[1])[:, None, None]
            for fmt in ("f32", "f16", "bf16"):
                f = round_to(f0 - E, fmt) + E
                for _ in range(STEPS):
                    me, se, _, _ = o.run(cfg, body, f, chi, 1, sim_pts=pts)
                    f[:] = round_to(f - E, fmt) + E
                r1, x1, y1 = o.fields(cfg, body, chi, f)
                fm = np.abs(me[-1, :2] - mh[-1, :2]).max() / np.abs(mh[-1, :2]).max()
                fs = np.abs(se[-1, :2] - sh[-1, :2]).max() / np.abs(sh[-1, :2]).max()
                rec = {"fields": [rel(r1 - 1, r0 - 1), rel(x1, x0), rel(y1, y0)],
                       "force_mem": float(fm), "force_sim": float(fs)}
                out["cases"][f"{name}/{oname}/{fmt}"] = rec
                print(name, oname, fmt, rec, flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
