"""Writes storage_envelopes.json: how far the FP64 oracle moves from itself in
1000 steps when the populations it stores are rounded, after every step, to
the library's storage formats (FP32, FP16, BF16 offsets h = f - feq(1, u_ref),
rounded to nearest even, or for FP16 and BF16 also stochastically: then one
realization per seed of SR_SEEDS, and the largest error over them).  This is the error the storage precision alone
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

  python tests/golden/make_storage_envelopes.py [--threads N] [--formats f16sr,bf16sr]
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


SR_SEEDS = (2110, 2111, 2112, 2113)  # one realization of the random rounding per seed
RNG = np.random.Generator(np.random.PCG64(SR_SEEDS[0]))


def neighbours(h, fmt):
    """The two values of the 16-bit format around each FP64 value (toward
    and away from zero; equal where h is representable)."""
    if fmt.startswith("f16"):
        r = h.astype(np.float16)  # nearest
        rd = r.astype(np.float64)
        toward_inf = np.nextafter(r, np.float16(np.inf)).astype(np.float64)
        toward_minf = np.nextafter(r, np.float16(-np.inf)).astype(np.float64)
        lo = np.where(rd <= h, rd, toward_minf)
        hi = np.where(rd >= h, rd, toward_inf)
        return lo, hi
    m, e = np.frexp(h)  # bfloat16: 8 significant bits, FP32's exponent range
    return np.ldexp(np.floor(m * 256.0) / 256.0, e), np.ldexp(np.ceil(m * 256.0) / 256.0, e)


def round_to(h, fmt):
    """FP64 values rounded to the storage format: to nearest even, or (the
    "sr" formats) stochastically, up with probability (h - lo) / (hi - lo)."""
    if fmt == "f32":
        return h.astype(np.float32).astype(np.float64)
    if fmt == "f16":
        return h.astype(np.float16).astype(np.float64)
    if fmt == "bf16":
        m, e = np.frexp(h)
        return np.ldexp(np.round(m * 256.0) / 256.0, e)
    lo, hi = neighbours(h, fmt[:-2])
    span = hi - lo
    p = np.where(span > 0, (h - lo) / np.where(span > 0, span, 1.0), 0.0)
    return np.where(RNG.random(h.shape) < p, hi, lo)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def main():
    global RNG
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--formats", default="f32,f16,bf16,f16sr,bf16sr",
                    help="formats to (re)compute; the file's other entries are kept")
    args = ap.parse_args()
    o.set_threads(args.threads)
    formats = args.formats.split(",")
    out = {"source": "FP64 oracle with its stored offsets rounded each step, "
                     "tests/golden/make_storage_envelopes.py",
           "passage": "Secs. 2.2 and 3.1 (the NACA workload); the storage formats are the "
                      "library's, not the paper's",
           "steps": STEPS, "sr_seeds": list(SR_SEEDS), "cases": {}}
    if os.path.exists(OUT):
        out["cases"] = json.load(open(OUT))["cases"]
    for name, alpha in CASES.items():
        w = W.naca(alpha, dtype="f64", nx=512, ny=256, steps=STEPS)
        cfg, body, chi, f_ref, pts = oracle_setup(w)
        f0 = f_ref.copy()
        mh, sh, _, _ = o.run(cfg, body, f_ref, chi, STEPS, sim_pts=pts)
        r0, x0, y0 = o.fields(cfg, body, chi, f_ref)
        for oname, u_ref in OFFSETS.items():
            E = o.feq(1.0, u_ref[0], u_ref[1])[:, None, None]
            for fmt in formats:
                runs = []
                for seed in (SR_SEEDS if fmt.endswith("sr") else (None,)):
                    if seed is not None:
                        RNG = np.random.Generator(np.random.PCG64(seed))
                    f = round_to(f0 - E, fmt) + E
                    for _ in range(STEPS):
                        me, se, _, _ = o.run(cfg, body, f, chi, 1, sim_pts=pts)
                        f[:] = round_to(f - E, fmt) + E
                    r1, x1, y1 = o.fields(cfg, body, chi, f)
                    fm = np.abs(me[-1, :2] - mh[-1, :2]).max() / np.abs(mh[-1, :2]).max()
                    fs = np.abs(se[-1, :2] - sh[-1, :2]).max() / np.abs(sh[-1, :2]).max()
                    runs.append({"fields": [rel(r1 - 1, r0 - 1), rel(x1, x0), rel(y1, y0)],
                                 "force_mem": float(fm), "force_sim": float(fs)})
                # a stochastic format: the largest error over its realizations
                rec = {"fields": [max(r["fields"][k] for r in runs) for k in range(3)],
                       "force_mem": max(r["force_mem"] for r in runs),
                       "force_sim": max(r["force_sim"] for r in runs)}
                if len(runs) > 1:
                    rec["realizations"] = runs
                out["cases"][f"{name}/{oname}/{fmt}"] = rec
                print(name, oname, fmt, rec, flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
