"""Long-horizon parity of the time-averaged force coefficients (Sec. 3.1): the
NACA 0012 on the 512 x 256 lattice at alpha = 0, 5, 10, 15, 20 degrees, 30,000
steps from the initial state, Cd and Cl of MEM (Eq. MMEL) and SIM (Eq. defFf)
averaged over steps 20,001 .. 30,000, against the FP64 oracle's means over the
same steps (tests/golden/naca512_means.json, written by
tests/golden/make_naca512_means.py from the oracle alone).

The five angles run as one batch (graph-replayed steps), and the means come
from the library's running force sums, reset after step 20,000.  The error of a
coefficient is |x - x_oracle| / max(|x_oracle|, 1e-2) (the floor keeps the lift
at zero incidence, which vanishes by symmetry, from dividing by zero).
"""
import json
import os

import numpy as np
import pytest

from paper_2110_00967_gb300 import vplbm as V
from paper_2110_00967_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "naca512_means.json")
KEYS = ("cd_mem", "cl_mem", "cd_sim", "cl_sim")


def gpu_means(dtype):
    ref = json.load(open(GOLDEN))
    steps, (w0, w1) = ref["steps"], ref["window"]
    angles = [float(a) for a in ref["angles"]]
    works = [W.naca(a, dtype=dtype, nx=512, ny=256) for a in angles]
    lats = [V.Lattice(V.config_of(w, history_len=64)) for w in works]
    for w, lat in zip(works, lats):
        lat.set_body(V.body_of(w))
    batch = V.Batch(lats)
    batch.step(w0 - 1)
    for lat in lats:
        lat.reset_sums()
    batch.step(steps - (w0 - 1))
    out = {}
    for a, w, lat in zip(angles, works, lats):
        lat.check()
        sums, n = lat.sums()
        assert n[0] == n[1] == w1 - w0 + 1
        q = 0.5 * w.u_in[0] ** 2 * w.body.length
        out[a] = {"cd_mem": sums[0] / n[0] / q, "cl_mem": sums[1] / n[0] / q,
                  "cd_sim": sums[3] / n[1] / q, "cl_sim": sums[4] / n[1] / q}
    batch.close()
    return ref, out


def errors(ref, got):
    err = {}
    for a, g in got.items():
        r = ref["angles"][f"{a:g}"]
        err[a] = {k: abs(g[k] - r[k]) / max(abs(r[k]), 1e-2) for k in KEYS}
    return err


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    V.lib()
    yield


def test_fp32_time_means_within_1e3_of_the_oracle():
    """FP32 storage: every mean coefficient within 1e-3 of the oracle's, at the
    steady angles (0 .. 15 degrees) and at 20 degrees, where the flow sheds
    vortices and the means average over the shedding cycles."""
    ref, got = gpu_means("f32")
    err = errors(ref, got)
    for a in err:
        print("f32", a, {k: f"{got[a][k]:.5f} ({err[a][k]:.1e})" for k in KEYS})
    worst = max(max(e.values()) for e in err.values())
    assert worst <= 1e-3, err


def test_f16_stochastic_time_means_within_1e3_of_the_oracle():
    """FP16 offsets rounded stochastically when stored (the f16sr form): every
    mean coefficient within 1e-3 of the oracle's, but for the lift at zero
    incidence.  There the oracle's lift vanishes by the airfoil's mirror
    symmetry, which the per-node random rounding does not keep: the served
    lift is the mean of that rounding's noise, and it is held to 1e-3 in
    absolute terms (|Cl - Cl_oracle| <= 1e-3) instead of relative to the 1e-2
    floor.  FP16 rounded to nearest misses the 1e-3 bar at every angle (its
    rounding error does not average out over the window), which is why the
    stochastic form exists."""
    ref, got = gpu_means("f16sr")
    err = errors(ref, got)
    for a in err:
        print("f16sr", a, {k: f"{got[a][k]:.5f} ({err[a][k]:.1e})" for k in KEYS})
    for a, e in err.items():
        for k in KEYS:
            if a == 0.0 and k.startswith("cl"):
                r = ref["angles"][f"{a:g}"][k]
                assert abs(got[a][k] - r) <= 1e-3, (a, k, got[a][k], r)
            else:
                assert e[k] <= 1e-3, (a, k, e[k])
