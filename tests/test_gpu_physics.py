"""A calibration, not evidence: the sedimentation case of Sec. 3.2 run on the
GPU against the terminal particle Reynolds numbers the paper prints.

The paper does not give its channel's width.  The workload takes 4 D, and 4 D
was chosen because it reproduces the paper's terminal Reynolds numbers for the
two heavier disks (6 D and 8 D give 30 % and more above them).  So this test
cannot show that the coupled path (penalized flow, force estimator, rigid-body
update, re-rasterised mask) is right: it records that the chosen width still
reproduces the numbers it was chosen for, and fails if a later change moves
the coupled result away from them.  The parity of that path is shown against
the FP64 oracle elsewhere (the sedimentation trajectories)."""
import numpy as np
import pytest

from paper_2110_00967_gb300 import vplbm as V
from paper_2110_00967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_sedimentation_terminal_reynolds_numbers():
    """Calibration of the 4 D channel width: the two heavier disks (rho_r =
    1.01, 1.03), each driven by MEM and by SIM, after 2 s of fall (40,560
    steps): Re = U D / nu within 15 % of the paper's 3.23 and 8.33, the disk
    near the channel's mid-line, and the fall velocity steady (changing by
    less than 3 % over the last 0.2 s)."""
    cases = [(r, e) for r in (1.01, 1.03) for e in ("mem", "sim")]
    works = [W.sedimentation_paper(r, e) for r, e in cases]
    lats = []
    for w in works:
        lat = V.Lattice(V.config_of(w))
        lat.set_body(V.body_of(w))
        lats.append(lat)
    batch = V.Batch(lats)
    steps = 2 * round(1.0 / W.sedimentation_paper_dt())
    batch.step(steps - 4056)
    before = [lat.get_body()[3] for lat in lats]
    batch.step(4056)
    nu = (works[0].tau_plus - 0.5) / 3.0
    for (r, e), w, lat, u0 in zip(cases, works, lats, before):
        lat.check()
        x, y, th, ux, uy, om = lat.get_body()
        re = ux * w.body.length / nu
        re_paper = W.RE_TERMINAL_PAPER[W.RHO_R_PAPER.index(r)]
        assert abs(re - re_paper) <= 0.15 * re_paper, (r, e, re)
        assert abs(ux - u0) <= 0.03 * ux, (r, e, ux, u0)
        assert abs(y - (w.ny - 1) / 2.0) <= 0.1 * w.body.length, (r, e, y)
    batch.close()
