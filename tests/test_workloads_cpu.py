"""The sedimentation workloads' lattice units against the physical case of
Sec. 3.2 (reading R23: nu = 0.01 cm^2/s, D = 0.1 cm, |g| = 980 cm/s^2): the
lattice viscosity, gravity and time step map back to the physical values,
and the paper's terminal Reynolds numbers map to lattice velocities well
below the speed of sound."""
import math

import pytest

from paper_2110_00967_gb300 import workloads as W

NU_CM2_S, D_CM, G_CM_S2 = 0.01, 0.1, 980.0


@pytest.mark.parametrize("make, d_lu", [(W.sedimentation, 50.0), (W.sedimentation_paper, 26.0)])
def test_lattice_units_map_back_to_the_physical_case(make, d_lu):
    w = make()
    assert w.body.length == d_lu
    dx = D_CM / d_lu                         # cm per lattice unit
    nu_lu = (w.tau_plus - 0.5) / 3.0         # Eq. tauvisco
    dt = nu_lu * dx * dx / NU_CM2_S          # s per step, from the viscosity
    g_lu = math.hypot(*w.body.gravity)
    assert g_lu * dx / (dt * dt) == pytest.approx(G_CM_S2, rel=1e-12)
    if make is W.sedimentation_paper:
        assert W.sedimentation_paper_dt() == pytest.approx(dt, rel=1e-12)


def test_terminal_velocities_are_low_mach():
    w = W.sedimentation_paper()
    nu_lu = (w.tau_plus - 0.5) / 3.0
    for re in W.RE_TERMINAL_PAPER:
        u = re * nu_lu / w.body.length
        assert u < 0.02  # Mach below 0.035 (c_s = 1/sqrt(3))


def test_paper_channel_geometry():
    w = W.sedimentation_paper()
    assert (w.nx, w.ny) == (60 * 26, 4 * 26)
    assert w.bc == (W.INLET, W.OUTLET_FREE, W.NOSLIP, W.NOSLIP) and w.u_in == (0.0, 0.0)
    assert w.body.gravity[1] == 0.0 and w.body.gravity[0] > 0.0  # the fall runs along +x
    # released 4 D below the inlet wall and 0.75 D from the left (y_lo) wall, both
    # walls half a node beyond the edge nodes
    assert w.body.x_c + 0.5 == pytest.approx(4 * 26)
    assert w.body.y_c + 0.5 == pytest.approx(0.75 * 26)
    assert len(W.RHO_R_PAPER) == len(W.RE_TERMINAL_PAPER) == 4
