"""Host-side checks of the CUDA library that need no GPU: it builds for
sm_103a, loads, exports every entry point include/vplbm.h declares, and its
pure host calls (workspace sizing, configuration checks) behave."""
import ctypes as C
import os
import re

import pytest

from paper_2110_00967_gb300 import build as B
from paper_2110_00967_gb300 import vplbm as V
from paper_2110_00967_gb300 import workloads as W

HEADER = os.path.join(B.ROOT, "include", "vplbm.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vplbm_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = C.CDLL(path)
    names = declared_entry_points()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared entry points
    assert sorted(n for n, _, _ in V._SIGS) == names


def test_workspace_bytes_and_config_checks():
    cfg = V.config_of(W.naca(10.0))
    n = V.vplbm_workspace_bytes(cfg)
    # two FP32 population arrays (pitch 2048) dominate
    assert 2 * 9 * 1024 * 2048 * 4 < n < 2 * 9 * 1024 * 2048 * 4 + 64 << 20
    cfg16 = V.config_of(W.naca(10.0), dtype="bf16")
    assert V.vplbm_workspace_bytes(cfg16) < n

    bad = [
        dict(nx=2), dict(ny=2), dict(tau_plus=0.5), dict(eta=0.0), dict(dtype=9),
        dict(bc=(V.OUTLET_CONVECTIVE, V.INLET_BB, V.PERIODIC, V.PERIODIC)),
        dict(bc=(V.PERIODIC, V.INLET_BB, V.PERIODIC, V.PERIODIC)),
        dict(bc=(V.INLET_BB, V.OUTLET_CONVECTIVE, V.INLET_BB, V.SYMMETRY)),
        dict(bc=(V.INLET_BB, V.OUTLET_CONVECTIVE, V.PERIODIC, V.SYMMETRY)),
        dict(collision=V.TRT, lambda_trt=0.0), dict(sim_order=2), dict(sim_order=-1),
    ]
    for over in bad:
        c = V.config(**{**dict(nx=64, ny=32), **over})
        with pytest.raises(V.VplbmError) as e:
            V.vplbm_workspace_bytes(c)
        assert e.value.status == V.EINVAL
        assert V.vplbm_last_error(None)


def test_workloads_are_parameters_only():
    w = W.sedimentation()
    assert w.body.x_c == 37.0 and w.body.y_c == 1399.5
    reqs = W.serving_requests(256)
    assert len(reqs) == 256 and reqs[0].arrival == 0.0
    assert all(0 <= r.alpha_deg <= 20 for r in reqs)
    assert reqs == W.serving_requests(256)  # seeded
