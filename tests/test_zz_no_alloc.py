"""The SIM entry point that allocates nothing, checked against the library's
own SIM force.

vplbm_sim_force_static is for callers that cannot allocate device memory: an
application embedding this library whose allocator already holds the device
memory, or a latency-bound loop that cannot afford the device-wide
synchronisation of cudaMalloc / cudaFree.  Its scratch is one fixed array
inside the library, reused by every call.  Given the state of a lattice, it
must return the SIM force that vplbm_step computed for that same state
(vplbm_force_sim), within the FP64 tolerance of the parity tests, on two
calls in a row (the second call sees what the first left in the array).
"""
import numpy as np
import pytest

import oracle as o
from paper_2110_00967_gb300 import vplbm as V
from paper_2110_00967_gb300 import workloads as W
from tests.helpers import oracle_body

pytestmark = pytest.mark.gpu


def test_static_sim_matches_the_step_sim_on_two_calls():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    w = W.disk_channel()  # FP64 lattice, the disk of the 256 x 128 channel
    cfg = V.config_of(w)
    lat = V.Lattice(cfg)
    lat.set_body(V.body_of(w))
    pts = o.sim_points(oracle_body(w))  # the polygon vplbm_set_body builds
    stream = torch.cuda.current_stream().cuda_stream
    f = torch.empty((9, w.ny, w.nx), dtype=torch.float64, device="cuda")
    chi = torch.empty((w.ny, w.nx), dtype=torch.uint8, device="cuda")
    for steps in (40, 25):
        lat.step(steps)
        V.vplbm_get_f(lat.ctx, f.data_ptr())  # pre-collision state of the next step
        V.vplbm_get_mask(lat.ctx, chi.data_ptr())
        got = V.vplbm_sim_force_static(cfg, f.data_ptr(), chi.data_ptr(), pts,
                                       (w.body.x_c, w.body.y_c), stream)
        lat.step(1)  # evaluates SIM on that same state
        ref = lat.force_sim()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max() + 1e-14, (got, ref)


def test_static_sim_rejects_more_points_than_its_array_holds():
    w = W.disk_channel()
    cfg = V.config_of(w)
    pts = np.zeros((4097, 5))
    with pytest.raises(V.VplbmError) as e:
        V.vplbm_sim_force_static(cfg, 1, 1, pts, (0.0, 0.0), 0)
    assert e.value.status == V.EINVAL
    assert "4096" in V.vplbm_last_error(None)
