"""The SIM entry point that allocates nothing, checked against the FP64 oracle's
SIM and against the library's own SIM force.

vplbm_sim_force_static is for callers that cannot allocate device memory: an
application embedding this library whose allocator already holds the device
memory, or a latency-bound loop that cannot afford the device-wide
synchronisation of cudaMalloc / cudaFree.  Its scratch is one fixed array
inside the library, reused by every call.  Given the state of a lattice, it
must return the SIM force of Eq. defFf that the oracle computes on that same
state, and the force vplbm_step computed for it (vplbm_force_sim), within the
FP64 tolerance of the parity tests, on two calls in a row (the second call
sees what the first left in the array).
"""
import numpy as np
import pytest

import oracle as o
from paper_2110_00967_gb300 import vplbm as V
from paper_2110_00967_gb300 import workloads as W
from tests.helpers import oracle_body, oracle_config

pytestmark = pytest.mark.gpu


def test_static_sim_matches_the_oracle_and_the_step_sim_on_two_calls():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    w = W.disk_channel()  # FP64 lattice, the disk of the 256 x 128 channel
    cfg = V.config_of(w)
    lat = V.Lattice(cfg)
    lat.set_body(V.body_of(w))
    ocfg, obody = oracle_config(w), oracle_body(w)
    pts = o.sim_points(obody)  # the polygon vplbm_set_body builds
    stream = torch.cuda.current_stream().cuda_stream
    f = torch.empty((9, w.ny, w.nx), dtype=torch.float64, device="cuda")
    chi = torch.empty((w.ny, w.nx), dtype=torch.uint8, device="cuda")
    for steps in (40, 25):
        lat.step(steps)
        V.vplbm_get_f_dev(lat.ctx, f.data_ptr())  # pre-collision state of the next step
        V.vplbm_get_mask_dev(lat.ctx, chi.data_ptr())
        got = V.vplbm_sim_force_static(cfg, f.data_ptr(), chi.data_ptr(), pts,
                                       (w.body.x_c, w.body.y_c), stream)
        # the oracle's SIM (Eq. defFf, reading R6) on the same state
        ref_o, _, missing = o.sim(ocfg, obody, chi.cpu().numpy(), f.cpu().numpy(), pts)
        assert missing == 0
        assert np.abs(got - ref_o).max() <= 1e-12 * np.abs(ref_o).max() + 1e-14, (got, ref_o)
        lat.step(1)  # evaluates SIM on that same state
        ref = lat.force_sim()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max() + 1e-14, (got, ref)


def test_static_sim_rejects_what_it_does_not_evaluate():
    w = W.disk_channel()
    cfg = V.config_of(w)
    with pytest.raises(V.VplbmError) as e:
        V.vplbm_sim_force_static(cfg, 1, 1, np.zeros((4097, 5)), (0.0, 0.0), 0)
    assert e.value.status == V.EINVAL
    assert "4096" in V.vplbm_last_error(None)
    # the first-order stress is the step's option only
    with pytest.raises(V.VplbmError) as e:
        V.vplbm_sim_force_static(V.config_of(w, sim_order=1), 1, 1, np.zeros((8, 5)), (0.0, 0.0), 0)
    assert e.value.status == V.EINVAL
    # point rows must hold five values
    with pytest.raises(ValueError):
        V.vplbm_sim_force_static(cfg, 1, 1, np.zeros((8, 3)), (0.0, 0.0), 0)
