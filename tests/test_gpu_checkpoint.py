"""Checkpoint and restart (vplbm_state_bytes / vplbm_save_state /
vplbm_load_state): a lattice restored from a snapshot continues bit for bit as
the saved one did -- populations, outlet column, mask, force histories,
running sums, step counter and the FP64 body state -- in FP32 and 16-bit
storage, with a fixed airfoil and with a sedimenting disk."""
import numpy as np
import pytest

from paper_2110_00967_gb300 import vplbm as V
from paper_2110_00967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    V.lib()
    yield


def lattice(w, **over):
    lat = V.Lattice(V.config_of(w, **over))
    lat.set_body(V.body_of(w))
    return lat


def record(lat, n):
    rec = {"f": lat.get_f(), "mask": lat.get_mask(), "body": lat.get_body(), "steps": lat.steps}
    for est in (V.MEM, V.SIM, V.ANGOT):
        rec[f"hist{est}"] = lat.history(est, n)
    rec["sums"] = lat.sums()
    return rec


def assert_same(a, b):
    assert a["steps"] == b["steps"]
    for k in ("f", "mask", "body", f"hist{V.MEM}", f"hist{V.SIM}", f"hist{V.ANGOT}"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    np.testing.assert_array_equal(a["sums"][0], b["sums"][0])
    np.testing.assert_array_equal(a["sums"][1], b["sums"][1])


CASES = {
    "naca-f16": lambda: W.naca(12.0, dtype="f16", nx=512, ny=256),
    "naca-f32": lambda: W.naca(12.0, dtype="f32", nx=512, ny=256),
    # stochastic rounding: the snapshot carries the rounding counter
    "naca-f16sr": lambda: W.naca(12.0, dtype="f16sr", nx=512, ny=256),
    # a disk of the sedimentation box's proportions falling in a closed box,
    # rigid body driven by SIM; chi re-rasterised every step
    "fall-f32": lambda: W.Workload(
        name="fall", nx=96, ny=192, dtype="f32", collision="trt", tau_plus=0.6, u_in=(0.0, 0.0),
        bc=("noslip",) * 4,
        body=W.Body("disk", length=16.0, x_c=12.5, y_c=150.0, moving=True, density_ratio=1.5,
                    gravity=(0.0, -6e-4), estimator="sim"), steps=0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_restore_continues_bit_for_bit(case):
    w = CASES[case]()
    lat = lattice(w, history_len=512)
    lat.step(500)
    snap = lat.save_state()
    assert snap.nbytes == V.vplbm_state_bytes(lat.ctx)
    lat.step(500)
    a = record(lat, 500)
    # back to step 500 in the same lattice
    lat.load_state(snap)
    assert lat.steps == 500
    lat.step(500)
    assert_same(a, record(lat, 500))
    # and in a fresh lattice of the same configuration (another workspace)
    fresh = V.Lattice(V.config_of(w, history_len=512))
    fresh.load_state(snap)
    fresh.step(500)
    assert_same(a, record(fresh, 500))
    if w.body.moving:
        assert a["body"][1] < w.body.y_c - 1.0  # the disk fell


def test_restore_mid_run_in_a_batch():
    """A snapshot taken at an odd step, restored into a batch member: the batch
    continues it as the lattice alone does."""
    w = W.naca(5.0, dtype="f32", nx=256, ny=128)
    lat = lattice(w, history_len=512)
    lat.step(37)
    snap = lat.save_state()
    lat.step(100)
    member, other = lattice(w, history_len=512), lattice(W.disk_channel())
    member.load_state(snap)
    batch = V.Batch([member, other])
    batch.step(100)
    assert_same(record(lat, 137), record(member, 137))
    batch.close()


def test_snapshot_checks():
    w = W.naca(5.0, dtype="f32", nx=256, ny=128)
    lat = lattice(w)
    lat.step(3)
    snap = lat.save_state()
    other = V.Lattice(V.config_of(w, tau_plus=0.6))
    with pytest.raises(V.VplbmError) as e:
        other.load_state(snap)
    assert e.value.status == V.EINVAL
    bad = snap.copy()
    bad[0] ^= 0xFF
    with pytest.raises(V.VplbmError) as e:
        lat.load_state(bad)
    assert e.value.status == V.EINVAL
    with pytest.raises(V.VplbmError) as e:
        lat.load_state(snap[:100])
    assert e.value.status == V.EINVAL
    bare = V.Lattice(V.config_of(w))
    with pytest.raises(V.VplbmError) as e:
        V.vplbm_save_state(bare.ctx)
    assert e.value.status == V.ESTATE
