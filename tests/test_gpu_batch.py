"""Batches (vplbm_batch_*): several lattices stepped in lockstep on one stream,
runs of 32 steps replayed from one CUDA graph.  The lattices share no data, so
every member must end bit-identical -- state, force histories, sums, body --
to the same lattice stepped alone."""
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


def falling_disk(est):
    return W.Workload(name="fall", nx=48, ny=96, dtype="f64", collision="trt", tau_plus=0.6,
                      u_in=(0.0, 0.0), bc=("noslip",) * 4,
                      body=W.Body("disk", length=12.0, x_c=20.3, y_c=70.0, moving=True,
                                  density_ratio=1.5, gravity=(0.0, -6e-4), estimator=est),
                      steps=100)


MEMBERS = [
    lambda: (W.disk_channel(), {}),
    lambda: (W.naca(10.0, dtype="f32", nx=512, ny=256), {}),
    lambda: (W.naca(5.0, dtype="f16", nx=256, ny=128), {}),
    lambda: (falling_disk("sim"), {}),
]


def same_state(a, b, n):
    assert np.array_equal(a.get_f(), b.get_f())
    assert a.steps == b.steps == n
    for est in (V.MEM, V.SIM):
        try:
            ha = a.history(est, min(n, 64))
        except V.VplbmError:
            continue
        np.testing.assert_array_equal(ha, b.history(est, min(n, 64)))
    sa, na = a.sums()
    sb, nb = b.sums()
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(na, nb)
    np.testing.assert_array_equal(a.get_body(), b.get_body())
    assert np.array_equal(a.get_mask(), b.get_mask())


def test_batch_equals_each_lattice_alone():
    ws = [m() for m in MEMBERS]
    alone = [lattice(w, **o) for w, o in ws]
    batched = [lattice(w, **o) for w, o in ws]
    batch = V.Batch(batched)
    for n in (1, 69, 32, 3):  # the pre step, graph runs, an odd level, single steps
        batch.step(n)
        for lat in alone:
            lat.step(n)
    total = 105
    for a, b in zip(alone, batched):
        same_state(a, b, total)
    # the same kernels ran, whether from the batch graph or one by one
    assert batch.launches == sum(l.launches for l in alone)
    batch.close()


def test_batch_with_sparse_sim_steps_one_by_one():
    w = W.naca(15.0, dtype="f32", nx=256, ny=128)
    a, b = lattice(w, sim_every=3), lattice(w, sim_every=3)
    c, d = lattice(W.disk_channel()), lattice(W.disk_channel())
    batch = V.Batch([b, d])
    batch.step(70)
    a.step(70)
    c.step(70)
    same_state(a, b, 70)
    same_state(c, d, 70)


def test_set_body_between_batch_steps_is_seen():
    w0 = W.naca(0.0, dtype="f32", nx=256, ny=128)
    w1 = W.naca(12.0, dtype="f32", nx=256, ny=128)
    a, b = lattice(w0), lattice(w0)
    other_a, other_b = lattice(W.disk_channel()), lattice(W.disk_channel())
    batch = V.Batch([b, other_b])
    batch.step(65)
    a.step(65)
    other_a.step(65)
    for lat in (a, b):
        lat.set_body(V.body_of(w1))  # restarts the solve around the new body
    batch.step(66)
    a.step(66)
    other_a.step(66)
    same_state(a, b, 66)
    same_state(other_a, other_b, 131)


def test_batch_on_a_separate_stream_is_ordered():
    import torch
    w = W.naca(8.0, dtype="f32", nx=256, ny=128)
    a, b = lattice(w), lattice(w)
    s = torch.cuda.Stream()
    batch = V.Batch([b], stream=s)
    batch.step(40)
    a.step(40)
    # b's own stream (the default one) reads after the batch's steps
    same_state(a, b, 40)


def test_batch_errors():
    w = W.naca(0.0, nx=256, ny=128)
    lat = lattice(w)
    with pytest.raises(V.VplbmError) as e:
        V.vplbm_batch_create([], 0)
    assert e.value.status == V.EINVAL
    with pytest.raises(V.VplbmError) as e:
        V.vplbm_batch_create([lat.ctx, lat.ctx], 0)
    assert e.value.status == V.EINVAL and "repeats" in V.vplbm_last_error(None)
    bare = V.Lattice(V.config_of(w))  # no body placed
    batch = V.Batch([lat, bare])
    with pytest.raises(V.VplbmError) as e:
        batch.step(1)
    assert e.value.status == V.ESTATE
    assert lat.steps == 0  # nothing was queued
    with pytest.raises(V.VplbmError) as e:
        V.vplbm_batch_step(batch.handle, -1)
    assert e.value.status == V.EINVAL
    batch.close()
    V.vplbm_batch_destroy(None)


@pytest.mark.parametrize("lengths", [(1, 20, 7, 45), (2, 5, 20), (1, 1, 63, 64)])
def test_runs_of_any_length_equal_single_steps(lengths):
    """Runs of any length, from either buffer, are replayed from the graphs of
    1, 2, 4, ..., 32 steps: a lattice and a batch stepped in those runs end
    bit-identical to a lattice stepped one step per call."""
    w = W.naca(7.0, dtype="f32", nx=256, ny=128)
    runs, ref = lattice(w), lattice(w)
    member, other = lattice(w), lattice(W.disk_channel())
    other_ref = lattice(W.disk_channel())
    batch = V.Batch([member, other])
    for n in lengths:
        runs.step(n)
        batch.step(n)
    total = sum(lengths)
    for _ in range(total):
        ref.step(1)
        other_ref.step(1)
    same_state(ref, runs, total)
    same_state(ref, member, total)
    same_state(other_ref, other, total)
    batch.close()


def test_prepared_lengths_replay_one_graph_and_change_nothing():
    """vplbm_prepare / vplbm_batch_prepare capture the graph of a 20-step run:
    the run then replays one graph per lattice (2 * 20 + 1 launches instead of
    the 42 of 16 + 4), and the lattices end bit-identical to unprepared ones
    stepped the same way, for a lattice alone and in a batch."""
    w = W.naca(7.0, dtype="f32", nx=256, ny=128)
    plain, prepared = lattice(w), lattice(w)
    for lat in (plain, prepared):
        lat.step(1)  # the first step (pre-collision state)
    prepared.prepare(20)
    l0, l1 = plain.launches, prepared.launches
    plain.step(20)
    prepared.step(20)
    assert plain.launches - l0 == (2 * 16 + 1) + (2 * 4 + 1)
    assert prepared.launches - l1 == 2 * 20 + 1
    same_state(plain, prepared, 21)
    # in a batch, and across a change of the bulk kernel's launch form
    members = [lattice(w), lattice(W.disk_channel())]
    alone = [lattice(w), lattice(W.disk_channel())]
    batch = V.Batch(members)
    batch.step(1)
    batch.prepare(20)
    for m in members:
        m.bulk_variant = 1  # drops the graphs; the prepared length is captured again
    batch.step(52)  # 32 + 20
    for a in alone:
        a.bulk_variant = 1
        a.step(53)
    for a, m in zip(alone, members):
        same_state(a, m, 53)
    batch.close()


def test_prepared_batch_call_is_one_graph_launch_and_changes_nothing():
    """After vplbm_batch_prepare(20) a batch call of 20 steps replays one
    graph holding every lattice's steps (from the current buffers, or from the
    other ones after an odd count); calls of other lengths, and calls after a
    member's launch form changed, take the per-lattice path.  Every lattice
    (FP32 and FP16-stochastic airfoils, a falling disk) ends bit-identical,
    forces, sums and body included, to the same lattice stepped alone."""
    works = [W.naca(7.0, dtype="f32", nx=256, ny=128), W.naca(3.0, dtype="f16sr", nx=384, ny=192),
             W.sedimentation("sim", steps=100)]
    members = [lattice(w) for w in works]
    alone = [lattice(w) for w in works]
    batch = V.Batch(members)
    batch.step(1)
    batch.prepare(20)
    counts = []
    for n in (20, 20, 5, 20, 3, 20):
        l0 = batch.launches
        batch.step(n)
        counts.append(batch.launches - l0)
    members[0].bulk_variant = 2  # the batch graph goes stale: per-lattice path
    batch.step(20)
    batch.close()
    total = 1 + 20 + 20 + 5 + 20 + 3 + 20 + 20
    for w, a in zip(works, alone):
        a.step(1 + 20 + 20 + 5 + 20 + 3 + 20)
    alone[0].bulk_variant = 2
    for a in alone:
        a.step(20)
    for a, m in zip(alone, members):
        same_state(a, m, total)
        np.testing.assert_array_equal(a.get_body(), m.get_body())
        np.testing.assert_array_equal(a.get_mask(), m.get_mask())
    # fixed bodies: 2 launches per step + 1 finalize; the falling disk adds
    # one mask launch per graph
    assert counts[0] == 2 * 20 * 3 + 3 + 1


@pytest.mark.parametrize("dtype", ["f32", "f16sr"])
def test_placing_the_body_again_restarts_the_solve_exactly(dtype):
    """vplbm_set_body on a lattice that has stepped: with the same body (its
    step graphs kept) and with another angle (graphs captured again), the
    lattice then steps exactly as a fresh lattice with that body does."""
    w5, w7 = (W.naca(a, dtype=dtype, nx=256, ny=128) for a in (5.0, 7.0))
    again, other, fresh5, fresh7 = lattice(w5), lattice(w5), lattice(w5), lattice(w7)
    for lat in (again, other):
        lat.step(37)
    again.set_body(V.body_of(w5))
    other.set_body(V.body_of(w7))
    for lat in (again, other, fresh5, fresh7):
        lat.step(45)
    same_state(again, fresh5, 45)
    same_state(other, fresh7, 45)


def test_batch_on_its_own_stream_orders_the_lattices_streams():
    """Lattices created on streams of their own, batched on a third stream:
    work queued on a lattice's stream before a batch call runs before it,
    and work queued there after the call runs after it (the batch call is a
    prepared one-graph launch and an unprepared one), so that the states and
    the host read-backs match lattices stepped alone."""
    import torch
    w = W.naca(9.0, dtype="f32", nx=256, ny=128)
    streams = [torch.cuda.Stream() for _ in range(2)]
    members = []
    for st in streams:
        lat = V.Lattice(V.config_of(w), stream=st)
        lat.set_body(V.body_of(w))
        members.append(lat)
    alone = lattice(w)
    batch_stream = torch.cuda.Stream()
    batch = V.Batch(members, stream=batch_stream)
    members[0].step(3)  # on its own stream, before the batch's calls
    batch.step(1)
    batch.prepare(16)
    batch.step(16)
    batch.step(7)
    for lat in members:
        lat.step(2)  # on its own stream, after the batch's calls
    batch.close()
    alone.step(3 + 1 + 16 + 7 + 2)
    same_state(alone, members[0], 29)
    other = lattice(w)
    other.step(1 + 16 + 7 + 2)
    same_state(other, members[1], 26)
