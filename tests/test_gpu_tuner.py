"""The bulk kernel's launch forms and their tuner, through the C ABI: every
form gives the same populations bit for bit (storage forms, ragged lattice
sizes, with and without a body force), the tuner leaves the solution
unchanged, remembers its choice per lattice shape, and rejects bad input."""
import numpy as np
import pytest

from paper_2110_00967_gb300 import vplbm as V
from paper_2110_00967_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_VARIANTS = 3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    V.lib()
    yield


def lattice(w, variant=None, **over):
    lat = V.Lattice(V.config_of(w, **over))
    lat.set_body(V.body_of(w))
    if variant is not None:
        lat.bulk_variant = variant
    return lat


def ragged_naca(dtype, body_force=(0.0, 0.0)):
    # 300 x 131: a ragged last tile column and row counts that are not
    # multiples of the 2-, 4- and 8-row blocks
    w = W.naca(8.0, dtype=dtype, nx=300, ny=131, chord=40.0)
    return w.with_(body_force=body_force)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16", "bf16", "f16sr", "bf16sr"])
@pytest.mark.parametrize("force", [False, True])
def test_every_form_gives_the_same_populations(dtype, force):
    w = ragged_naca(dtype, body_force=(1e-6, -2e-6) if force else (0.0, 0.0))
    ref = None
    for v in range(N_VARIANTS):
        lat = lattice(w, variant=v)
        assert lat.bulk_variant == v
        lat.step(70)  # two 32-step graphs and single steps
        lat.check()
        f = lat.get_f()
        if ref is None:
            ref = f
        else:
            assert np.array_equal(f, ref), f"form {v} differs from form 0"


def tuning_steps(trials):
    """Steps a tuner call advances: three passes over the forms, each form 32
    untimed steps (one step graph) and `trials` timed ones."""
    return 3 * N_VARIANTS * (32 + trials)


def test_tuner_steps_are_ordinary_steps():
    """A lattice tuned between steps ends bit-identical (populations and the
    force histories) to one stepped the same number of steps; a batch stepped
    after a change of a member's form matches single steps."""
    w = W.naca(10.0, dtype="f16", nx=512, ny=256)
    tuned = lattice(w)
    tuned.step(20)
    v = tuned.autotune(4)
    assert 0 <= v < N_VARIANTS and tuned.bulk_variant == v
    tuned.step(20)
    n = 40 + tuning_steps(4)
    assert tuned.steps == n
    plain = lattice(w)
    plain.step(n)
    assert np.array_equal(tuned.get_f(), plain.get_f())
    np.testing.assert_array_equal(tuned.history(V.MEM, 40), plain.history(V.MEM, 40))
    np.testing.assert_array_equal(tuned.history(V.SIM, 40), plain.history(V.SIM, 40))
    ref = lattice(w)
    ref.step(40)
    a, b = lattice(w), lattice(w)
    batch = V.Batch([a, b])
    batch.step(10)
    a.bulk_variant = (a.bulk_variant + 1) % N_VARIANTS
    batch.step(30)
    batch.close()
    assert np.array_equal(a.get_f(), ref.get_f())
    assert np.array_equal(b.get_f(), ref.get_f())


def test_batch_tuner_steps_are_ordinary_steps():
    w = W.naca(5.0, dtype="bf16", nx=384, ny=192)
    lats = [lattice(w) for _ in range(3)]
    batch = V.Batch(lats)
    batch.step(10)
    v = batch.autotune(2)
    assert len(v) == 3 and len(set(v)) == 1 and 0 <= v[0] < N_VARIANTS
    assert all(l.bulk_variant == v[0] for l in lats)
    batch.step(20)
    batch.close()
    plain = lattice(w)
    plain.step(30 + tuning_steps(2))
    for l in lats:
        assert np.array_equal(l.get_f(), plain.get_f())


def test_batch_tuner_picks_a_form_per_size_class():
    """Members of one size and storage type share a form; two classes give
    each lattice 2 * 9 * (32 + trials) tuning steps, ordinary steps again."""
    works = [W.naca(5.0, dtype="f16", nx=384, ny=192), W.naca(12.0, dtype="f32", nx=256, ny=128),
             W.naca(7.0, dtype="f16", nx=384, ny=192)]
    lats = [lattice(w) for w in works]
    batch = V.Batch(lats)
    v = batch.autotune(2)
    assert v[0] == v[2] and all(0 <= x < N_VARIANTS for x in v)
    assert [l.bulk_variant for l in lats] == v
    batch.step(5)
    batch.close()
    for w, l in zip(works, lats):
        plain = lattice(w)
        plain.step(5 + 2 * tuning_steps(2))
        assert l.steps == plain.steps
        assert np.array_equal(l.get_f(), plain.get_f())


def test_tuner_rejects_bad_input():
    w = W.naca(0.0, dtype="f32", nx=256, ny=128)
    lat = V.Lattice(V.config_of(w))
    with pytest.raises(V.VplbmError) as e:
        lat.autotune(5)
    assert e.value.status == V.ESTATE
    lat.set_body(V.body_of(w))
    for bad in (-1, N_VARIANTS):
        with pytest.raises(V.VplbmError) as e:
            lat.bulk_variant = bad
        assert e.value.status == V.EINVAL
    with pytest.raises(V.VplbmError) as e:
        lat.autotune(0)
    assert e.value.status == V.EINVAL


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16", "f16sr", "bf16sr"])
@pytest.mark.parametrize("force", [False, True])
def test_bulk_and_special_kernels_update_a_node_alike(dtype, force):
    """A fluid node gets the same bits from the bulk kernel (any launch form)
    as from the special kernel: one step from the same pre-collision state,
    once pulled by the bulk kernel's tiles and once updated in place by the
    special kernel on every tile (the first step after a pre-collision state),
    ends bit-identical.  (FP32 and 16-bit storage share one FP32 arithmetic
    for fluid nodes, written for one node and for packed pairs.)"""
    w = W.Workload(name="box", nx=300, ny=37, dtype=dtype, collision="trt", tau_plus=0.6,
                   u_in=(0.04, 0.01), bc=("periodic",) * 4, body=W.Body("none"), steps=1,
                   body_force=(1e-6, -2e-6) if force else (0.0, 0.0), u_ref=(0.04, 0.0))
    ft = W.random_field(13, (9, w.ny, w.nx), lo=0.05, hi=0.15)
    for v in range(N_VARIANTS):
        pulled = lattice(w, variant=v)
        pulled.set_state(ft, ft, post_collision=True)  # the next step pulls (bulk kernel)
        pre = pulled.get_f()                           # the pre-collision state it pulls
        inplace = lattice(w, variant=v)
        inplace.set_state(pre, post_collision=False)   # the next step: special kernel, every tile
        pulled.step(1)
        inplace.step(1)
        assert np.array_equal(pulled.get_f(), inplace.get_f()), f"form {v}"


@pytest.mark.parametrize("dtype", ["f16sr", "bf16sr"])
def test_stochastic_rounding_is_reproducible_and_unbiased(dtype):
    """The stochastically rounded storage forms: two runs of the same lattice
    are bit-identical (the rounding bits come from a hash of the step count,
    node and population), they differ from rounding to nearest, and each
    stored value is one of the two 16-bit neighbours of the value rounding to
    nearest would store, at most one unit apart."""
    w = ragged_naca(dtype)
    a, b = lattice(w), lattice(w)
    rne = lattice(w.with_(dtype=dtype[:-2]))
    for lat in (a, b, rne):
        lat.step(40)
    fa, fb, fr = a.get_f(), b.get_f(), rne.get_f()
    assert np.array_equal(fa, fb)
    assert not np.array_equal(fa, fr)
    # one step from the same state: SR and RNE stores are neighbours
    st = a.get_f()
    for lat in (a, rne):
        lat.set_state(st, post_collision=False)
        lat.step(1)
    E = lat_E(w)
    ha, hr = a.get_f() - E, rne.get_f() - E
    # the larger of the two gaps next to the nearest value (at a power of two
    # the stochastic choice may be the neighbour in the larger binade)
    if dtype.startswith("f16"):
        h16 = hr.astype(np.float16)
        spacing = np.maximum(
            np.abs(np.nextafter(h16, np.float16(np.inf)).astype(np.float64) - hr),
            np.abs(np.nextafter(h16, np.float16(-np.inf)).astype(np.float64) - hr))
    else:
        m, e = np.frexp(hr)
        spacing = np.ldexp(1.0 / 256.0, e)
    # (f - E in FP64 carries up to an FP64 unit of E, about 1e-16)
    assert np.all(np.abs(ha - hr) <= spacing * (1 + 1e-6) + 1e-15)
    frac_diff = np.mean(ha != hr)
    assert 0.01 < frac_diff < 0.99, frac_diff


def lat_E(w):
    """E_a = feq_a(1, u_ref) of the workload, broadcast over the lattice."""
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    wt = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    ux, uy = (float(np.float32(v)) for v in w.u_ref)
    cu = cx * ux + cy * uy
    return (wt * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy)))[:, None, None]
