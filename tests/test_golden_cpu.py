"""The stored oracle values under tests/golden/ against what the mathematics
fixes, so that a corrupted or hand-edited file fails here before any GPU test
compares with it: the lift of the symmetric airfoil at zero incidence
vanishes, drag is positive and grows with incidence over the steady angles,
lift grows with incidence there, the window means are the means of their
blocks, and the storage envelopes grow as the formats lose precision."""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not written yet")
    return json.load(open(path))


def test_long_means_obey_symmetry_and_monotonicity():
    d = load("naca512_means.json")
    ang = d["angles"]
    for est in ("mem", "sim"):
        assert abs(ang["0"][f"cl_{est}"]) <= 1e-10  # mirror-symmetric body and lattice
        cds = [ang[a][f"cd_{est}"] for a in ("0", "5", "10", "15")]
        cls = [ang[a][f"cl_{est}"] for a in ("0", "5", "10", "15")]
        assert all(c > 0 for c in cds) and np.all(np.diff(cds) > 0)
        assert np.all(np.diff(cls) > 0)
    for a, r in ang.items():
        for k in ("cd_mem", "cl_mem", "cd_sim", "cl_sim"):
            assert len(r[f"{k}_blocks"]) * d["block"] == d["window"][1] - d["window"][0] + 1
            assert abs(np.mean(r[f"{k}_blocks"]) - r[k]) <= 1e-12 * max(1.0, abs(r[k]))


def test_storage_envelopes_grow_with_the_rounding_unit():
    d = load("storage_envelopes.json")
    for case in ("naca0-512", "naca10-512"):
        for offs in ("free-stream", "weights"):
            f32, f16, bf16 = (d["cases"][f"{case}/{offs}/{f}"] for f in ("f32", "f16", "bf16"))
            # velocity errors scale with the unit of the format: 2^-24, 2^-11, 2^-8
            assert max(f32["fields"][1:]) < max(f16["fields"][1:]) < max(bf16["fields"][1:])
            assert max(f32["fields"][1:]) < 1e-5


def test_serving_subset_is_the_seeded_mix():
    from paper_2110_00967_gb300 import workloads as W
    d = load("serving_subset.json")
    reqs = W.serving_requests(256)[:len(d["requests"])]
    for r, g in zip(reqs, d["requests"]):
        assert (r.rid, r.nx, r.ny) == (g["rid"], g["nx"], g["ny"])
        assert r.alpha_deg == g["alpha_deg"]
        assert g["cd_mem"] > 0 and g["cd_sim"] > 0
        assert g["cl_mem"] * g["alpha_deg"] >= 0  # lift follows the incidence


def test_stochastic_storage_envelopes_are_ordered_by_format():
    """Stochastic rounding to a format moves the oracle by the same order as
    rounding to nearest in that format: FP16 (unit 2^-11) well below BF16
    (2^-8), and both far above FP32."""
    d = load("storage_envelopes.json")
    for case in ("naca0-512", "naca10-512"):
        for offs in ("free-stream", "weights"):
            c = {f: d["cases"][f"{case}/{offs}/{f}"] for f in ("f32", "f16", "f16sr", "bf16sr")}
            u = {f: max(v["fields"][1:]) for f, v in c.items()}
            assert u["f32"] < u["f16sr"] < u["bf16sr"]
            assert 0.25 * u["f16"] <= u["f16sr"] <= 4 * u["f16"]


def test_sedimentation_trajectory_is_a_settling_fall():
    """The stored trajectories of the disk in the closed box: it starts from
    rest and falls (v < 0 along y) ever faster over the first samples, never
    faster than free fall with buoyancy and no drag, ((1 - 1/rho_r) g t);
    the fluid force opposes the fall (F_y > 0); the positions are the
    trapezoid integral of the sampled velocities; MEM and SIM, two estimates
    of the same force, give fall displacements within 5 % of each other."""
    from paper_2110_00967_gb300 import workloads as W
    d = load("sedimentation_trajectory.json")
    every = d["every"]
    falls = {}
    for est, c in d["cases"].items():
        w = W.sedimentation(est)
        b, f = np.array(c["body"]), np.array(c["force"])
        g = w.body.gravity[1]
        t = every * np.arange(1, len(b) + 1)
        v = b[:, 4]
        assert np.all(v < 0) and np.all(np.diff(v[:10]) < 0)
        assert np.all(np.abs(v) < (1 - 1 / w.body.density_ratio) * abs(g) * t)
        assert np.all(f[5:, 1] > 0)
        # y(t_k) - y0 against the trapezoid integral of v through the samples
        # (v = 0 at t = 0); the sampling error is far below 1 % of the fall
        y = b[:, 1] - w.body.y_c
        integral = np.concatenate(([0.5 * every * v[0]],
                                   0.5 * every * v[0] + np.cumsum(0.5 * every * (v[1:] + v[:-1]))))
        assert np.all(np.abs(y[10:] - integral[10:]) <= 0.01 * np.abs(y[10:]))
        falls[est] = -y[-1]
    assert abs(falls["mem"] - falls["sim"]) <= 0.05 * falls["mem"]


def test_naca2048_run_is_a_lifting_airfoil_in_a_low_mach_stream():
    """The stored 4000-step run of the 2048 x 1024 airfoil at 20 degrees:
    the sampled nodes are the seeded draw the file names; the stream stays at
    low Mach number (|u| well below the lattice sound speed 1/sqrt(3), rho
    within 5 % of 1); drag and lift are positive at a positive angle of
    attack, lift above drag, in the mean over the second half of the run
    (acoustic waves of the impulsive start still cross the lattice, and the
    force of a single step can change sign); MEM and SIM, two estimates of
    one force, agree within 5 % in that mean."""
    d = load("naca2048_run.json")
    n = len(d["nodes"])
    idx = np.random.Generator(np.random.PCG64(d["seed"])).integers(0, 2048 * 1024, n)
    assert np.array_equal(idx, np.array(d["nodes"]))
    rho, ux, uy = (np.array(d[k]) for k in ("rho", "ux", "uy"))
    assert np.abs(rho - 1).max() < 0.05 and np.hypot(ux, uy).max() < 0.2
    mem, sim = np.array(d["mem"]), np.array(d["sim"])
    assert len(mem) == len(sim) == d["steps"] // d["every"]
    late = slice(len(mem) // 2, None)
    fm, fs = mem[late, :2].mean(axis=0), sim[late, :2].mean(axis=0)
    for f in (fm, fs):
        assert f[0] > 0 and f[1] > f[0]
    assert np.all(np.abs(fm - fs) <= 0.05 * np.abs(fs))


def test_stochastic_rounding_emulation_is_unbiased_and_picks_neighbours():
    """The oracle-side emulation of stochastic rounding that the storage
    envelopes use: each rounded value is one of the two 16-bit neighbours of
    the FP64 value (equal to it when representable), and the mean of many
    roundings of one value is the value (unbiased), for FP16 (normal and
    subnormal) and BF16, both signs."""
    import importlib.util
    path = os.path.join(GOLDEN, "make_storage_envelopes.py")
    spec = importlib.util.spec_from_file_location("make_storage_envelopes", path)
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    m.RNG = np.random.Generator(np.random.PCG64(7))
    n = 200_000
    for fmt, vals in (("f16sr", (1.0 + 0.3 * 2 ** -10, -0.75 - 0.71 * 2 ** -11, 0.4 * 2 ** -24,
                                 3.0e-6, 0.25)),
                      ("bf16sr", (1.0 + 0.3 * 2 ** -7, -0.011 - 0.6 * 2 ** -14, 0.5))):
        for v in vals:
            h = np.full(n, v)
            lo, hi = m.neighbours(h[:1], fmt[:-2])
            r = m.round_to(h, fmt)
            assert np.all((r == lo[0]) | (r == hi[0])), (fmt, v)
            gap = hi[0] - lo[0]
            if gap == 0:
                assert np.all(r == v)
                continue
            p = (v - lo[0]) / gap
            # the mean's error within five standard errors of a Bernoulli draw
            assert abs(r.mean() - v) <= 5 * gap * np.sqrt(p * (1 - p) / n) + 1e-300, (fmt, v)
