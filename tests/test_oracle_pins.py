"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: the paper's own formula written
in another form (velocity set), a textbook identity (equilibrium and forcing
moments, Gauss circle counts), a closed-form solution (uniform flow, free
fall), an exact symmetry, or an independent library routine (numpy.roll).
"""
import math

import numpy as np
import pytest

import oracle as o

CS2 = 1.0 / 3.0


# --------------------------------------------------------------------------
# lattice and equilibrium (Sec. 2.2)
# --------------------------------------------------------------------------
def test_velocity_set_matches_paper_trig_formula():
    """c_a from the cos/sin expressions of the D2Q9 velocity set (Sec. 2.2)."""
    cx, cy, opp, w = o.lattice()
    for a in range(9):
        if a == 0:
            ref = (0.0, 0.0)
        elif a <= 4:
            ang = (a - 1) * math.pi / 2
            ref = (math.cos(ang), math.sin(ang))
        else:
            ang = (2 * a - 9) * math.pi / 4
            ref = (math.sqrt(2) * math.cos(ang), math.sqrt(2) * math.sin(ang))
        assert (cx[a], cy[a]) == (round(ref[0]), round(ref[1]))
        assert (cx[opp[a]], cy[opp[a]]) == (-cx[a], -cy[a])
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-17)


def test_weights_isotropy():
    """sum w = 1, sum w c = 0, sum w c c = cs2 I, odd third moments vanish."""
    cx, cy, _, w = o.lattice()
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * cx).sum()) < 1e-16 and abs((w * cy).sum()) < 1e-16
    assert abs((w * cx * cx).sum() - CS2) < 1e-15
    assert abs((w * cx * cy).sum()) < 1e-16
    assert abs((w * cx * cx * cx).sum()) < 1e-16


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    """Textbook moments of the second-order equilibrium:
    sum feq = rho, sum c feq = rho u, sum c c feq = rho cs2 I + rho u u."""
    rng = np.random.default_rng(seed)
    rho = 1 + 0.1 * rng.standard_normal()
    u = 0.1 * rng.standard_normal(2)
    cx, cy, _, _ = o.lattice()
    f = o.feq(rho, *u)
    assert abs(f.sum() - rho) < 1e-14
    assert abs((cx * f).sum() - rho * u[0]) < 1e-15
    assert abs((cy * f).sum() - rho * u[1]) < 1e-15
    assert abs((cx * cx * f).sum() - (rho * CS2 + rho * u[0] ** 2)) < 1e-14
    assert abs((cx * cy * f).sum() - rho * u[0] * u[1]) < 1e-15
    assert abs((cy * cy * f).sum() - (rho * CS2 + rho * u[1] ** 2)) < 1e-14


@pytest.mark.parametrize("seed", range(5))
def test_guo_forcing_moments(seed):
    """Guo et al. forcing: sum F = 0, sum c F = G, sum c c F = u G + G u."""
    rng = np.random.default_rng(100 + seed)
    u = 0.1 * rng.standard_normal(2)
    g = 1e-3 * rng.standard_normal(2)
    cx, cy, _, _ = o.lattice()
    F = o.guo(u[0], u[1], g[0], g[1])
    assert abs(F.sum()) < 1e-18
    assert abs((cx * F).sum() - g[0]) < 1e-18
    assert abs((cy * F).sum() - g[1]) < 1e-18
    assert abs((cx * cx * F).sum() - 2 * u[0] * g[0]) < 1e-18
    assert abs((cx * cy * F).sum() - (u[0] * g[1] + u[1] * g[0])) < 1e-18
    assert abs((cy * cy * F).sum() - 2 * u[1] * g[1]) < 1e-18


# --------------------------------------------------------------------------
# penalized velocity (Eqs. updatestep .. updatestepm) and collision (Eq. TRT)
# --------------------------------------------------------------------------
def _random_pops(rng):
    _, _, _, w = o.lattice()
    return w * (1 + 0.2 * rng.random(9))


@pytest.mark.parametrize("chi", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_penalized_velocity_solves_implicit_equation(chi, seed):
    """u of the oracle satisfies Eq. updatestep2 itself,
    rho u = sum c f - (1/2) rho (chi/eta)(u - u_s), and G = rho F with
    F = -(chi/eta)(u - u_s) (Eq. (1) sign); residuals at round-off."""
    rng = np.random.default_rng(seed)
    eta = 1e-6
    cfg = o.make_config(4, 4, eta=eta)
    us = 0.05 * rng.standard_normal(2)
    body = o.make_body(o.BODY_DISK, length=2, xg=0, yg=0, u=tuple(us))
    fl = _random_pops(rng)
    cx, cy, _, _ = o.lattice()
    rho, ux, uy, gx, gy = o.node_moments(cfg, body, fl, chi, 0, 0)
    jx, jy = (cx * fl).sum(), (cy * fl).sum()
    pen = chi / eta
    # Eq. updatestep with the total force density G
    assert abs(rho * ux - (jx + 0.5 * gx)) < 1e-15 * max(1, abs(gx))
    assert abs(rho * uy - (jy + 0.5 * gy)) < 1e-15 * max(1, abs(gy))
    # implicit Eq. updatestep2 residual, scaled by the stiffness chi/eta
    res = rho * ux - jx + 0.5 * rho * pen * (ux - us[0])
    assert abs(res) < 1e-9
    if chi:
        # the velocity is driven onto u_s (Sec. 2.2, last paragraph)
        assert abs(ux - us[0]) < 2 * eta * abs(jx / rho - us[0]) + 1e-16
        assert abs(uy - us[1]) < 2 * eta * abs(jy / rho - us[1]) + 1e-16
    else:
        assert abs(ux - jx / rho) < 1e-16 and abs(uy - jy / rho) < 1e-16
        assert gx == 0 and gy == 0


@pytest.mark.parametrize("seed", range(4))
def test_rearranged_penalization_matches_literal(seed):
    """Reading R3: the rearranged G equals the literal -rho chi/eta (u - u_s)
    (u from Eq. updatestepm) to the conditioning of the literal form."""
    rng = np.random.default_rng(seed)
    eta = 1e-6
    cfg = o.make_config(4, 4, eta=eta)
    us = 0.05 * rng.standard_normal(2)
    body = o.make_body(o.BODY_DISK, length=2, u=tuple(us))
    fl = _random_pops(rng)
    cx, cy, _, _ = o.lattice()
    rho, ux, uy, gx, gy = o.node_moments(cfg, body, fl, 1)
    lit = o.penalization_literal(rho, (cx * fl).sum(), (cy * fl).sum(), 1, eta, us[0], us[1])
    assert abs(lit[0] - ux) < 1e-16 and abs(lit[1] - uy) < 1e-16
    assert abs(lit[2] - gx) <= 1e-9 * abs(gx) + 1e-12
    assert abs(lit[3] - gy) <= 1e-9 * abs(gy) + 1e-12


@pytest.mark.parametrize("coll,forcing", [(o.BGK, 0), (o.TRT, o.FORCING_PAPER), (o.TRT, o.FORCING_SPLIT)])
def test_collision_conserves_mass_and_adds_momentum(coll, forcing):
    """Mass is conserved; the momentum gained per collision is G times
    1 (BGK, split) or 1 + 1/(2 tau-) - 1/(2 tau+) (Eq. TRT read literally,
    where (1 - 1/(2 tau+)) multiplies all of F_a)."""
    rng = np.random.default_rng(7)
    tp, lam = 0.53, 1.0 / 6.0
    cfg = o.make_config(4, 4, collision=coll, forcing=forcing, tau_plus=tp, lambda_trt=lam)
    cx, cy, _, _ = o.lattice()
    fl = _random_pops(rng)
    g = 1e-3 * rng.standard_normal(2)
    rho = fl.sum()
    jx, jy = (cx * fl).sum(), (cy * fl).sum()
    ux, uy = (jx + g[0] / 2) / rho, (jy + g[1] / 2) / rho
    ft = o.collide_node(cfg, fl, rho, ux, uy, g[0], g[1])
    tm = lam / (tp - 0.5) + 0.5
    kappa = 1.0 if (coll == o.BGK or forcing == o.FORCING_SPLIT) else 1 + 1 / (2 * tm) - 1 / (2 * tp)
    assert abs(ft.sum() - rho) < 1e-15
    assert abs((cx * ft).sum() - (jx + kappa * g[0])) < 1e-15
    assert abs((cy * ft).sum() - (jy + kappa * g[1])) < 1e-15


def test_trt_reduces_to_bgk():
    """TRT with tau- = tau+ (Lambda = (tau - 1/2)^2) is BGK (Eq. TRT vs the BGK operator)."""
    rng = np.random.default_rng(3)
    tau = 0.7
    bgk = o.make_config(4, 4, collision=o.BGK, tau_plus=tau)
    trt = o.make_config(4, 4, collision=o.TRT, tau_plus=tau, lambda_trt=(tau - 0.5) ** 2,
                        forcing=o.FORCING_PAPER)
    for _ in range(5):
        fl = _random_pops(rng)
        args = (fl.sum(), 0.03, -0.02, 1e-4, 2e-4)
        np.testing.assert_allclose(o.collide_node(trt, fl, *args), o.collide_node(bgk, fl, *args),
                                   rtol=0, atol=1e-16)


def test_bgk_tau_one_gives_equilibrium_plus_half_force():
    """BGK at tau = 1: f~ = feq + F/2 (special case of the BGK operator)."""
    rng = np.random.default_rng(4)
    cfg = o.make_config(4, 4, collision=o.BGK, tau_plus=1.0)
    fl = _random_pops(rng)
    rho, u, g = fl.sum(), (0.02, 0.01), (1e-4, -3e-4)
    ft = o.collide_node(cfg, fl, rho, *u, *g)
    np.testing.assert_allclose(ft, o.feq(rho, *u) + 0.5 * o.guo(*u, *g), rtol=0, atol=1e-16)


def test_bgk_second_moment_relaxation():
    """BGK relaxes the non-equilibrium momentum flux by (1 - 1/tau) and adds
    (1 - 1/(2 tau))(u G + G u) (moments of the BGK+Guo operator)."""
    rng = np.random.default_rng(5)
    tau = 0.8
    cfg = o.make_config(4, 4, collision=o.BGK, tau_plus=tau)
    cx, cy, _, _ = o.lattice()
    fl = _random_pops(rng)
    u, g = (0.02, 0.01), (1e-4, -3e-4)
    rho = fl.sum()
    ft = o.collide_node(cfg, fl, rho, *u, *g)
    fe = o.feq(rho, *u)
    for ax, bx, uv in ((cx, cx, 2 * u[0] * g[0]), (cx, cy, u[0] * g[1] + u[1] * g[0])):
        pi_neq = (ax * bx * (fl - fe)).sum()
        expect = (ax * bx * fe).sum() + (1 - 1 / tau) * pi_neq + (1 - 1 / (2 * tau)) * uv
        assert abs((ax * bx * ft).sum() - expect) < 1e-15


# --------------------------------------------------------------------------
# streaming and boundaries (Eq. eqBd, Sec. 3.1, 3.2)
# --------------------------------------------------------------------------
def test_periodic_streaming_is_numpy_roll():
    """Fully periodic streaming is f_a(x + c_a) = f~_a(x): numpy.roll, bit-exact."""
    rng = np.random.default_rng(11)
    nx, ny = 13, 7
    cfg = o.make_config(nx, ny)
    cx, cy, _, _ = o.lattice()
    ft = rng.random((9, ny, nx))
    out = o.stream(cfg, ft, ft)
    for a in range(9):
        assert np.array_equal(out[a], np.roll(ft[a], (cy[a], cx[a]), axis=(0, 1)))


@pytest.mark.parametrize("bc", [
    (o.BC_PERIODIC, o.BC_PERIODIC, o.BC_NOSLIP, o.BC_NOSLIP),
    (o.BC_NOSLIP, o.BC_NOSLIP, o.BC_NOSLIP, o.BC_NOSLIP),
    (o.BC_PERIODIC, o.BC_PERIODIC, o.BC_SYMMETRY, o.BC_SYMMETRY),
    (o.BC_NOSLIP, o.BC_NOSLIP, o.BC_SYMMETRY, o.BC_NOSLIP),
])
def test_walls_stream_a_permutation(bc):
    """Bounce-back and specular reflection only move values: the streamed
    field is a permutation of the post-collision field (exact mass)."""
    rng = np.random.default_rng(12)
    nx, ny = 9, 6
    cfg = o.make_config(nx, ny, bc=bc)
    ft = rng.random((9, ny, nx))
    out = o.stream(cfg, ft, ft)
    assert np.array_equal(np.sort(out.ravel()), np.sort(ft.ravel()))


def test_symmetry_wall_equals_mirrored_periodic_domain():
    """Specular walls at y = -1/2 and y = NY - 1/2 give the same streaming as a
    periodic domain of height 2 NY holding the mirror image of the field."""
    rng = np.random.default_rng(13)
    nx, ny = 8, 5
    cx, cy, _, _ = o.lattice()
    mir = [0, 1, 4, 3, 2, 8, 7, 6, 5]  # c_y -> -c_y
    ft = rng.random((9, ny, nx))
    big = np.zeros((9, 2 * ny, nx))
    big[:, :ny] = ft
    for a in range(9):
        big[mir[a], ny:] = ft[a, ::-1]
    ref = o.stream(o.make_config(nx, 2 * ny), big, big)[:, :ny]
    out = o.stream(o.make_config(nx, ny, bc=(0, 0, o.BC_SYMMETRY, o.BC_SYMMETRY)), ft, ft)
    assert np.array_equal(out, ref)


def test_uniform_inflow_is_an_exact_steady_state():
    """f = feq(1, u_in) everywhere is a fixed point of inlet bounce-back
    (odd part of feq equals 2 w rho c.u / cs2), the convective outlet and the
    collision, so one step returns it to round-off."""
    nx, ny = 12, 6
    u = (0.05, 0.0)
    cfg = o.make_config(nx, ny, bc=(o.BC_INLET, o.BC_OUTLET, 0, 0), tau_plus=0.6, u_in=u,
                        collision=o.TRT)
    body = o.make_body()
    chi = np.zeros((ny, nx), np.uint8)
    f = o.init(cfg, body, chi)
    f0 = f.copy()
    o.run(cfg, body, f, chi, 3)
    np.testing.assert_allclose(f, f0, rtol=0, atol=2e-16)


def test_inlet_without_velocity_is_noslip_bounce_back():
    rng = np.random.default_rng(14)
    nx, ny = 6, 5
    ft = rng.random((9, ny, nx))
    a = o.stream(o.make_config(nx, ny, bc=(o.BC_INLET, o.BC_NOSLIP, 0, 0)), ft, ft)
    b = o.stream(o.make_config(nx, ny, bc=(o.BC_NOSLIP, o.BC_NOSLIP, 0, 0)), ft, ft)
    assert np.array_equal(a, b)


def test_convective_outlet_special_cases():
    """U_c = 0 keeps the previous outlet value; a field uniform in x is a fixed point."""
    rng = np.random.default_rng(15)
    nx, ny = 7, 4
    ft = rng.random((9, ny, nx))
    prev = rng.random((9, ny, nx))
    out = o.stream(o.make_config(nx, ny, bc=(o.BC_NOSLIP, o.BC_OUTLET, 0, 0)), ft, prev)
    for a in (3, 6, 7):
        assert np.array_equal(out[a, :, -1], prev[a, :, -1])
    col = rng.random((9, ny, 1))
    uni = np.repeat(col, nx, axis=2)
    cfg = o.make_config(nx, ny, bc=(o.BC_PERIODIC, o.BC_PERIODIC, 0, 0), u_in=(0.05, 0))
    ref = o.stream(cfg, uni, uni)
    cfg.bc[0], cfg.bc[1] = o.BC_NOSLIP, o.BC_OUTLET
    out = o.stream(cfg, uni, ref)
    for a in (3, 6, 7):
        np.testing.assert_allclose(out[a, :, -1], ref[a, :, -1], rtol=0, atol=4e-16)


def test_free_outlet_is_the_convective_limit():
    """The free outlet (reading R21) is the convective outlet as U_c grows
    without bound: equal to 1e-10 at U_c = 1e12 on random fields (with no-slip
    and periodic y sides, so that corners are covered); every population that
    does not enter through the outlet is streamed the same way; a field
    uniform in x is a fixed point."""
    rng = np.random.default_rng(21)
    nx, ny = 9, 5
    ft, prev = rng.random((9, ny, nx)), rng.random((9, ny, nx))
    for ys in (o.BC_NOSLIP, o.BC_PERIODIC):
        free = o.stream(o.make_config(nx, ny, bc=(o.BC_NOSLIP, o.BC_OUTLET_FREE, ys, ys)), ft, prev)
        conv = o.stream(o.make_config(nx, ny, bc=(o.BC_NOSLIP, o.BC_OUTLET, ys, ys),
                                      u_in=(1e12, 0.0)), ft, prev)
        assert np.abs(free - conv).max() <= 1e-10
        keep = np.ones_like(free, bool)
        keep[[3, 6, 7], :, -1] = False
        wall = o.stream(o.make_config(nx, ny, bc=(o.BC_NOSLIP, o.BC_NOSLIP, ys, ys)), ft, prev)
        assert np.array_equal(free[keep], wall[keep])
    uni = np.repeat(rng.random((9, ny, 1)), nx, axis=2)
    ref = o.stream(o.make_config(nx, ny, bc=(o.BC_PERIODIC, o.BC_PERIODIC, 0, 0)), uni, uni)
    out = o.stream(o.make_config(nx, ny, bc=(o.BC_NOSLIP, o.BC_OUTLET_FREE, 0, 0)), uni, uni)
    assert np.array_equal(out[[3, 6, 7], :, -1], ref[[3, 6, 7], :, -1])


# --------------------------------------------------------------------------
# whole steps: conservation and closed-form flows
# --------------------------------------------------------------------------
def test_mass_conserved_with_penalized_body():
    """Fully periodic box with a fixed penalized disk: total mass is conserved
    (sum_a F_a = 0 and streaming is a permutation)."""
    rng = np.random.default_rng(21)
    nx, ny = 24, 20
    cfg = o.make_config(nx, ny, collision=o.TRT, tau_plus=0.6)
    body = o.make_body(o.BODY_DISK, length=8, xg=11.3, yg=9.6)
    chi = o.raster(body, nx, ny)
    f = o.init(cfg, body, chi) * (1 + 0.01 * rng.random((9, ny, nx)))
    m0 = f.sum()
    o.run(cfg, body, f, chi, 50)
    assert abs(f.sum() - m0) < 1e-12 * m0


def test_quiescent_fluid_is_exact_and_force_free():
    """rho = 1, u = 0 around a fixed body: f stays feq to round-off, MEM = 0 (links
    pair up along each lattice line) and SIM = 0 (closed polygon)."""
    nx, ny = 40, 32
    cfg = o.make_config(nx, ny, collision=o.TRT, tau_plus=0.6)
    body = o.make_body(o.BODY_DISK, length=12, xg=19.5, yg=15.2)
    chi = o.raster(body, nx, ny)
    f = o.init(cfg, body, chi)
    f0 = f.copy()
    pts = o.sim_points(body)
    mh, sh, _, bad = o.run(cfg, body, f, chi, 5, sim_pts=pts)
    assert bad == 0
    np.testing.assert_allclose(f, f0, rtol=0, atol=2e-16)
    assert np.abs(mh).max() < 1e-15
    assert np.abs(sh[:, :2]).max() < 1e-13 and np.abs(sh[:, 2]).max() < 1e-12


def test_body_moving_with_the_flow_feels_no_force():
    """Uniform flow u0 and a body translating with u0: feq(1, u0) stays a fixed
    point (G = 0 in the solid) and the link terms of Eq. MMEL cancel in pairs."""
    nx, ny = 40, 30
    u0 = (0.04, -0.015)
    cfg = o.make_config(nx, ny, collision=o.TRT, tau_plus=0.6)
    body = o.make_body(o.BODY_DISK, length=10, xg=20.2, yg=14.7, u=u0)
    chi = o.raster(body, nx, ny)
    f = np.zeros((9, ny, nx))
    f[:] = o.feq(1.0, *u0)[:, None, None]
    f0 = f.copy()
    mh, _, _, _ = o.run(cfg, body, f, chi, 3)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-15)
    assert np.abs(mh[:, :2]).max() < 1e-14


def _poiseuille(nx, ny, g, tau, steps, chi=None, forcing=o.FORCING_SPLIT, lam=3.0 / 16.0,
                bc=(0, 0, o.BC_NOSLIP, o.BC_NOSLIP)):
    cfg = o.make_config(nx, ny, bc=bc, collision=o.TRT, forcing=forcing, tau_plus=tau,
                        lambda_trt=lam, body_force=(g, 0.0))
    body = o.make_body(o.BODY_NONE)
    if chi is None:
        chi = np.zeros((ny, nx), np.uint8)
    f = o.init(cfg, body, chi)
    mh, _, _, _ = o.run(cfg, body, f, chi, steps)
    return cfg, body, chi, f, mh


@pytest.mark.slow
def test_poiseuille_trt_magic_exact_parabola_and_stress():
    """Body-force driven channel with half-way bounce-back walls at y = -1/2 and
    y = NY - 1/2: TRT with Lambda = 3/16 reproduces u(y) = g (y + 1/2)(NY - 1/2 - y)/(2 nu)
    to round-off (a known TRT property).  The SIM stress sigma_xy equals
    rho nu u'(y) = (g/2)(NY - 1 - 2y) (Sec. 2.3.2 stress formula, tau = tau+)."""
    nx, ny, g, tau = 3, 12, 1e-5, 0.8
    nu = CS2 * (tau - 0.5)
    cfg, body, chi, f, _ = _poiseuille(nx, ny, g, tau, 6000)
    rho, ux, uy = o.fields(cfg, body, chi, f)
    y = np.arange(ny)
    exact = g * (y + 0.5) * (ny - 0.5 - y) / (2 * nu)
    np.testing.assert_allclose(ux[:, 1], exact, rtol=1e-9, atol=0)
    assert np.abs(uy).max() < 1e-9 * exact.max()
    for j in range(ny):
        sxy = o.stress(cfg, f[:, j, 1])[1]
        assert abs(sxy - 0.5 * g * (ny - 1 - 2 * j)) < 1e-9 * g * ny


@pytest.mark.slow
@pytest.mark.parametrize("forcing", [o.FORCING_SPLIT, o.FORCING_PAPER])
def test_mem_balances_body_force_between_penalized_slabs(forcing):
    """Channel bounded by penalized slabs (chi = 1 rows), fully periodic: at
    steady state the momentum leaving the fluid through the fluid-solid links
    (Eq. MMEL with u_Gamma = 0) balances what the collisions add to the fluid
    nodes, kappa * g * N_fluid, kappa = 1 (split) or
    1 + 1/(2 tau-) - 1/(2 tau+) (Eq. TRT read literally).  The profile is the
    parabola vanishing on the last solid nodes to O(1e-2): the penalized
    velocity is u_s on chi = 1 nodes (Eq. updatestepm), so the wall sits at
    most a fraction of a cell into the fluid."""
    nx, ny, s, g, tau, lam = 3, 20, 2, 1e-6, 0.8, 1.0 / 6.0
    chi = np.zeros((ny, nx), np.uint8)
    chi[:s] = 1
    cfg, body, chi, f, mh = _poiseuille(nx, ny, g, tau, 8000, chi=chi, forcing=forcing, lam=lam,
                                        bc=(0, 0, 0, 0))
    tm = lam / (tau - 0.5) + 0.5
    kappa = 1.0 if forcing == o.FORCING_SPLIT else 1 + 1 / (2 * tm) - 1 / (2 * tau)
    n_fluid = int((chi == 0).sum())
    assert abs(mh[-1, 0] - kappa * g * n_fluid) < 1e-6 * g * n_fluid
    assert abs(mh[-1, 1]) < 1e-14  # round-off of O(0.1) link terms
    if forcing == o.FORCING_SPLIT:
        rho, ux, _ = o.fields(cfg, body, chi, f)
        nu = CS2 * (tau - 0.5)
        y = np.arange(s, ny)
        exact = g * (y - (s - 1)) * (ny - y) / (2 * nu)
        err = np.abs(ux[s:, 1] - exact).max() / exact.max()
        assert err < 4e-2


# --------------------------------------------------------------------------
# geometry: mask (Eq. fcar) and SIM polygon
# --------------------------------------------------------------------------
def test_disk_mask_gauss_circle_counts():
    """Number of lattice nodes with x^2 + y^2 <= r^2 (Gauss circle problem,
    OEIS A000328 for r = 0..10)."""
    counts = [1, 5, 13, 29, 49, 81, 113, 149, 197, 253, 317]
    for r, n in enumerate(counts):
        b = o.make_body(o.BODY_DISK, length=2 * r, xg=15, yg=14)
        assert int(o.raster(b, 31, 29).sum()) == n


def test_naca_mask_is_mirror_symmetric_at_zero_angle():
    """Chord line at y = 511.5 (between two rows): chi(j) == chi(1023 - j) bit-exactly."""
    b = o.make_body(o.BODY_NACA, length=200, thickness=0.12, xg=850.0, yg=511.5, theta=0.0)
    chi = o.raster(b, 1100, 1024)
    assert np.array_equal(chi, chi[::-1])
    assert chi.sum() > 0


def test_naca_mask_area_and_nose_up_rotation():
    """Area of the NACA 00t section is 0.68508 t C^2 (integral of the
    thickness law); the lattice count agrees within the perimeter.  A positive
    angle lifts the leading edge above the pivot."""
    C, t = 200.0, 0.12
    area = 10 * t * (0.2969 * 2 / 3 - 0.1260 / 2 - 0.3516 / 3 + 0.2843 / 4 - 0.1015 / 5) * C * C
    for deg in (0, 7, 15):
        b = o.make_body(o.BODY_NACA, length=C, thickness=t, xg=300.0, yg=255.5,
                        theta=math.radians(deg))
        chi = o.raster(b, 600, 512)
        assert abs(chi.sum() - area) < 2.2 * C
        js, is_ = np.nonzero(chi)
        a = math.radians(deg)
        # leading edge 0.25 C ahead of the pivot, raised by 0.25 C sin a;
        # trailing edge 0.75 C behind it, lowered by 0.75 C sin a
        assert abs(js[is_ == is_.min()].mean() - (255.5 + 0.25 * C * math.sin(a))) < 2.0
        assert abs(is_.min() - (300.0 - 0.25 * C * math.cos(a))) < 2.0
        assert abs(js[is_ == is_.max()].mean() - (255.5 - 0.75 * C * math.sin(a))) < 2.0


def test_sim_polygon_closed_and_oriented():
    """The integration points form a closed polygon: sum S n = 0, perimeter
    2 N R sin(pi/N) for the disk, area from the divergence theorem
    (1/2) sum S x.n equal to the shoelace area and close to the analytic area."""
    r = 25.0
    b = o.make_body(o.BODY_DISK, length=2 * r, xg=10, yg=10)
    pts = o.sim_points(b)
    n = len(pts)
    assert n == math.ceil(2 * math.pi * r / 0.5)
    assert np.abs((pts[:, 4:5] * pts[:, 2:4]).sum(0)).max() < 1e-12
    assert abs(pts[:, 4].sum() - 2 * n * r * math.sin(math.pi / n)) < 1e-10
    area = 0.5 * (pts[:, 4] * (pts[:, 0] * pts[:, 2] + pts[:, 1] * pts[:, 3])).sum()
    assert abs(area - 0.5 * n * r * r * math.sin(2 * math.pi / n)) < 1e-9

    C, t = 200.0, 0.12
    b = o.make_body(o.BODY_NACA, length=C, thickness=t, theta=math.radians(10))
    pts = o.sim_points(b)
    assert len(pts) == 849
    assert np.abs((pts[:, 4:5] * pts[:, 2:4]).sum(0)).max() < 1e-10
    area = 0.5 * (pts[:, 4] * (pts[:, 0] * pts[:, 2] + pts[:, 1] * pts[:, 3])).sum()
    exact = 10 * t * (0.2969 * 2 / 3 - 0.1260 / 2 - 0.3516 / 3 + 0.2843 / 4 - 0.1015 / 5) * C * C
    assert abs(area - exact) < 2e-4 * exact
    # outward: normals point away from the chord line
    cen = pts[:, :2].mean(0)
    assert (((pts[:, :2] - cen) * pts[:, 2:4]).sum(1) > 0).mean() > 0.97


def test_sim_direction_rule():
    """argmax c_a.n/|c_a| with ties going to the lowest index."""
    s = math.sqrt(0.5)
    assert [o.sim_direction(*n) for n in [(1, 0), (0, 1), (-1, 0), (0, -1)]] == [1, 2, 3, 4]
    assert [o.sim_direction(*n) for n in [(s, s), (-s, s), (-s, -s), (s, -s)]] == [5, 6, 7, 8]


# --------------------------------------------------------------------------
# rigid body (Eqs. dep1, theta2)
# --------------------------------------------------------------------------
def test_free_fall_is_exact_for_trapezoid():
    """No fluid force: X_n = X_0 + a n^2 / 2 with a = (1 - 1/rho_r) g,
    and a constant torque gives theta_n = T n^2 / (2 I), I = m R^2 / 2, m = rho_r pi R^2."""
    R, rr = 5.0, 1.5
    b = o.make_body(o.BODY_DISK, length=2 * R, xg=10.0, yg=50.0, moving=1, density_ratio=rr,
                    gravity=(0.0, -1e-4))
    m = rr * math.pi * R * R
    inertia = 0.5 * m * R * R
    a = (1 - 1 / rr) * -1e-4
    T = 3e-3
    for n in range(1, 41):
        o.rigid_update(b, [0.0, 0.0, T])
        assert abs(b.yg - (50.0 + 0.5 * a * n * n)) < 1e-12
        assert abs(b.u[1] - a * n) < 1e-15
        assert abs(b.theta - 0.5 * (T / inertia) * n * n) < 1e-12
    b2 = o.make_body(o.BODY_DISK, length=2 * R, moving=1, density_ratio=rr)
    o.rigid_update(b2, [m * 2e-3, 0.0, 0.0])
    assert abs(b2.u[0] - 2e-3) < 1e-16


# --------------------------------------------------------------------------
# the disk case: symmetry and force sign
# --------------------------------------------------------------------------
def test_disk_channel_symmetry_and_drag_sign():
    """Disk on the mid-line of a periodic-in-y channel (inlet u = 0.05 in +x):
    both estimators give |Cl| <= 1e-10 and a positive drag."""
    nx, ny = 96, 48
    cfg = o.make_config(nx, ny, bc=(o.BC_INLET, o.BC_OUTLET, 0, 0), collision=o.BGK,
                        tau_plus=0.65, u_in=(0.05, 0.0))
    body = o.make_body(o.BODY_DISK, length=10, xg=24.0, yg=24.0)
    chi = o.raster(body, nx, ny)
    f = o.init(cfg, body, chi)
    mh, sh, _, bad = o.run(cfg, body, f, chi, 150, sim_pts=o.sim_points(body))
    assert bad == 0
    scale = 0.5 * 0.05 ** 2 * 10
    assert np.abs(mh[:, 1]).max() / scale < 1e-10
    assert np.abs(sh[:, 1]).max() / scale < 1e-10
    assert mh[-1, 0] > 0 and sh[-1, 0] > 0


def test_sim_of_a_linear_pressure_field_is_buoyancy():
    """Fluid at rest with rho = 1 + beta x: sigma = -rho cs2 I, and the SIM sum
    approaches -cs2 beta * area (divergence theorem) with the O(1/R) offset of
    the sampling nodes; fixes the sign, S_i and the outward normals."""
    nx, ny, R, beta = 80, 80, 20.0, 1e-4
    cfg = o.make_config(nx, ny, collision=o.TRT, tau_plus=0.6)
    body = o.make_body(o.BODY_DISK, length=2 * R, xg=40.0, yg=40.0)
    chi = o.raster(body, nx, ny)
    f = np.zeros((9, ny, nx))
    for i in range(nx):
        f[:, :, i] = o.feq(1 + beta * i, 0.0, 0.0)[:, None]
    out, nodes, missing = o.sim(cfg, body, chi, f, o.sim_points(body))
    assert missing == 0 and (nodes >= 0).all()
    expect = -CS2 * beta * math.pi * R * R
    assert abs(out[0] - expect) < 0.15 * abs(expect)
    assert abs(out[1]) < 1e-3 * abs(expect)


def test_torque_lever_arm_identity():
    """Moving the reference point by d changes both torques by -d x F (Eqs.
    fluidtorque and defFf), with the same links and sampling nodes."""
    nx, ny = 96, 48
    cfg = o.make_config(nx, ny, bc=(o.BC_INLET, o.BC_OUTLET, 0, 0), collision=o.TRT,
                        tau_plus=0.6, u_in=(0.05, 0.0))
    body = o.make_body(o.BODY_DISK, length=12, xg=30.3, yg=22.7)
    chi = o.raster(body, nx, ny)
    f = o.init(cfg, body, chi)
    pts = o.sim_points(body)
    o.run(cfg, body, f, chi, 40, sim_pts=pts)
    ft = o.collide(cfg, body, chi, f)
    d = (3.0, -2.0)
    moved = o.make_body(o.BODY_DISK, length=12, xg=30.3 + d[0], yg=22.7 + d[1])
    m0, m1 = o.mem(cfg, body, chi, ft), o.mem(cfg, moved, chi, ft)
    assert abs(m1[2] - (m0[2] - (d[0] * m0[1] - d[1] * m0[0]))) < 1e-13
    pts1 = pts.copy()
    pts1[:, 0] -= d[0]
    pts1[:, 1] -= d[1]
    s0, n0, _ = o.sim(cfg, body, chi, f, pts)
    s1, n1, _ = o.sim(cfg, moved, chi, f, pts1)
    assert np.array_equal(n0, n1)
    assert abs(s1[2] - (s0[2] - (d[0] * s0[1] - d[1] * s0[0]))) < 1e-12


def test_naca_zero_angle_lift_vanishes():
    """NACA 0012 at alpha = 0 centred between two rows of a channel with
    symmetry walls: mirror symmetry gives Cl = 0 for both estimators."""
    nx, ny, C = 200, 96, 40.0
    cfg = o.make_config(nx, ny, bc=(o.BC_INLET, o.BC_OUTLET, o.BC_SYMMETRY, o.BC_SYMMETRY),
                        collision=o.TRT, tau_plus=0.56, u_in=(0.05, 0.0))
    body = o.make_body(o.BODY_NACA, length=C, thickness=0.12, xg=60.0 + 0.25 * C, yg=47.5)
    chi = o.raster(body, nx, ny)
    f = o.init(cfg, body, chi)
    mh, sh, _, bad = o.run(cfg, body, f, chi, 60, sim_pts=o.sim_points(body))
    assert bad == 0
    scale = 0.5 * 0.05 ** 2 * C
    assert np.abs(mh[:, 1]).max() / scale < 1e-10
    assert np.abs(sh[:, 1]).max() / scale < 1e-10
    assert mh[-1, 0] > 0 and sh[-1, 0] > 0


# ---------------------------------------------------------------------------
# volume-integral force (Eq. Angotforce, reading R19)
# ---------------------------------------------------------------------------
def test_angot_force_closed_form_for_a_uniform_state():
    """f = feq(1, u0) on every node around a fixed disk: at a solid node
    j = u0, u_s = 0, so rho (chi/eta)(u - u_s) = (1/eta) u0 / (1 + 1/(2 eta)),
    and the force is the solid-node count times 2 u0 / (2 eta + 1); the
    torque is that node force crossed with the solid nodes' first moment."""
    nx, ny = 41, 33
    u0 = np.array([0.03, -0.02])
    for eta in (1e-6, 0.5, 3.0):
        cfg = o.make_config(nx, ny, collision=o.TRT, tau_plus=0.6, eta=eta)
        body = o.make_body(o.BODY_DISK, length=14, xg=20.3, yg=16.1)
        chi = o.raster(body, nx, ny)
        f = np.zeros((9, ny, nx))
        f[:] = o.feq(1.0, *u0)[:, None, None]
        n = int(chi.sum())
        per_node = 2.0 * u0 / (2.0 * eta + 1.0)
        F = o.angot(cfg, body, chi, f)
        np.testing.assert_allclose(F[:2], n * per_node, rtol=1e-12)
        jj, ii = np.nonzero(chi)
        rx, ry = (ii - 20.3).sum(), (jj - 16.1).sum()
        assert abs(F[2] - (rx * per_node[1] - ry * per_node[0])) <= 1e-12 * n * abs(per_node).max() * 10


def test_angot_force_vanishes_at_rest_and_with_the_body_moving_with_the_flow():
    nx, ny = 40, 30
    cfg = o.make_config(nx, ny, collision=o.TRT, tau_plus=0.6)
    body = o.make_body(o.BODY_DISK, length=10, xg=20.2, yg=14.7)
    chi = o.raster(body, nx, ny)
    f = o.init(cfg, body, chi)  # rho = 1, u = 0
    assert np.abs(o.angot(cfg, body, chi, f)).max() == 0.0
    u0 = (0.04, -0.015)
    moving = o.make_body(o.BODY_DISK, length=10, xg=20.2, yg=14.7, u=u0)
    f[:] = o.feq(1.0, *u0)[:, None, None]
    # round-off of j - rho u_s in each solid node (~1e-17), times about 2 per
    # node and lever arms of a few nodes
    assert np.abs(o.angot(cfg, moving, chi, f)).max() < 1e-13


# ---------------------------------------------------------------------------
# first-order SIM (reading R20)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gdir", [(1, 0), (0, 1), (1, 1), (-1, 1)])
def test_first_order_sim_is_exact_for_a_stress_linear_along_the_ray(gdir):
    """Fluid at rest with rho = 1 + beta (g.x): sigma = -rho/3 I is linear.
    For every point whose sampling direction c is parallel to g, the
    first-order stress equals the exact -rho(x_i)/3 (the field does not vary
    across the ray), while the zeroth-order copy misses it by the distance
    from the point to the sampled node."""
    nx, ny, R, beta = 80, 80, 15.3, 1e-3
    cfg = o.make_config(nx, ny, collision=o.TRT, tau_plus=0.6)
    body = o.make_body(o.BODY_DISK, length=2 * R, xg=40.2, yg=39.7)
    chi = o.raster(body, nx, ny)
    jj, ii = np.mgrid[0:ny, 0:nx]
    rho = 1 + beta * (gdir[0] * ii + gdir[1] * jj)
    f = np.stack([o.feq(1.0, 0.0, 0.0)[a] * rho for a in range(9)])
    pts = o.sim_points(body)
    _, _, miss1, sig1 = o.sim_order(cfg, body, chi, f, pts, 1)
    _, _, miss0, sig0 = o.sim_order(cfg, body, chi, f, pts, 0)
    assert miss1 == 0 and miss0 == 0
    cx, cy, _, _ = o.lattice()
    dirs = np.array([o.sim_direction(p[2], p[3]) for p in pts])
    sel = np.array([(cx[a], cy[a]) in (gdir, (-gdir[0], -gdir[1])) for a in dirs])
    assert sel.sum() >= 8
    x, y = 40.2 + pts[:, 0], 39.7 + pts[:, 1]
    exact = -(1 + beta * (gdir[0] * x + gdir[1] * y)) / 3.0
    np.testing.assert_allclose(sig1[sel, 0], exact[sel], rtol=0, atol=1e-15)
    np.testing.assert_allclose(sig1[sel, 2], exact[sel], rtol=0, atol=1e-15)
    assert np.abs(sig1[sel, 1]).max() < 1e-15
    assert np.abs(sig0[sel, 0] - exact[sel]).max() > 1e-5  # the copy is off by O(beta d)


def test_first_order_sim_falls_back_to_the_copy_without_a_second_fluid_node():
    """Points whose second node along the ray is solid or outside use the
    copy: on a lattice one node wider than the body, first and zeroth order
    coincide wherever the ray leaves the lattice after one node."""
    nx, ny = 24, 24
    cfg = o.make_config(nx, ny, collision=o.TRT, tau_plus=0.6)
    body = o.make_body(o.BODY_DISK, length=20.0, xg=11.5, yg=11.5)
    chi = o.raster(body, nx, ny)
    f = o.init(cfg, body, chi)
    rng = np.random.default_rng(3)
    f = f * (1 + 1e-3 * rng.random(f.shape))
    pts = o.sim_points(body)
    out0, n0, m0, s0 = o.sim_order(cfg, body, chi, f, pts, 0)
    out1, n1, m1, s1 = o.sim_order(cfg, body, chi, f, pts, 1)
    assert m0 == m1 and np.array_equal(n0, n1)
    cx, cy, _, _ = o.lattice()
    for k, p in enumerate(pts):
        if n0[k] < 0:
            continue
        a = o.sim_direction(p[2], p[3])
        qi, qj = n0[k] % nx, n0[k] // nx
        ni, nj = qi + cx[a], qj + cy[a]
        if not (0 <= ni < nx and 0 <= nj < ny) or chi[nj, ni]:
            np.testing.assert_array_equal(s1[k], s0[k])
