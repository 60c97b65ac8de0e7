"""Seeded synthetic workloads shaped like the paper's cases.

Parameters only: lattice sizes, relaxation times, boundary kinds, body
geometry, step counts, and seeded random draws (test fields, request mixes).
Nothing here evaluates the method; both the CUDA library and the CPU oracle
take these numbers as inputs.

Relaxation times follow from Eq. tauvisco, nu = (tau - 1/2)/3, with
nu = U0 L / Re; they are stated as numbers here:
  disk channel, Re 20 on D = 20, U0 = 0.05: nu = 0.05   -> tau = 0.65
  NACA 0012, Re 1000 on C = 200, U0 = 0.05: nu = 0.01   -> tau+ = 0.53
  sedimentation (the paper's tau, Sec. 3.2):              tau+ = 0.6
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

# side kinds and options by name (mapped to the ABI values by the callers)
PERIODIC, INLET, OUTLET, SYMMETRY, NOSLIP = "periodic", "inlet", "outlet", "symmetry", "noslip"
OUTLET_FREE = "outlet_free"


@dataclass(frozen=True)
class Body:
    kind: str  # "none" | "disk" | "naca"
    length: float = 0.0
    thickness: float = 0.12
    x_c: float = 0.0
    y_c: float = 0.0
    angle_deg: float = 0.0
    pivot_chord_frac: float = 0.25
    moving: bool = False
    density_ratio: float = 1.0
    gravity: tuple = (0.0, 0.0)
    estimator: str = "mem"
    n_sim_points: int = 0

    @property
    def angle(self) -> float:
        return math.radians(self.angle_deg)


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    dtype: str  # "f64" | "f32" | "f16" | "bf16" | "f16sr" | "bf16sr" (stochastic rounding)
    collision: str  # "bgk" | "trt"
    tau_plus: float
    u_in: tuple
    bc: tuple  # x_lo, x_hi, y_lo, y_hi
    body: Body
    steps: int
    lambda_trt: float = 1.0 / 6.0
    eta: float = 1e-6  # Sec. 3: eta = 1e-6 for all cases
    forcing: str = "paper"
    body_force: tuple = (0.0, 0.0)
    sim_every: int = 1
    u_ref: tuple = (0.0, 0.0)  # stored offsets f - feq(1, u_ref); (0, 0): f - w

    @property
    def reference_length(self) -> float:
        return self.body.length

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def disk_channel() -> Workload:
    """Disk D = 20 at (64, 64) in a 256 x 128 channel, inlet u = 0.05, periodic
    top/bottom, Re 20, BGK, FP64, 2000 steps, MEM and SIM every step."""
    return Workload(
        name="disk-channel-256x128-f64", nx=256, ny=128, dtype="f64", collision="bgk",
        tau_plus=0.65, u_in=(0.05, 0.0), bc=(INLET, OUTLET, PERIODIC, PERIODIC),
        body=Body("disk", length=20.0, x_c=64.0, y_c=64.0), steps=2000)


def naca(alpha_deg: float = 0.0, dtype: str = "f32", nx: int = 2048, ny: int = 1024,
         chord: float | None = None, steps: int = 200_000, u_ref=None, u0: float = 0.05,
         tau_plus: float = 0.53) -> Workload:
    """NACA 0012 at Re 1000 on the chord (C = 200 on 2048 x 1024): leading edge
    at x = 4C, chord line half-way between the two middle rows, rotation about
    the quarter chord (nose up for alpha > 0), inlet u = 0.05, convective
    outlet, symmetry top and bottom, TRT with Lambda = 1/6 (Sec. 2.2, 3.1).
    Smaller grids scale the geometry with nx (C = nx * 200 / 2048).
    Reduced-precision forms store offsets from the free-stream equilibrium
    (u_ref = u_in) unless u_ref is given; (0, 0) gives the f - w offsets."""
    c = chord if chord is not None else nx * 200.0 / 2048.0
    if u_ref is None:
        u_ref = (0.0, 0.0) if dtype == "f64" else (u0, 0.0)
    return Workload(
        name=f"naca0012-{nx}x{ny}-a{alpha_deg:g}-{dtype}", nx=nx, ny=ny, dtype=dtype,
        collision="trt", tau_plus=tau_plus,
        u_in=(u0, 0.0), bc=(INLET, OUTLET, SYMMETRY, SYMMETRY),
        body=Body("naca", length=c, thickness=0.12, x_c=4.0 * c + 0.25 * c,
                  y_c=(ny - 1) / 2.0, angle_deg=alpha_deg),
        steps=steps, u_ref=tuple(u_ref))


NACA_ANGLES = (0.0, 5.0, 10.0, 15.0, 20.0)


def naca_paper(alpha_deg: float = 0.0, dtype: str = "f32", steps: int = 200_000) -> Workload:
    """The paper's own NACA 0012 case (Sec. 3.1): chord C = 278, U0 = 0.0599,
    tau = 0.55 (Re = U0 C / nu = 999), the leading edge 4C from the inlet and
    9C to the outlet (13C = 3614 columns), 7C high (1946 rows) with the chord
    line 3.5C from the bottom wall (mid-height, the wall half-way below row 0),
    rotation about the quarter chord, half-way bounce-back inlet, convective
    outlet, symmetry top and bottom, TRT Lambda = 1/6, 849 SIM points."""
    c = 278.0
    return naca(alpha_deg, dtype=dtype, nx=int(13 * c), ny=int(7 * c), chord=c, steps=steps,
                u0=0.0599, tau_plus=0.55)


# angles of attack of the paper's sweep (Sec. 3.1: 0 to 28 degrees; 7, 10, 24
# and 26 are the angles it discusses, 26 the stall)
PAPER_ANGLES = (0.0, 4.0, 7.0, 10.0, 12.0, 16.0, 20.0, 24.0, 26.0, 28.0)


# kinematic viscosity of the sedimentation cases (Sec. 3.2), cm^2/s: the
# paper prints mu = 0.1 g/(cm s) with rho = 1 g/cm^3, but with it the printed
# terminal Reynolds numbers would need drag coefficients below the Stokes-Oseen
# value of a cylinder (at Re 0.52 the buoyant weight of the disk balances
# Cd = 0.86, where Lamb's law alone gives about 18); nu = 0.01 cm^2/s (water)
# is consistent with them
NU_SEDIMENTATION = 0.01


def sedimentation(estimator: str = "mem", steps: int = 100_000) -> Workload:
    """Disk D = 50, rho_s/rho = 1.03, released at rest 0.75 D from the left wall
    and 4 D below the top of a closed 400 x 1600 box (no-slip on all sides),
    TRT tau = 0.6, FP32 lattice, FP64 rigid body driven by MEM or SIM.
    Gravity in lattice units from the paper's physical case (Sec. 3.2):
    D = 0.1 cm on 50 nodes gives dx = 0.002 cm; tau = 0.6 gives nu = 1/30 in
    lattice units, so with nu = 0.01 cm^2/s dt = (1/30) dx^2 / 0.01 =
    1.3333e-5 s, and |g| = 980 cm/s^2 becomes 980 dt^2 / dx = 8.7111e-5."""
    d_lu, tau = 50.0, 0.6
    dx = 0.1 / d_lu
    dt = (1.0 / 30.0) * dx * dx / NU_SEDIMENTATION
    g_lu = 980.0 * dt * dt / dx
    return Workload(
        name=f"sedimentation-400x1600-{estimator}", nx=400, ny=1600, dtype="f32",
        collision="trt", tau_plus=tau, u_in=(0.0, 0.0), bc=(NOSLIP, NOSLIP, NOSLIP, NOSLIP),
        body=Body("disk", length=d_lu, x_c=-0.5 + 0.75 * d_lu, y_c=1599.5 - 4.0 * d_lu,
                  moving=True, density_ratio=1.03, gravity=(0.0, -g_lu), estimator=estimator),
        steps=steps)


# density ratios of the paper's sedimentation runs (Sec. 3.2); the third value
# is printed as a repeat of the first, read as 1.01 (between the terminal
# Reynolds numbers 1.03 and 8.33 it is listed with)
RHO_R_PAPER = (1.0015, 1.003, 1.01, 1.03)
RE_TERMINAL_PAPER = (0.52, 1.03, 3.23, 8.33)


def sedimentation_paper(density_ratio: float = 1.03, estimator: str = "sim",
                        steps: int = 1000, length_d: int = 60, width_d: int = 4) -> Workload:
    """The paper's own sedimentation case (Sec. 3.2): disk D = 26, TRT tau = 0.6,
    a channel width_d D wide and length_d D long with no-slip side walls, a
    zero-velocity inlet at the top and a free outlet at the bottom, the disk
    released at rest 0.75 D from the left wall and 4 D below the top.  The
    paper gives no width; 4 D is the width at which the terminal Reynolds
    numbers it prints for the two heavier disks are reproduced (within 5 % with
    MEM, 12 % with SIM; 6 D and 8 D give 30 % and more above them).  60 D is long enough for
    2 s of fall of the heaviest disk (about 17 D).  The fall
    runs along +x (the top is x_lo, the bottom x_hi, the left wall y_lo: the
    paper's frame turned by a quarter turn, which keeps the sense of rotation),
    so that the inlet and outlet sit on the x sides where the library has them.
    Gravity in lattice units: D = 0.1 cm on 26 nodes gives dx = 0.1/26 cm;
    nu = 1/30 in lattice units and 0.01 cm^2/s gives dt = (1/30) dx^2 / 0.01
    s, so |g| = 980 cm/s^2 becomes 980 dt^2 / dx."""
    d_lu, tau = 26.0, 0.6
    dx, dt = 0.1 / d_lu, sedimentation_paper_dt()
    g_lu = 980.0 * dt * dt / dx
    nx, ny = int(length_d * d_lu), int(width_d * d_lu)
    return Workload(
        name=f"sedimentation-paper-{nx}x{ny}-rho{density_ratio}-{estimator}", nx=nx, ny=ny,
        dtype="f32", collision="trt", tau_plus=tau, u_in=(0.0, 0.0),
        bc=(INLET, OUTLET_FREE, NOSLIP, NOSLIP),
        body=Body("disk", length=d_lu, x_c=-0.5 + 4.0 * d_lu, y_c=-0.5 + 0.75 * d_lu,
                  moving=True, density_ratio=density_ratio, gravity=(g_lu, 0.0),
                  estimator=estimator),
        steps=steps)


def sedimentation_paper_dt() -> float:
    """Physical seconds per lattice step of the paper's sedimentation case."""
    dx = 0.1 / 26.0
    return (1.0 / 30.0) * dx * dx / NU_SEDIMENTATION


SERVING_GRIDS = ((512, 256), (768, 384), (1024, 512), (1536, 768), (2048, 1024))


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start
    alpha_deg: float
    nx: int
    ny: int


def serving_requests(n: int = 256, rate: float = 1.0, seed: int = 2110) -> list:
    """Seeded mix of NACA 0012 solves: alpha ~ U[0, 20] degrees, grid drawn
    uniformly from SERVING_GRIDS, Poisson arrivals of the given rate (1/s)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    alphas = rng.uniform(0.0, 20.0, n)
    grids = rng.integers(0, len(SERVING_GRIDS), n)
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps) - gaps[0]
    return [Request(k, float(t[k]), float(alphas[k]), *SERVING_GRIDS[int(grids[k])])
            for k in range(n)]


# ---------------------------------------------------------------------------
# seeded random fields for tests
# ---------------------------------------------------------------------------
def random_field(seed: int, shape, lo: float = 0.01, hi: float = 0.2) -> np.ndarray:
    """Uniform random values in [lo, hi) (populations for streaming tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return lo + (hi - lo) * rng.random(shape)


def perturbation(seed: int, shape, amplitude: float) -> np.ndarray:
    """Multiplicative perturbation 1 + amplitude * U[-1, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1.0 + amplitude * (2.0 * rng.random(shape) - 1.0)
