"""ctypes binding of the FP64 CPU oracle (vplbm_oracle.c).

Test infrastructure only.  Everything here follows the paper's Sec. 2 and 3;
the C file states, per function, which equation it implements.  Arrays are
numpy float64 / uint8, populations laid out f[a, j, i] (a = 0..8).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vplbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_INLET, BC_OUTLET, BC_SYMMETRY, BC_NOSLIP, BC_OUTLET_FREE = 0, 1, 2, 3, 4, 5
BGK, TRT = 0, 1
FORCING_PAPER, FORCING_SPLIT = 0, 1
BODY_NONE, BODY_DISK, BODY_NACA = 0, 1, 2
MEM, SIM = 0, 1


class Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc", C.c_int32 * 4),
        ("collision", C.c_int32), ("forcing", C.c_int32),
        ("tau_plus", C.c_double), ("lambda_trt", C.c_double), ("eta", C.c_double),
        ("u_in", C.c_double * 2), ("body_force", C.c_double * 2),
    ]


class Body(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("moving", C.c_int32), ("n_sim", C.c_int32), ("pad", C.c_int32),
        ("length", C.c_double), ("thickness", C.c_double),
        ("xg", C.c_double), ("yg", C.c_double), ("theta", C.c_double),
        ("pivot_frac", C.c_double), ("u", C.c_double * 2), ("omega", C.c_double),
        ("density_ratio", C.c_double), ("gravity", C.c_double * 2),
    ]


def make_config(nx, ny, bc=(BC_PERIODIC,) * 4, collision=BGK, forcing=FORCING_PAPER,
                tau_plus=0.8, lambda_trt=1.0 / 6.0, eta=1e-6, u_in=(0.0, 0.0),
                body_force=(0.0, 0.0)) -> Config:
    c = Config()
    c.nx, c.ny = nx, ny
    for k in range(4):
        c.bc[k] = bc[k]
    c.collision, c.forcing = collision, forcing
    c.tau_plus, c.lambda_trt, c.eta = tau_plus, lambda_trt, eta
    c.u_in[0], c.u_in[1] = u_in
    c.body_force[0], c.body_force[1] = body_force
    return c


def make_body(kind=BODY_NONE, length=0.0, thickness=0.12, xg=0.0, yg=0.0, theta=0.0,
              pivot_frac=0.25, u=(0.0, 0.0), omega=0.0, moving=0, density_ratio=1.0,
              gravity=(0.0, 0.0), n_sim=0) -> Body:
    b = Body()
    b.kind, b.moving, b.n_sim = kind, moving, n_sim
    b.length, b.thickness = length, thickness
    b.xg, b.yg, b.theta, b.pivot_frac = xg, yg, theta, pivot_frac
    b.u[0], b.u[1] = u
    b.omega, b.density_ratio = omega, density_ratio
    b.gravity[0], b.gravity[1] = gravity
    return b


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction into FMA, OpenMP rows)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-D_DEFAULT_SOURCE", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.POINTER
        dp = P(C.c_double)
        u8p = P(C.c_uint8)
        i32p = P(C.c_int32)
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_set_threads.restype = C.c_int
        L.orc_lattice.argtypes = [i32p, i32p, i32p, dp]
        L.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.orc_guo.argtypes = [C.c_double] * 4 + [dp]
        L.orc_raster.argtypes = [P(Body), C.c_int32, C.c_int32, u8p]
        L.orc_node_moments.argtypes = [P(Config), P(Body), dp, C.c_int32, C.c_int32, C.c_int32, dp]
        L.orc_penalization_literal.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int,
                                               C.c_double, C.c_double, C.c_double, dp]
        L.orc_collide_node.argtypes = [P(Config), dp] + [C.c_double] * 5 + [dp]
        L.orc_stress.argtypes = [P(Config), dp, dp]
        L.orc_init.argtypes = [P(Config), P(Body), u8p, dp]
        L.orc_collide.argtypes = [P(Config), P(Body), u8p, dp, dp]
        L.orc_fields.argtypes = [P(Config), P(Body), u8p, dp, dp, dp, dp]
        L.orc_stream.argtypes = [P(Config), dp, dp, dp]
        L.orc_mem.argtypes = [P(Config), P(Body), u8p, dp, dp]
        L.orc_angot.argtypes = [P(Config), P(Body), u8p, dp, dp]
        L.orc_sim_order.argtypes = [P(Config), P(Body), u8p, dp, C.c_int32, dp, C.c_int32, dp, i32p, dp]
        L.orc_sim_order.restype = C.c_int
        L.orc_sim_points.argtypes = [P(Body), C.c_int32, dp]
        L.orc_sim_points.restype = C.c_int
        L.orc_sim_direction.argtypes = [C.c_double, C.c_double]
        L.orc_sim_direction.restype = C.c_int
        L.orc_sim.argtypes = [P(Config), P(Body), u8p, dp, C.c_int32, dp, dp, i32p]
        L.orc_sim.restype = C.c_int
        L.orc_rigid_update.argtypes = [P(Body), dp]
        L.orc_run.argtypes = [P(Config), P(Body), dp, u8p, C.c_int32, C.c_int32, C.c_int32, dp,
                              dp, dp, dp]
        L.orc_run.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _u8p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def lattice():
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    opp = np.zeros(9, np.int32)
    w = np.zeros(9)
    lib().orc_lattice(_i32p(cx), _i32p(cy), _i32p(opp), _dp(w))
    return cx, cy, opp, w


def feq(rho, ux, uy):
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _dp(out))
    return out


def guo(ux, uy, gx, gy):
    out = np.zeros(9)
    lib().orc_guo(ux, uy, gx, gy, _dp(out))
    return out


def raster(body: Body, nx: int, ny: int) -> np.ndarray:
    chi = np.zeros((ny, nx), np.uint8)
    lib().orc_raster(C.byref(body), nx, ny, _u8p(chi))
    return chi


def node_moments(cfg: Config, body: Body | None, fl, chi: int, i: int = 0, j: int = 0):
    fl = np.ascontiguousarray(fl, np.float64)
    out = np.zeros(5)
    lib().orc_node_moments(C.byref(cfg), C.byref(body) if body is not None else None, _dp(fl),
                           int(chi), i, j, _dp(out))
    return out  # rho, ux, uy, Gx, Gy


def penalization_literal(rho, jx, jy, chi, eta, usx, usy):
    out = np.zeros(4)
    lib().orc_penalization_literal(rho, jx, jy, int(chi), eta, usx, usy, _dp(out))
    return out  # ux, uy, Gx, Gy


def collide_node(cfg: Config, fl, rho, ux, uy, gx, gy):
    fl = np.ascontiguousarray(fl, np.float64)
    out = np.zeros(9)
    lib().orc_collide_node(C.byref(cfg), _dp(fl), rho, ux, uy, gx, gy, _dp(out))
    return out


def stress(cfg: Config, fl):
    fl = np.ascontiguousarray(fl, np.float64)
    out = np.zeros(3)
    lib().orc_stress(C.byref(cfg), _dp(fl), _dp(out))
    return out  # sxx, sxy, syy


def init(cfg: Config, body: Body, chi: np.ndarray) -> np.ndarray:
    f = np.zeros((9, cfg.ny, cfg.nx))
    lib().orc_init(C.byref(cfg), C.byref(body), _u8p(chi), _dp(f))
    return f


def collide(cfg: Config, body: Body, chi, f):
    ft = np.zeros_like(f)
    lib().orc_collide(C.byref(cfg), C.byref(body), _u8p(chi), _dp(f), _dp(ft))
    return ft


def fields(cfg: Config, body: Body, chi, f):
    rho = np.zeros((cfg.ny, cfg.nx))
    ux = np.zeros_like(rho)
    uy = np.zeros_like(rho)
    lib().orc_fields(C.byref(cfg), C.byref(body), _u8p(chi), _dp(f), _dp(rho), _dp(ux), _dp(uy))
    return rho, ux, uy


def stream(cfg: Config, ft, f_prev):
    ft = np.ascontiguousarray(ft, np.float64)
    f_prev = np.ascontiguousarray(f_prev, np.float64)
    out = np.zeros_like(ft)
    lib().orc_stream(C.byref(cfg), _dp(ft), _dp(f_prev), _dp(out))
    return out


def mem(cfg: Config, body: Body, chi, ft):
    out = np.zeros(3)
    lib().orc_mem(C.byref(cfg), C.byref(body), _u8p(chi), _dp(np.ascontiguousarray(ft)), _dp(out))
    return out


def angot(cfg: Config, body: Body, chi, f):
    """Volume-integral force (F_x, F_y, T) of Eq. Angotforce on the pre-collision
    field f (reading R19 of the C file)."""
    out = np.zeros(3)
    lib().orc_angot(C.byref(cfg), C.byref(body), _u8p(chi), _dp(np.ascontiguousarray(f)),
                    _dp(out))
    return out


def default_sim_points(body: Body) -> int:
    """Disk: ceil(2 pi R / 0.5) edges; airfoil: 849 (the count of Sec. 3.1)."""
    if body.n_sim > 0:
        return body.n_sim
    if body.kind == BODY_DISK:
        return int(np.ceil(2.0 * np.pi * (0.5 * body.length) / 0.5))
    return 849


def sim_points(body: Body, n: int | None = None) -> np.ndarray:
    n = default_sim_points(body) if n is None else n
    pts = np.zeros((n, 5))
    rc = lib().orc_sim_points(C.byref(body), n, _dp(pts))
    if rc != 0:
        raise ValueError("bad SIM point count")
    return pts


def sim_direction(nx, ny) -> int:
    return lib().orc_sim_direction(nx, ny)


def sim_order(cfg: Config, body: Body, chi, f, pts, order: int):
    """SIM with the stress copied (order 0) or extrapolated linearly (order 1)
    to each point; returns (F_x, F_y, T), sampled nodes, missing count and the
    per-point stresses (xx, xy, yy)."""
    out = np.zeros(3)
    nodes = np.zeros(len(pts), np.int32)
    sig = np.zeros((len(pts), 3))
    missing = lib().orc_sim_order(C.byref(cfg), C.byref(body), _u8p(chi),
                                  _dp(np.ascontiguousarray(f)), len(pts),
                                  _dp(np.ascontiguousarray(pts)), int(order), _dp(out),
                                  _i32p(nodes), _dp(sig))
    return out, nodes, missing, sig


def sim(cfg: Config, body: Body, chi, f, pts):
    out = np.zeros(3)
    nodes = np.zeros(len(pts), np.int32)
    missing = lib().orc_sim(C.byref(cfg), C.byref(body), _u8p(chi), _dp(np.ascontiguousarray(f)),
                            len(pts), _dp(np.ascontiguousarray(pts)), _dp(out), _i32p(nodes))
    return out, nodes, missing


def rigid_update(body: Body, force):
    force = np.ascontiguousarray(force, np.float64)
    lib().orc_rigid_update(C.byref(body), _dp(force))


def run(cfg: Config, body: Body, f, chi, nsteps: int, estimator: int = MEM,
        sim_pts: np.ndarray | None = None, histories: bool = True):
    """Advance f (pre-collision, modified in place) and chi by nsteps.

    Returns (mem_hist, sim_hist, body_hist, missing_sim_points)."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    assert chi.dtype == np.uint8 and chi.flags.c_contiguous
    mem_h = np.zeros((nsteps, 3)) if histories else None
    sim_h = np.zeros((nsteps, 3)) if histories else None
    body_h = np.zeros((nsteps, 6)) if histories else None
    n_sim = 0 if sim_pts is None else len(sim_pts)
    pts = None if sim_pts is None else np.ascontiguousarray(sim_pts)
    bad = lib().orc_run(C.byref(cfg), C.byref(body), _dp(f), _u8p(chi), nsteps, estimator, n_sim,
                        _dp(pts), _dp(mem_h), _dp(sim_h), _dp(body_h))
    return mem_h, sim_h, body_h, bad
