"""Python binding of the VP-LBM C ABI (include/vplbm.h).

The module-level functions carry the C names and only marshal arguments; every
step of the method runs in the CUDA library.  PyTorch provides the device
workspace, the stream and the device buffers of the field read-back calls.
`Lattice` bundles one context with its workspace.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

# enums (values of include/vplbm.h)
OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = range(7)
F64, F32, F16_OFS, BF16_OFS, F16_SR, BF16_SR = range(6)
BGK, TRT = 0, 1
FORCING_PAPER, FORCING_SPLIT = 0, 1
PERIODIC, INLET_BB, OUTLET_CONVECTIVE, SYMMETRY, NOSLIP_BB, OUTLET_FREE = range(6)
BODY_NONE, BODY_DISK, BODY_NACA4 = range(3)
MEM, SIM, ANGOT = 0, 1, 2

_STATUS = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA",
           EUNSTABLE: "EUNSTABLE", ETIMEOUT: "ETIMEOUT", ESTATE: "ESTATE"}


class VplbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class vplbm_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("dtype", C.c_int32), ("collision", C.c_int32),
        ("forcing", C.c_int32), ("bc", C.c_int32 * 4), ("sim_every", C.c_int32),
        ("max_sim_points", C.c_int32), ("history_len", C.c_int32), ("sim_order", C.c_int32),
        ("tau_plus", C.c_double), ("lambda_trt", C.c_double), ("eta", C.c_double),
        ("u_in", C.c_double * 2), ("body_force", C.c_double * 2), ("u_ref", C.c_double * 2),
    ]


class vplbm_body(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("moving", C.c_int32), ("n_sim_points", C.c_int32),
        ("estimator", C.c_int32), ("length", C.c_double), ("thickness", C.c_double),
        ("x_c", C.c_double), ("y_c", C.c_double), ("angle", C.c_double),
        ("pivot_chord_frac", C.c_double), ("u", C.c_double * 2), ("omega", C.c_double),
        ("density_ratio", C.c_double), ("gravity", C.c_double * 2),
    ]


def config(nx, ny, dtype=F32, collision=TRT, forcing=FORCING_PAPER,
           bc=(PERIODIC, PERIODIC, PERIODIC, PERIODIC), sim_every=1, max_sim_points=0,
           history_len=0, tau_plus=0.8, lambda_trt=1.0 / 6.0, eta=1e-6, u_in=(0.0, 0.0),
           body_force=(0.0, 0.0), u_ref=(0.0, 0.0), sim_order=0) -> vplbm_config:
    c = vplbm_config()
    c.nx, c.ny, c.dtype, c.collision, c.forcing = nx, ny, dtype, collision, forcing
    for k in range(4):
        c.bc[k] = bc[k]
    c.sim_every, c.max_sim_points, c.history_len = sim_every, max_sim_points, history_len
    c.sim_order = sim_order
    c.tau_plus, c.lambda_trt, c.eta = tau_plus, lambda_trt, eta
    c.u_in[0], c.u_in[1] = u_in
    c.body_force[0], c.body_force[1] = body_force
    c.u_ref[0], c.u_ref[1] = u_ref
    return c


def body(kind=BODY_NONE, length=0.0, thickness=0.12, x_c=0.0, y_c=0.0, angle=0.0,
         pivot_chord_frac=0.25, u=(0.0, 0.0), omega=0.0, moving=0, density_ratio=1.0,
         gravity=(0.0, 0.0), n_sim_points=0, estimator=MEM) -> vplbm_body:
    b = vplbm_body()
    b.kind, b.moving, b.n_sim_points, b.estimator = kind, moving, n_sim_points, estimator
    b.length, b.thickness, b.x_c, b.y_c, b.angle = length, thickness, x_c, y_c, angle
    b.pivot_chord_frac = pivot_chord_frac
    b.u[0], b.u[1] = u
    b.omega, b.density_ratio = omega, density_ratio
    b.gravity[0], b.gravity[1] = gravity
    return b


_lib = None

# (name, argtypes, restype) of every entry point of include/vplbm.h
_P = C.POINTER
_vp = C.c_void_p
_SIGS = [
    ("vplbm_workspace_bytes", [_P(vplbm_config), _P(C.c_size_t)], C.c_int),
    ("vplbm_create", [_P(vplbm_config), _vp, C.c_size_t, _vp, _P(_vp)], C.c_int),
    ("vplbm_set_stream", [_vp, _vp], C.c_int),
    ("vplbm_set_body", [_vp, _P(vplbm_body)], C.c_int),
    ("vplbm_step", [_vp, C.c_int32], C.c_int),
    ("vplbm_prepare", [_vp, C.c_int32], C.c_int),
    ("vplbm_force_mem", [_vp, _P(C.c_double), _P(C.c_double)], C.c_int),
    ("vplbm_force_sim", [_vp, _P(C.c_double), _P(C.c_double)], C.c_int),
    ("vplbm_force_angot", [_vp, _P(C.c_double), _P(C.c_double)], C.c_int),
    ("vplbm_forces_async", [_vp, _vp], C.c_int),
    ("vplbm_force_history", [_vp, C.c_int32, C.c_int32, _P(C.c_double)], C.c_int),
    ("vplbm_force_history_async", [_vp, C.c_int32, _vp], C.c_int),
    ("vplbm_force_sums", [_vp, _P(C.c_double), _P(C.c_int64)], C.c_int),
    ("vplbm_reset_sums", [_vp], C.c_int),
    ("vplbm_step_count", [_vp, _P(C.c_int64)], C.c_int),
    ("vplbm_get_f", [_vp, _vp], C.c_int),
    ("vplbm_get_fields", [_vp, _vp, _vp, _vp], C.c_int),
    ("vplbm_get_f_dev", [_vp, _vp], C.c_int),
    ("vplbm_get_fields_dev", [_vp, _vp, _vp, _vp], C.c_int),
    ("vplbm_set_state", [_vp, _vp, _vp, C.c_int32], C.c_int),
    ("vplbm_get_mask", [_vp, _vp], C.c_int),
    ("vplbm_get_mask_dev", [_vp, _vp], C.c_int),
    ("vplbm_state_bytes", [_vp, _P(C.c_size_t)], C.c_int),
    ("vplbm_save_state", [_vp, _vp, C.c_size_t], C.c_int),
    ("vplbm_load_state", [_vp, _vp, C.c_size_t], C.c_int),
    ("vplbm_get_body", [_vp, _P(C.c_double)], C.c_int),
    ("vplbm_get_sim_nodes", [_vp, _P(C.c_int32), C.c_int32, _P(C.c_int32)], C.c_int),
    ("vplbm_check", [_vp], C.c_int),
    ("vplbm_launch_count", [_vp, _P(C.c_int64)], C.c_int),
    ("vplbm_autotune", [_vp, C.c_int32, _P(C.c_int32)], C.c_int),
    ("vplbm_set_bulk_variant", [_vp, C.c_int32], C.c_int),
    ("vplbm_bulk_variant", [_vp, _P(C.c_int32)], C.c_int),
    ("vplbm_batch_create", [_P(_vp), C.c_int32, _vp, _P(_vp)], C.c_int),
    ("vplbm_batch_step", [_vp, C.c_int32], C.c_int),
    ("vplbm_batch_prepare", [_vp, C.c_int32], C.c_int),
    ("vplbm_batch_autotune", [_vp, C.c_int32, _P(C.c_int32)], C.c_int),
    ("vplbm_batch_destroy", [_vp], None),
    ("vplbm_sim_force_static", [_P(vplbm_config), _vp, _vp, C.c_int32, _P(C.c_double),
                                _P(C.c_double), _P(C.c_double), _vp], C.c_int),
    ("vplbm_destroy", [_vp], None),
    ("vplbm_last_error", [_vp], C.c_char_p),
]


def library_path() -> str:
    return _build.LIB_PATH


def lib():
    """Loads libvplbm.so (building it when sources are newer).  Raises when the
    library cannot be built or loaded: there is no fallback path."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(path)
        for name, args, res in _SIGS:
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(st, ctx=None):
    if st != OK:
        msg = lib().vplbm_last_error(ctx)
        raise VplbmError(st, msg.decode() if msg else "")


def _dptr(t) -> int:
    return t.data_ptr()


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def vplbm_workspace_bytes(cfg: vplbm_config) -> int:
    n = C.c_size_t()
    _check(lib().vplbm_workspace_bytes(C.byref(cfg), C.byref(n)))
    return n.value


def vplbm_create(cfg: vplbm_config, workspace_ptr: int, nbytes: int, stream: int):
    ctx = _vp()
    _check(lib().vplbm_create(C.byref(cfg), workspace_ptr, nbytes, stream, C.byref(ctx)))
    return ctx


def vplbm_set_stream(ctx, stream: int):
    _check(lib().vplbm_set_stream(ctx, stream), ctx)


def vplbm_set_body(ctx, b: vplbm_body):
    _check(lib().vplbm_set_body(ctx, C.byref(b)), ctx)


def vplbm_step(ctx, nsteps: int):
    _check(lib().vplbm_step(ctx, nsteps), ctx)


def vplbm_prepare(ctx, nsteps: int):
    _check(lib().vplbm_prepare(ctx, nsteps), ctx)


def _force(fn, ctx):
    F = (C.c_double * 2)()
    T = C.c_double()
    _check(fn(ctx, F, C.byref(T)), ctx)
    return np.array([F[0], F[1], T.value])


def vplbm_force_mem(ctx):
    return _force(lib().vplbm_force_mem, ctx)


def vplbm_force_sim(ctx):
    return _force(lib().vplbm_force_sim, ctx)


def vplbm_force_angot(ctx):
    return _force(lib().vplbm_force_angot, ctx)


def vplbm_forces_async(ctx, host_ptr: int):
    _check(lib().vplbm_forces_async(ctx, host_ptr), ctx)


def vplbm_force_history(ctx, estimator: int, count: int):
    out = np.zeros((count, 3))
    _check(lib().vplbm_force_history(ctx, estimator, count,
                                     out.ctypes.data_as(_P(C.c_double))), ctx)
    return out


def vplbm_force_sums(ctx):
    s = np.zeros(6)
    n = np.zeros(2, np.int64)
    _check(lib().vplbm_force_sums(ctx, s.ctypes.data_as(_P(C.c_double)),
                                  n.ctypes.data_as(_P(C.c_int64))), ctx)
    return s, n


def vplbm_reset_sums(ctx):
    _check(lib().vplbm_reset_sums(ctx), ctx)


def vplbm_step_count(ctx) -> int:
    n = C.c_int64()
    _check(lib().vplbm_step_count(ctx, C.byref(n)), ctx)
    return n.value


def _host_ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def vplbm_get_f(ctx, f: np.ndarray):
    """Pre-collision populations into a host float64 array [9][ny][nx]."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    _check(lib().vplbm_get_f(ctx, _host_ptr(f)), ctx)


def vplbm_get_fields(ctx, rho: np.ndarray, ux: np.ndarray, uy: np.ndarray):
    for a in (rho, ux, uy):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _check(lib().vplbm_get_fields(ctx, _host_ptr(rho), _host_ptr(ux), _host_ptr(uy)), ctx)


def vplbm_get_f_dev(ctx, f_dev_ptr: int):
    _check(lib().vplbm_get_f_dev(ctx, f_dev_ptr), ctx)


def vplbm_get_fields_dev(ctx, rho_ptr: int, ux_ptr: int, uy_ptr: int):
    _check(lib().vplbm_get_fields_dev(ctx, rho_ptr, ux_ptr, uy_ptr), ctx)


def vplbm_set_state(ctx, f_dev_ptr: int, prev_dev_ptr, post_collision: int):
    _check(lib().vplbm_set_state(ctx, f_dev_ptr, prev_dev_ptr, post_collision), ctx)


def vplbm_get_mask(ctx, chi: np.ndarray):
    assert chi.dtype == np.uint8 and chi.flags.c_contiguous
    _check(lib().vplbm_get_mask(ctx, _host_ptr(chi)), ctx)


def vplbm_get_mask_dev(ctx, chi_dev_ptr: int):
    _check(lib().vplbm_get_mask_dev(ctx, chi_dev_ptr), ctx)


def vplbm_state_bytes(ctx) -> int:
    n = C.c_size_t()
    _check(lib().vplbm_state_bytes(ctx, C.byref(n)), ctx)
    return n.value


def vplbm_save_state(ctx) -> np.ndarray:
    """The lattice's snapshot as a host byte array."""
    buf = np.zeros(vplbm_state_bytes(ctx), np.uint8)
    _check(lib().vplbm_save_state(ctx, _host_ptr(buf), buf.nbytes), ctx)
    return buf


def vplbm_load_state(ctx, snapshot: np.ndarray):
    snap = np.ascontiguousarray(snapshot, np.uint8)
    _check(lib().vplbm_load_state(ctx, _host_ptr(snap), snap.nbytes), ctx)


def vplbm_force_history_async(ctx, count: int, out_ptr: int):
    """Queues the last `count` history rows ([count][9] float64) into host
    memory at out_ptr (page-locked for an asynchronous copy)."""
    _check(lib().vplbm_force_history_async(ctx, count, out_ptr), ctx)


def vplbm_get_body(ctx):
    s = (C.c_double * 6)()
    _check(lib().vplbm_get_body(ctx, s), ctx)
    return np.array(list(s))


def vplbm_get_sim_nodes(ctx, capacity: int):
    out = np.zeros(max(capacity, 1), np.int32)
    n = C.c_int32()
    _check(lib().vplbm_get_sim_nodes(ctx, out.ctypes.data_as(_P(C.c_int32)), capacity,
                                     C.byref(n)), ctx)
    return out[:n.value]


def vplbm_check(ctx):
    _check(lib().vplbm_check(ctx), ctx)


def vplbm_launch_count(ctx) -> int:
    n = C.c_int64()
    _check(lib().vplbm_launch_count(ctx, C.byref(n)), ctx)
    return n.value


def vplbm_autotune(ctx, trials: int = 20) -> int:
    v = C.c_int32()
    _check(lib().vplbm_autotune(ctx, trials, C.byref(v)), ctx)
    return v.value


def vplbm_set_bulk_variant(ctx, variant: int):
    _check(lib().vplbm_set_bulk_variant(ctx, variant), ctx)


def vplbm_bulk_variant(ctx) -> int:
    v = C.c_int32()
    _check(lib().vplbm_bulk_variant(ctx, C.byref(v)), ctx)
    return v.value


def vplbm_batch_create(ctxs, stream: int):
    arr = (_vp * len(ctxs))(*ctxs)
    b = _vp()
    _check(lib().vplbm_batch_create(arr, len(ctxs), stream, C.byref(b)))
    return b


def vplbm_batch_step(batch, nsteps: int):
    _check(lib().vplbm_batch_step(batch, nsteps))


def vplbm_batch_prepare(batch, nsteps: int):
    _check(lib().vplbm_batch_prepare(batch, nsteps))


def vplbm_batch_autotune(batch, n: int, trials: int = 20) -> list:
    """Per-lattice launch forms chosen by the batch tuner (n lattices)."""
    v = (C.c_int32 * n)()
    _check(lib().vplbm_batch_autotune(batch, trials, v))
    return list(v)


def vplbm_batch_destroy(batch):
    lib().vplbm_batch_destroy(batch)


def vplbm_sim_force_static(cfg: vplbm_config, f_dev_ptr: int, chi_dev_ptr: int, pts, ref,
                           stream: int):
    """SIM force of a supplied state with no device allocation (see
    include/vplbm.h); pts is an (n, 5) float64 host array."""
    pts = np.ascontiguousarray(pts, np.float64)
    ref = np.ascontiguousarray(ref, np.float64)
    if pts.ndim != 2 or pts.shape[1] != 5:
        raise ValueError(f"pts must have shape (n, 5), not {pts.shape}")
    if ref.shape != (2,):
        raise ValueError(f"ref must hold two values, not shape {ref.shape}")
    out = np.zeros(3)
    _check(lib().vplbm_sim_force_static(C.byref(cfg), f_dev_ptr, chi_dev_ptr, len(pts),
                                        pts.ctypes.data_as(_P(C.c_double)),
                                        ref.ctypes.data_as(_P(C.c_double)),
                                        out.ctypes.data_as(_P(C.c_double)), stream))
    return out


def vplbm_destroy(ctx):
    lib().vplbm_destroy(ctx)


def vplbm_last_error(ctx=None) -> str:
    m = lib().vplbm_last_error(ctx)
    return m.decode() if m else ""


# ---------------------------------------------------------------------------
# one lattice with its workspace
# ---------------------------------------------------------------------------
class Lattice:
    """A lattice in a PyTorch-allocated device workspace."""

    def __init__(self, cfg: vplbm_config, device=None, stream=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.nbytes = vplbm_workspace_bytes(cfg)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            self._ws_ptr = (base + 255) // 256 * 256
            self.ctx = vplbm_create(cfg, self._ws_ptr, self.nbytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            vplbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        vplbm_set_stream(self.ctx, stream.cuda_stream)

    def set_body(self, b: vplbm_body):
        self.body_cfg = b
        vplbm_set_body(self.ctx, b)

    def step(self, n: int = 1):
        vplbm_step(self.ctx, n)

    def prepare(self, n: int):
        vplbm_prepare(self.ctx, n)

    def force_mem(self):
        return vplbm_force_mem(self.ctx)

    def force_sim(self):
        return vplbm_force_sim(self.ctx)

    def force_angot(self):
        return vplbm_force_angot(self.ctx)

    def history(self, estimator: int, count: int):
        return vplbm_force_history(self.ctx, estimator, count)

    def sums(self):
        return vplbm_force_sums(self.ctx)

    def reset_sums(self):
        vplbm_reset_sums(self.ctx)

    @property
    def steps(self) -> int:
        return vplbm_step_count(self.ctx)

    def get_f(self) -> np.ndarray:
        out = np.empty((9, self.cfg.ny, self.cfg.nx))
        vplbm_get_f(self.ctx, out)
        return out

    def get_fields(self):
        rho, ux, uy = (np.empty((self.cfg.ny, self.cfg.nx)) for _ in range(3))
        vplbm_get_fields(self.ctx, rho, ux, uy)
        return rho, ux, uy

    def set_state(self, f: np.ndarray, prev: np.ndarray | None = None, post_collision=False):
        t = self.torch
        with t.cuda.stream(self.stream):
            fd = t.as_tensor(np.ascontiguousarray(f, np.float64)).to(self.device)
            pd = None if prev is None else t.as_tensor(np.ascontiguousarray(prev, np.float64)).to(self.device)
            vplbm_set_state(self.ctx, _dptr(fd), None if pd is None else _dptr(pd),
                            1 if post_collision else 0)
            self.stream.synchronize()

    def get_mask(self) -> np.ndarray:
        out = np.empty((self.cfg.ny, self.cfg.nx), np.uint8)
        vplbm_get_mask(self.ctx, out)
        return out

    def save_state(self) -> np.ndarray:
        return vplbm_save_state(self.ctx)

    def load_state(self, snapshot: np.ndarray):
        vplbm_load_state(self.ctx, snapshot)

    def get_body(self):
        return vplbm_get_body(self.ctx)

    def sim_nodes(self):
        n = 8192 if self.cfg.max_sim_points == 0 else self.cfg.max_sim_points
        return vplbm_get_sim_nodes(self.ctx, n)

    def check(self):
        vplbm_check(self.ctx)

    @property
    def launches(self) -> int:
        return vplbm_launch_count(self.ctx)

    def autotune(self, trials: int = 20) -> int:
        return vplbm_autotune(self.ctx, trials)

    @property
    def bulk_variant(self) -> int:
        return vplbm_bulk_variant(self.ctx)

    @bulk_variant.setter
    def bulk_variant(self, v: int):
        vplbm_set_bulk_variant(self.ctx, v)


# ---------------------------------------------------------------------------
# workloads -> ABI structures
# ---------------------------------------------------------------------------
_DTYPES = {"f64": F64, "f32": F32, "f16": F16_OFS, "bf16": BF16_OFS, "f16sr": F16_SR,
           "bf16sr": BF16_SR}
_BCS = {"periodic": PERIODIC, "inlet": INLET_BB, "outlet": OUTLET_CONVECTIVE,
        "symmetry": SYMMETRY, "noslip": NOSLIP_BB, "outlet_free": OUTLET_FREE}
_KINDS = {"none": BODY_NONE, "disk": BODY_DISK, "naca": BODY_NACA4}


def config_of(w, dtype: str | None = None, **over) -> vplbm_config:
    kw = dict(nx=w.nx, ny=w.ny, dtype=_DTYPES[dtype or w.dtype],
              collision=BGK if w.collision == "bgk" else TRT,
              forcing=FORCING_PAPER if w.forcing == "paper" else FORCING_SPLIT,
              bc=tuple(_BCS[b] for b in w.bc), sim_every=w.sim_every, tau_plus=w.tau_plus,
              lambda_trt=w.lambda_trt, eta=w.eta, u_in=w.u_in, body_force=w.body_force,
              u_ref=w.u_ref)
    kw.update(over)
    return config(**kw)


def body_of(w) -> vplbm_body:
    b = w.body
    return body(kind=_KINDS[b.kind], length=b.length, thickness=b.thickness, x_c=b.x_c,
                y_c=b.y_c, angle=b.angle, pivot_chord_frac=b.pivot_chord_frac,
                moving=1 if b.moving else 0, density_ratio=b.density_ratio,
                gravity=b.gravity, n_sim_points=b.n_sim_points,
                estimator=SIM if b.estimator == "sim" else MEM)


# ---------------------------------------------------------------------------
# several lattices stepped together
# ---------------------------------------------------------------------------
class Batch:
    """Lattices stepped together (vplbm_batch_*): each lattice's steps run on a
    stream of their own, forked from and joined to the batch's stream, 32-step
    runs replayed from one CUDA graph.  Keeps the Lattice objects alive;
    close() (or garbage collection) releases the batch before them."""

    def __init__(self, lattices, stream=None):
        import torch
        self.lattices = list(lattices)
        dev = self.lattices[0].device
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        with torch.cuda.device(dev):
            self.handle = vplbm_batch_create([l.ctx for l in self.lattices],
                                             self.stream.cuda_stream)

    def step(self, n: int = 1):
        vplbm_batch_step(self.handle, n)

    def prepare(self, n: int):
        vplbm_batch_prepare(self.handle, n)

    def autotune(self, trials: int = 20) -> list:
        """Each member's launch form, tuned per size class."""
        return vplbm_batch_autotune(self.handle, len(self.lattices), trials)

    @property
    def launches(self) -> int:
        return sum(l.launches for l in self.lattices)

    def close(self):
        if getattr(self, "handle", None) is not None:
            vplbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
