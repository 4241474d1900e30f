"""Thin ctypes binding of liblbm (include/lbm.h): same names as the C ABI.

Argument marshalling only -- every step of the method runs in the CUDA
kernels of liblbm.so.  There is no CPU fallback: if the library cannot be
built or loaded, or no CUDA device is present, the calls raise.

Module-level functions mirror the C entry points one to one (``lbm_create``,
``lbm_step``, ...), taking and returning numpy arrays in the C layouts
([ny, nx] node fields, [9, ny, nx] distributions).  :class:`Lbm` wraps one
context; by default its distribution arrays live in a PyTorch CUDA tensor and
its work runs on a PyTorch CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_EINVAL = -1
LBM_ENOMEM = -2
LBM_ECUDA = -3
LBM_EUNSTABLE = -4
LBM_EUNSUPPORTED = -5
LBM_ETIMEOUT = -6
LBM_ENOCONTACT = -7

LBM_EOS_CARNAHAN_STARLING = 0
LBM_EOS_PIECEWISE = 1
LBM_WET_GEOMETRIC = 0
LBM_WET_MARTYS_CHEN = 1
LBM_KERNEL_AUTO = 0
LBM_KERNEL_REFERENCE = 1
LBM_KERNEL_FUSED = 2

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
DP = ctypes.POINTER(ctypes.c_double)


class lbm_eos(ctypes.Structure):
    _fields_ = [("kind", c_int), ("a", c_double), ("b", c_double), ("R", c_double),
                ("theta_v", c_double), ("theta_m", c_double), ("theta_l", c_double),
                ("rho1", c_double), ("rho2", c_double)]


class lbm_params(ctypes.Structure):
    _fields_ = [("A", c_double), ("kappa", c_double), ("G_w", c_double), ("n_iter", c_int),
                ("wetting", c_int), ("precision", c_int), ("kernel", c_int),
                ("s_e", c_double), ("s_eps", c_double), ("s_j", c_double), ("s_q", c_double),
                ("s_nu", c_double), ("check_every", c_int), ("rho_mid", c_double),
                ("rho_max", c_double), ("rho_ghost_max", c_double), ("graph_steps", c_int)]


class lbm_info(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("walls", c_int), ("precision", c_int),
                ("kernel_in_use", c_int), ("wetting", c_int), ("T", c_double), ("tau", c_double),
                ("rho_v", c_double), ("rho_l", c_double), ("rho_max", c_double),
                ("rho_mid", c_double), ("tile_w", c_int), ("tile_blocks", c_int),
                ("tile_stages", c_int), ("steps_done", ctypes.c_longlong)]


class lbm_instance_desc(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("eos", lbm_eos), ("T", c_double), ("tau", c_double),
                ("theta", DP), ("params", lbm_params)]


class lbm_batch_config(ctypes.Structure):
    _fields_ = [("threads", c_int), ("ctas_per_sm", c_int), ("stages", c_int), ("band_rows", c_int * 4),
                ("steps_per_launch", c_int), ("graph_launches", c_int), ("wait_seconds", c_double),
                ("hold_instance", c_int)]


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lbm_strerror(status)} ({status})")


_lib = None
_lock = threading.Lock()

# C signatures: name -> (restype, argtypes)
_SIGS = {
    "lbm_strerror": (ctypes.c_char_p, [c_int]),
    "lbm_params_default": (c_int, [ctypes.POINTER(lbm_params)]),
    "lbm_eos_critical": (c_int, [ctypes.POINTER(lbm_eos), DP, DP]),
    "lbm_coexistence": (c_int, [ctypes.POINTER(lbm_eos), c_double, DP, DP]),
    "lbm_eos_bounds": (c_int, [ctypes.POINTER(lbm_eos), c_double, DP, DP, DP, DP]),
    "lbm_create": (c_int, [c_int, c_int, ctypes.POINTER(lbm_eos), c_double, c_double, DP, c_void_p,
                           ctypes.POINTER(lbm_params), c_void_p, ctypes.POINTER(c_void_p)]),
    "lbm_required_state_bytes": (c_size_t, [c_int, c_int, c_int]),
    "lbm_create_with_buffer": (c_int, [c_int, c_int, ctypes.POINTER(lbm_eos), c_double, c_double, DP,
                                       c_void_p, ctypes.POINTER(lbm_params), c_void_p, c_void_p,
                                       c_size_t, ctypes.POINTER(c_void_p)]),
    "lbm_set_rho": (c_int, [c_void_p, DP]),
    "lbm_init_droplets": (c_int, [c_void_p, c_int, DP, DP, ctypes.POINTER(c_int), c_double]),
    "lbm_step": (c_int, [c_void_p, c_int]),
    "lbm_status": (c_int, [c_void_p]),
    "lbm_get_rho": (c_int, [c_void_p, DP]),
    "lbm_get_u": (c_int, [c_void_p, DP, DP]),
    "lbm_get_f": (c_int, [c_void_p, DP]),
    "lbm_set_f": (c_int, [c_void_p, DP]),
    "lbm_get_fields": (c_int, [c_void_p, DP, DP, DP, DP, DP, DP, DP, DP]),
    "lbm_contact_angle": (c_int, [c_void_p, c_int, c_int, c_int, DP, DP, DP]),
    "lbm_mass": (c_int, [c_void_p, DP]),
    "lbm_max_speed": (c_int, [c_void_p, DP]),
    "lbm_state_bytes": (c_size_t, [c_void_p]),
    "lbm_save": (c_int, [c_void_p, c_void_p, c_size_t]),
    "lbm_load": (c_int, [c_void_p, c_void_p, c_size_t]),
    "lbm_get_info": (c_int, [c_void_p, ctypes.POINTER(lbm_info)]),
    "lbm_launch_count": (ctypes.c_ulonglong, [c_void_p]),
    "lbm_sync": (c_int, [c_void_p]),
    "lbm_destroy": (None, [c_void_p]),
    "lbm_mass_noalloc": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]),
    "lbm_adjoint_record": (c_int, [c_void_p, c_int, c_int]),
    "lbm_adjoint_backward": (c_int, [c_void_p, DP, DP, DP, DP]),
    "lbm_adjoint_release": (c_int, [c_void_p]),
    "lbm_batch_config_default": (c_int, [ctypes.POINTER(lbm_batch_config)]),
    "lbm_batch_create": (c_int, [c_int, ctypes.POINTER(lbm_instance_desc), ctypes.POINTER(lbm_batch_config),
                                 c_void_p, ctypes.POINTER(c_void_p)]),
    "lbm_batch_size": (c_int, [c_void_p]),
    "lbm_batch_instance": (c_void_p, [c_void_p, c_int]),
    "lbm_batch_step": (c_int, [c_void_p, c_int]),
    "lbm_batch_status": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "lbm_batch_contact_angles": (c_int, [c_void_p, c_int, DP, DP, DP, ctypes.POINTER(c_int)]),
    "lbm_batch_autotune": (c_int, [c_void_p, c_int, ctypes.POINTER(lbm_batch_config)]),
    "lbm_batch_get_config": (c_int, [c_void_p, ctypes.POINTER(lbm_batch_config)]),
    "lbm_batch_set_config": (c_int, [c_void_p, ctypes.POINTER(lbm_batch_config)]),
    "lbm_batch_get_plan": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                   ctypes.POINTER(c_int)]),
    "lbm_batch_launch_count": (ctypes.c_ulonglong, [c_void_p]),
    "lbm_batch_node_updates": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_ulonglong)]),
    "lbm_batch_destroy": (None, [c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(rebuild: bool = True):
    """Load liblbm.so (building it first if a source is newer); raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if rebuild else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"liblbm.so not found at {path}; run paper_1501_05430_gb300/build.py")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    return list(_SIGS)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(DP)


def _c64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = np.ascontiguousarray(np.broadcast_to(a, shape))
    return a


def _check(st: int, where: str):
    if st != LBM_OK:
        raise LbmError(st, where)


# ---- C entry points, one Python function each -------------------------------

def lbm_strerror(status: int) -> str:
    return load().lbm_strerror(status).decode()


def lbm_params_default(**overrides) -> lbm_params:
    p = lbm_params()
    _check(load().lbm_params_default(ctypes.byref(p)), "lbm_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def carnahan_starling(a=1.0, b=4.0, R=1.0) -> lbm_eos:
    return lbm_eos(LBM_EOS_CARNAHAN_STARLING, a, b, R, 0, 0, 0, 0, 0)


def piecewise(theta_v, theta_m, theta_l, rho1, rho2) -> lbm_eos:
    return lbm_eos(LBM_EOS_PIECEWISE, 0, 0, 0, theta_v, theta_m, theta_l, rho1, rho2)


def lbm_eos_critical(eos: lbm_eos):
    tc, rc = c_double(), c_double()
    _check(load().lbm_eos_critical(ctypes.byref(eos), ctypes.byref(tc), ctypes.byref(rc)), "lbm_eos_critical")
    return tc.value, rc.value


def lbm_coexistence(eos: lbm_eos, T: float = 0.0):
    rv, rl = c_double(), c_double()
    _check(load().lbm_coexistence(ctypes.byref(eos), T, ctypes.byref(rv), ctypes.byref(rl)), "lbm_coexistence")
    return rv.value, rl.value


def lbm_eos_bounds(eos: lbm_eos, T: float = 0.0):
    """(rho_v, rho_l, rho_max, rho_mid) that lbm_create derives for this EOS and T."""
    v = [c_double() for _ in range(4)]
    _check(load().lbm_eos_bounds(ctypes.byref(eos), T, *[ctypes.byref(x) for x in v]), "lbm_eos_bounds")
    return tuple(x.value for x in v)


def lbm_required_state_bytes(nx, ny, precision) -> int:
    return load().lbm_required_state_bytes(nx, ny, precision)


def _geometry(nx, ny, theta, walls):
    th = None if theta is None else _c64(theta, (ny, nx))
    mask = None
    if walls:
        mask = np.zeros((ny, nx), np.uint8)
        mask[0] = 1
        mask[-1] = 1
    return th, mask


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def lbm_create(nx, ny, eos, T, tau, theta=None, walls=True, params=None, stream=None):
    """Returns the context handle (int).  theta: radians, scalar or [ny, nx]."""
    th, mask = _geometry(nx, ny, theta, walls)
    out = c_void_p()
    st = load().lbm_create(nx, ny, ctypes.byref(eos), T, tau, None if th is None else _dp(th),
                           None if mask is None else mask.ctypes.data_as(c_void_p),
                           None if params is None else ctypes.byref(params),
                           _stream_handle(stream), ctypes.byref(out))
    _check(st, "lbm_create")
    return out.value


def lbm_create_with_buffer(nx, ny, eos, T, tau, state_ptr, state_bytes, theta=None, walls=True, params=None,
                           stream=None):
    th, mask = _geometry(nx, ny, theta, walls)
    out = c_void_p()
    st = load().lbm_create_with_buffer(nx, ny, ctypes.byref(eos), T, tau, None if th is None else _dp(th),
                                       None if mask is None else mask.ctypes.data_as(c_void_p),
                                       None if params is None else ctypes.byref(params),
                                       _stream_handle(stream), c_void_p(state_ptr), state_bytes,
                                       ctypes.byref(out))
    _check(st, "lbm_create_with_buffer")
    return out.value


def lbm_set_rho(ctx, rho):
    rho = _c64(rho)
    _check(load().lbm_set_rho(ctx, _dp(rho)), "lbm_set_rho")


def lbm_init_droplets(ctx, xc, radius, wall, width=3.0):
    xc, radius = _c64(xc).ravel(), _c64(radius).ravel()
    w = np.ascontiguousarray(np.asarray(wall, dtype=np.int32).ravel())
    _check(load().lbm_init_droplets(ctx, len(xc), _dp(xc), _dp(radius),
                                    w.ctypes.data_as(ctypes.POINTER(c_int)), width), "lbm_init_droplets")


def lbm_step(ctx, nsteps=1):
    _check(load().lbm_step(ctx, nsteps), "lbm_step")


def lbm_status(ctx) -> int:
    return load().lbm_status(ctx)


def lbm_get_info(ctx) -> lbm_info:
    info = lbm_info()
    _check(load().lbm_get_info(ctx, ctypes.byref(info)), "lbm_get_info")
    return info


def _shape(ctx):
    i = lbm_get_info(ctx)
    return i.ny, i.nx


def lbm_get_rho(ctx, out=None):
    out = np.empty(_shape(ctx)) if out is None else out
    _check(load().lbm_get_rho(ctx, _dp(out)), "lbm_get_rho")
    return out


def lbm_get_u(ctx):
    shp = _shape(ctx)
    ux, uy = np.empty(shp), np.empty(shp)
    _check(load().lbm_get_u(ctx, _dp(ux), _dp(uy)), "lbm_get_u")
    return ux, uy


def lbm_get_f(ctx):
    ny, nx = _shape(ctx)
    out = np.empty((9, ny, nx))
    _check(load().lbm_get_f(ctx, _dp(out)), "lbm_get_f")
    return out


def lbm_set_f(ctx, f):
    f = _c64(f)
    _check(load().lbm_set_f(ctx, _dp(f)), "lbm_set_f")


def lbm_get_fields(ctx):
    shp = _shape(ctx)
    arrs = [np.empty(shp) for _ in range(8)]
    _check(load().lbm_get_fields(ctx, *[_dp(a) for a in arrs]), "lbm_get_fields")
    return dict(zip(["rho", "psi", "U", "Fx", "Fy", "Qxx", "Qyy", "Qxy"], arrs))


def lbm_contact_angle(ctx, wall, x0, x1):
    th, H, L = c_double(), c_double(), c_double()
    _check(load().lbm_contact_angle(ctx, wall, x0, x1, ctypes.byref(th), ctypes.byref(H), ctypes.byref(L)),
           "lbm_contact_angle")
    return th.value, H.value, L.value


def lbm_mass(ctx) -> float:
    m = c_double()
    _check(load().lbm_mass(ctx, ctypes.byref(m)), "lbm_mass")
    return m.value


def lbm_max_speed(ctx) -> float:
    m = c_double()
    _check(load().lbm_max_speed(ctx, ctypes.byref(m)), "lbm_max_speed")
    return m.value


def lbm_state_bytes(ctx) -> int:
    return load().lbm_state_bytes(ctx)


def lbm_save(ctx) -> bytes:
    n = lbm_state_bytes(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(load().lbm_save(ctx, buf, n), "lbm_save")
    return buf.raw


def lbm_load(ctx, image: bytes):
    buf = ctypes.create_string_buffer(image, len(image))
    _check(load().lbm_load(ctx, buf, len(image)), "lbm_load")


def lbm_launch_count(ctx) -> int:
    return load().lbm_launch_count(ctx)


def lbm_sync(ctx):
    _check(load().lbm_sync(ctx), "lbm_sync")


def lbm_destroy(ctx):
    if ctx:
        load().lbm_destroy(ctx)


def lbm_mass_noalloc(f_ptr, nx, ny, precision, walls, mass_ptr, stream=None):
    """Sum of rho over the fluid nodes of a caller-owned device array f_ptr
    ([9][ny][nx] of float32 or float64) into the device double at mass_ptr,
    without allocating device memory (see lbm.h).  Pointers are ints."""
    _check(load().lbm_mass_noalloc(c_void_p(f_ptr), nx, ny, precision, 1 if walls else 0, c_void_p(mass_ptr),
                                   _stream_handle(stream)), "lbm_mass_noalloc")


def lbm_adjoint_record(ctx, nsteps, checkpoint_every=100):
    _check(load().lbm_adjoint_record(ctx, nsteps, checkpoint_every), "lbm_adjoint_record")


def lbm_adjoint_backward(ctx, dl_drho, want_df0=False):
    """(dL/dtheta [2, nx], dL/dT, dL/df0 [9, ny, nx] or None) for dL/drho at the
    recorded final time ([ny, nx])."""
    ny, nx = _shape(ctx)
    g = _c64(dl_drho, (ny, nx))
    dth = np.zeros((2, nx))
    dT = c_double()
    df0 = np.zeros((9, ny, nx)) if want_df0 else None
    _check(load().lbm_adjoint_backward(ctx, _dp(g), _dp(dth), ctypes.byref(dT),
                                       _dp(df0) if want_df0 else None), "lbm_adjoint_backward")
    return dth, dT.value, df0


def lbm_adjoint_release(ctx):
    _check(load().lbm_adjoint_release(ctx), "lbm_adjoint_release")


def lbm_batch_config_default(**overrides) -> lbm_batch_config:
    c = lbm_batch_config()
    _check(load().lbm_batch_config_default(ctypes.byref(c)), "lbm_batch_config_default")
    for k, v in overrides.items():
        if k == "band_rows":
            for i, b in enumerate(v):
                c.band_rows[i] = b
        else:
            setattr(c, k, v)
    return c


def lbm_batch_create(instances, cfg=None, stream=None):
    """instances: list of dicts with nx, ny, eos (lbm_eos), T, tau, theta
    (radians, scalar or [ny, nx], optional) and params (lbm_params, precision
    32).  Returns the batch handle (int)."""
    n = len(instances)
    descs = (lbm_instance_desc * n)()
    keep = []
    for i, d in enumerate(instances):
        nx, ny = d["nx"], d["ny"]
        descs[i].nx, descs[i].ny = nx, ny
        descs[i].eos = d["eos"]
        descs[i].T, descs[i].tau = d["T"], d["tau"]
        th = d.get("theta")
        if th is not None:
            th = _c64(th, (ny, nx))
            keep.append(th)
            descs[i].theta = _dp(th)
        descs[i].params = d.get("params") or lbm_params_default(precision=32)
    out = c_void_p()
    st = load().lbm_batch_create(n, descs, None if cfg is None else ctypes.byref(cfg), _stream_handle(stream),
                                 ctypes.byref(out))
    _check(st, "lbm_batch_create")
    return out.value


def lbm_batch_size(b) -> int:
    return load().lbm_batch_size(b)


def lbm_batch_instance(b, i):
    ctx = load().lbm_batch_instance(b, i)
    if not ctx:
        raise LbmError(LBM_EINVAL, "lbm_batch_instance")
    return ctx


def lbm_batch_step(b, nsteps=1):
    _check(load().lbm_batch_step(b, nsteps), "lbm_batch_step")


def lbm_batch_status(b):
    """(batch status, per-instance statuses as an int32 array)."""
    n = lbm_batch_size(b)
    out = np.zeros(n, np.int32)
    st = load().lbm_batch_status(b, out.ctypes.data_as(ctypes.POINTER(c_int)))
    return st, out


def lbm_batch_contact_angles(b, wall=0):
    """(theta, H, L, status) arrays over the instances, full width of each."""
    n = lbm_batch_size(b)
    th, H, L = np.zeros(n), np.zeros(n), np.zeros(n)
    stv = np.zeros(n, np.int32)
    _check(load().lbm_batch_contact_angles(b, wall, _dp(th), _dp(H), _dp(L),
                                           stv.ctypes.data_as(ctypes.POINTER(c_int))), "lbm_batch_contact_angles")
    return th, H, L, stv


def lbm_batch_autotune(b, trial_steps=20) -> lbm_batch_config:
    c = lbm_batch_config()
    _check(load().lbm_batch_autotune(b, trial_steps, ctypes.byref(c)), "lbm_batch_autotune")
    return c


def lbm_batch_get_config(b) -> lbm_batch_config:
    c = lbm_batch_config()
    _check(load().lbm_batch_get_config(b, ctypes.byref(c)), "lbm_batch_get_config")
    return c


def lbm_batch_set_config(b, cfg: lbm_batch_config):
    _check(load().lbm_batch_set_config(b, ctypes.byref(cfg)), "lbm_batch_set_config")


def lbm_batch_get_plan(b):
    """dict(grid, items, smem_bytes, ctas_per_sm) of the current launch shape."""
    v = [c_int() for _ in range(4)]
    _check(load().lbm_batch_get_plan(b, *[ctypes.byref(x) for x in v]), "lbm_batch_get_plan")
    return dict(zip(("grid", "items", "smem_bytes", "ctas_per_sm"), (x.value for x in v)))


def lbm_batch_launch_count(b) -> int:
    return load().lbm_batch_launch_count(b)


def lbm_batch_node_updates(b) -> np.ndarray:
    n = lbm_batch_size(b)
    out = np.zeros(n, dtype=np.uint64)
    _check(load().lbm_batch_node_updates(b, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong))),
           "lbm_batch_node_updates")
    return out


def lbm_batch_destroy(b):
    if b:
        load().lbm_batch_destroy(b)


# ---- convenience wrapper ------------------------------------------------------

class Lbm:
    """One liblbm context.  With ``torch_state=True`` (default) the two
    distribution arrays are a PyTorch CUDA tensor owned by this object and
    passed to lbm_create_with_buffer; ``stream`` is a torch.cuda.Stream, a raw
    cudaStream_t as int, or None (legacy default stream)."""

    def __init__(self, nx, ny, eos, T, tau, theta=None, walls=True, params=None, stream=None,
                 torch_state=True):
        self.nx, self.ny = nx, ny
        self.stream = stream
        self._state = None
        if params is None:
            params = lbm_params_default()
        if torch_state:
            import torch
            nbytes = lbm_required_state_bytes(nx, ny, params.precision)
            self._state = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            self.ctx = lbm_create_with_buffer(nx, ny, eos, T, tau, self._state.data_ptr(), nbytes, theta, walls,
                                              params, stream)
        else:
            self.ctx = lbm_create(nx, ny, eos, T, tau, theta, walls, params, stream)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None
        self._state = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    info = property(lambda self: lbm_get_info(self.ctx))

    def set_rho(self, rho):
        lbm_set_rho(self.ctx, rho)

    def init_droplets(self, xc, radius, wall, width=3.0):
        lbm_init_droplets(self.ctx, xc, radius, wall, width)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def status(self):
        return lbm_status(self.ctx)

    def rho(self):
        return lbm_get_rho(self.ctx)

    def u(self):
        return lbm_get_u(self.ctx)

    def f(self):
        return lbm_get_f(self.ctx)

    def set_f(self, f):
        lbm_set_f(self.ctx, f)

    def fields(self):
        return lbm_get_fields(self.ctx)

    def contact_angle(self, wall, x0, x1):
        return lbm_contact_angle(self.ctx, wall, x0, x1)

    def mass(self):
        return lbm_mass(self.ctx)

    def max_speed(self):
        return lbm_max_speed(self.ctx)

    def save(self):
        return lbm_save(self.ctx)

    def load(self, image):
        lbm_load(self.ctx, image)

    def launches(self):
        return lbm_launch_count(self.ctx)

    def sync(self):
        lbm_sync(self.ctx)


class _Instance(Lbm):
    """A context owned by a batch (lbm_batch_instance): every Lbm method works
    on it; closing it does nothing."""

    def __init__(self, ctx, nx, ny, stream):
        self.nx, self.ny, self.stream, self._state, self.ctx = nx, ny, stream, None, ctx

    def close(self):
        self.ctx = None


class LbmBatch:
    """Many instances advanced by the batched persistent kernel (lbm_batch_*).
    ``instances`` as for lbm_batch_create; ``cfg`` an lbm_batch_config or None;
    ``stream`` a torch.cuda.Stream, a raw handle, or None."""

    def __init__(self, instances, cfg=None, stream=None):
        self.stream = stream
        self.b = lbm_batch_create(instances, cfg, stream)
        self.instances = [_Instance(lbm_batch_instance(self.b, i), d["nx"], d["ny"], stream)
                          for i, d in enumerate(instances)]

    def __len__(self):
        return len(self.instances)

    def __getitem__(self, i):
        return self.instances[i]

    def step(self, n=1):
        lbm_batch_step(self.b, n)

    def status(self):
        return lbm_batch_status(self.b)

    def contact_angles(self, wall=0):
        return lbm_batch_contact_angles(self.b, wall)

    def autotune(self, trial_steps=20):
        return lbm_batch_autotune(self.b, trial_steps)

    config = property(lambda self: lbm_batch_get_config(self.b))

    def set_config(self, cfg):
        lbm_batch_set_config(self.b, cfg)

    def plan(self):
        return lbm_batch_get_plan(self.b)

    def launches(self):
        return lbm_batch_launch_count(self.b)

    def node_updates(self) -> np.ndarray:
        """Fluid-node updates computed per instance (frozen instances stop counting)."""
        return lbm_batch_node_updates(self.b)

    def close(self):
        if getattr(self, "b", None):
            for inst in self.instances:
                inst.close()
            lbm_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
