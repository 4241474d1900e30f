"""FP64 CPU oracle for the pseudo-potential D2Q9 step with geometric wetting.

Test infrastructure only: the independent checker of the CUDA library.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may import this package.  It shares no code with
``paper_1501_05430_gb300``; the C source ``lbm_oracle.c`` is compiled here with
gcc (``-O2 -ffp-contract=off``, no fast-math) so that its arithmetic happens in
the written order.

``autodiff.py`` restates the same step with PyTorch CPU ops in FP64 so that
torch autograd gives the exact derivative of the oracle's step (the reference
for the adjoint kernels); it is pinned to the C step and to its finite
differences in ``tests/test_oracle_autodiff.py``.

Parity unpinned: nothing.  Every function is pinned in ``tests/test_oracle_*``
(see the header of each C function for what pins it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

EOS_CS = 0
EOS_PIECEWISE = 1
GEOMETRIC = 0
MARTYS_CHEN = 1


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into liblbm_oracle.so next to it (gcc, no FMA)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        DP = ctypes.POINTER(ctypes.c_double)
        IP = ctypes.POINTER(ctypes.c_int)
        sig = {
            "orc_pressure": (D, [I, DP, D, D]),
            "orc_psi_U": (None, [I, DP, D, D, DP, DP]),
            "orc_cs_critical": (I, [DP, DP, DP]),
            "orc_coexistence": (I, [I, DP, D, DP, DP]),
            "orc_piecewise_breakpoints": (I, [D, D, D, D, D, DP, DP]),
            "orc_rho_max": (D, [I, DP, D, D]),
            "orc_ghost": (D, [D, D, D, D, D, D, I, D]),
            "orc_collide": (None, [DP, D, D, D, D, D, D, DP, DP]),
            "orc_feq": (None, [D, D, D, DP]),
            "orc_create": (P, [I, I, I, I, I, DP, D, DP, I, I, DP, D, D]),
            "orc_destroy": (None, [P]),
            "orc_set_rho": (None, [P, DP]),
            "orc_set_f": (None, [P, DP]),
            "orc_get_f": (None, [P, DP]),
            "orc_step": (I, [P, I]),
            "orc_get_fields": (None, [P, DP, DP, DP, DP, DP, DP, DP, DP]),
            "orc_get_macro": (None, [P, DP, DP, DP]),
            "orc_mass": (D, [P]),
            "orc_contact_angle_field": (I, [DP, I, I, I, I, I, D, DP, DP, DP, IP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _darr(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


@dataclass(frozen=True)
class Eos:
    """Equation of state: Carnahan-Starling (a, b, R) or the Eq. 11 piecewise EOS."""
    kind: int = EOS_CS
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    theta_v: float = 0.0
    theta_m: float = 0.0
    theta_l: float = 0.0
    rho1: float = 0.0
    rho2: float = 0.0

    def vec(self) -> np.ndarray:
        return _darr([self.a, self.b, self.R, self.theta_v, self.theta_m,
                      self.theta_l, self.rho1, self.rho2])


def carnahan_starling(a=1.0, b=4.0, R=1.0) -> Eos:
    return Eos(EOS_CS, a, b, R)


def piecewise(theta_v, theta_m, theta_l, rho1, rho2) -> Eos:
    return Eos(EOS_PIECEWISE, 0.0, 0.0, 0.0, theta_v, theta_m, theta_l, rho1, rho2)


def pressure(eos: Eos, T: float, rho: float) -> float:
    return _load().orc_pressure(eos.kind, _dp(eos.vec()), T, rho)


def psi_U(eos: Eos, T: float, rho: float):
    p, u = ctypes.c_double(), ctypes.c_double()
    _load().orc_psi_U(eos.kind, _dp(eos.vec()), T, rho, ctypes.byref(p), ctypes.byref(u))
    return p.value, u.value


def cs_critical(eos: Eos):
    tc, rc = ctypes.c_double(), ctypes.c_double()
    _load().orc_cs_critical(_dp(eos.vec()), ctypes.byref(tc), ctypes.byref(rc))
    return tc.value, rc.value


def coexistence(eos: Eos, T: float = 0.0):
    rv, rl = ctypes.c_double(), ctypes.c_double()
    st = _load().orc_coexistence(eos.kind, _dp(eos.vec()), T, ctypes.byref(rv), ctypes.byref(rl))
    if st != 0:
        raise ValueError("no coexistence for these EOS parameters")
    return rv.value, rl.value


def piecewise_breakpoints(rho_v, rho_l, theta_v, theta_m, theta_l):
    r1, r2 = ctypes.c_double(), ctypes.c_double()
    st = _load().orc_piecewise_breakpoints(rho_v, rho_l, theta_v, theta_m, theta_l,
                                           ctypes.byref(r1), ctypes.byref(r2))
    if st != 0:
        raise ValueError("Eqs. 12-13 have no solution for these slopes")
    return r1.value, r2.value


def rho_max(eos: Eos, T: float, rho_l: float) -> float:
    return _load().orc_rho_max(eos.kind, _dp(eos.vec()), T, rho_l)


def ghost(r_im1_1, r_ip1_1, r_i1, r_i2, c, cot, n_iter, rho_max_=np.finfo(np.float64).max):
    return _load().orc_ghost(r_im1_1, r_ip1_1, r_i1, r_i2, c, cot, n_iter, rho_max_)


def collide(f, rho, Fx, Fy, Qxx, Qyy, Qxy, s):
    f = _darr(f)
    s = _darr(s)
    out = np.zeros(9)
    _load().orc_collide(_dp(f), rho, Fx, Fy, Qxx, Qyy, Qxy, _dp(s), _dp(out))
    return out


def feq(rho, vx, vy):
    out = np.zeros(9)
    _load().orc_feq(rho, vx, vy, _dp(out))
    return out


def contact_angle_field(rho, wall, x0, x1, rho_mid):
    """Apparent angle of the droplet on ``wall`` in columns [x0, x1) of a
    density field rho[ny, nx]; returns (theta, H, L, xc) or raises."""
    rho = _darr(rho)
    ny, nx = rho.shape
    th, H, L = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    xc = ctypes.c_int()
    st = _load().orc_contact_angle_field(_dp(rho), nx, ny, wall, x0, x1, rho_mid,
                                         ctypes.byref(th), ctypes.byref(H), ctypes.byref(L),
                                         ctypes.byref(xc))
    if st != 0:
        raise ValueError("no contact line found in the region")
    return th.value, H.value, L.value, xc.value


class Sim:
    """Two-array FP64 simulation: f[9, ny, nx], rows 0 and ny-1 solid if walls."""

    def __init__(self, nx, ny, eos: Eos, T, tau=1.0, walls=True, A=-0.6, kappa=0.5, G_w=0.0,
                 n_iter=4, wetting=GEOMETRIC, theta=None, rates=None, rho_max_=None, ghost_max=0.0):
        self.nx, self.ny, self.eos, self.T = nx, ny, eos, T
        lib = _load()
        if rates is None:
            s = 1.0 / tau
            rates = dict(s_rho=0.0, s_e=s, s_eps=s, s_j=s, s_q=s, s_nu=s)
        self.rates = rates
        params = _darr([A, kappa, G_w, rates["s_rho"], rates["s_e"], rates["s_eps"],
                        rates["s_j"], rates["s_q"], rates["s_nu"]])
        if theta is None:
            theta = np.full((ny, nx), np.pi / 2)
        th = _darr(np.broadcast_to(theta, (ny, nx)))
        if rho_max_ is None:
            rho_max_ = np.finfo(np.float64).max
        w = 1 if walls else 0
        self._h = lib.orc_create(nx, ny, w, w, eos.kind, _dp(eos.vec()), T, _dp(params),
                                 n_iter, wetting, _dp(th), rho_max_, ghost_max)
        self._lib = lib

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_rho(self, rho):
        rho = _darr(rho)
        assert rho.shape == (self.ny, self.nx)
        self._lib.orc_set_rho(self._h, _dp(rho))

    def set_f(self, f):
        f = _darr(f)
        assert f.shape == (9, self.ny, self.nx)
        self._lib.orc_set_f(self._h, _dp(f))

    def get_f(self):
        out = np.zeros((9, self.ny, self.nx))
        self._lib.orc_get_f(self._h, _dp(out))
        return out

    def step(self, n=1) -> int:
        return self._lib.orc_step(self._h, n)

    def fields(self):
        shp = (self.ny, self.nx)
        arrs = [np.zeros(shp) for _ in range(8)]
        self._lib.orc_get_fields(self._h, *[_dp(a) for a in arrs])
        keys = ["rho", "psi", "U", "Fx", "Fy", "Qxx", "Qyy", "Qxy"]
        return dict(zip(keys, arrs))

    def macro(self):
        shp = (self.ny, self.nx)
        rho, ux, uy = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        self._lib.orc_get_macro(self._h, _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy

    def rho(self):
        return self.macro()[0]

    def mass(self) -> float:
        return self._lib.orc_mass(self._h)

    def contact_angle(self, wall, x0, x1, rho_mid):
        return contact_angle_field(self.rho(), wall, x0, x1, rho_mid)
