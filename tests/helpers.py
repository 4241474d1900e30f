"""Test helpers: build an oracle simulation and a liblbm context with the
same parameters, from the seeded workloads of paper_1501_05430_gb300.inputs."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1501_05430_gb300 import inputs as I
from paper_1501_05430_gb300 import lbm as L

BIG = np.finfo(np.float64).max


def cs_T(t_over_tc: float, a=1.0, b=4.0, R=1.0) -> float:
    tc, _ = O.cs_critical(O.carnahan_starling(a, b, R))
    return t_over_tc * tc


def resolve_rates(tau, rates=None):
    inv = 1.0 / tau
    r = dict(s_rho=0.0, s_e=inv, s_eps=inv, s_j=inv, s_q=inv, s_nu=inv)
    for k, v in (rates or {}).items():
        if v:
            r[k] = v
    return r


class Case:
    """The inputs of one simulation on both sides: the oracle Sim and the
    liblbm parameters (lbm_params, EOS, T, tau, theta) built from the same
    numbers.

    The library derives its own density bounds (rho_max: ghost clamp and
    instability bound; rho_mid: the angle contour) from the EOS, as a user's
    context does; the oracle's values go into lbm_params only with
    oracle_bounds=True."""

    def __init__(self, nx, ny, *, t_over_tc=0.8, tau=1.0, eos="cs", pw=None, theta=np.pi / 2, walls=True,
                 A=-0.6, kappa=0.5, G_w=0.0, n_iter=4, wetting=0, rates=None, precision=64,
                 kernel=L.LBM_KERNEL_AUTO, check_every=0, oracle_bounds=False):
        self.nx, self.ny, self.tau, self.walls = nx, ny, tau, walls
        if eos == "pw":
            eos = dict(kind="pw", theta_v=pw[0], theta_m=pw[1], theta_l=pw[2], rho1=pw[3], rho2=pw[4])
        elif eos == "cs":
            eos = dict(kind="cs", a=1.0, b=4.0, R=1.0)
        if eos["kind"] == "cs":
            self.oeos = O.carnahan_starling(eos["a"], eos["b"], eos["R"])
            self.geos = L.carnahan_starling(eos["a"], eos["b"], eos["R"])
            self.T = t_over_tc * O.cs_critical(self.oeos)[0]
            self.rho_v, self.rho_l = O.coexistence(self.oeos, self.T)
        else:
            args = (eos["theta_v"], eos["theta_m"], eos["theta_l"], eos["rho1"], eos["rho2"])
            self.oeos = O.piecewise(*args)
            self.geos = L.piecewise(*args)
            self.T = 0.0
            self.rho_v, self.rho_l = O.coexistence(self.oeos)
        self.rho_max = O.rho_max(self.oeos, self.T, self.rho_l)
        self.rho_mid = 0.5 * (self.rho_v + self.rho_l)
        r = resolve_rates(tau, rates)
        self.theta = np.broadcast_to(np.asarray(theta, dtype=float), (ny, nx)).copy()
        self.orc = O.Sim(nx, ny, self.oeos, self.T, tau=tau, walls=walls, A=A, kappa=kappa, G_w=G_w,
                         n_iter=n_iter, wetting=wetting, theta=self.theta, rates=r, rho_max_=self.rho_max)
        self.params = L.lbm_params_default(A=A, kappa=kappa, G_w=G_w, n_iter=n_iter, wetting=wetting,
                                           precision=precision, kernel=kernel, s_e=r["s_e"], s_eps=r["s_eps"],
                                           s_j=r["s_j"], s_q=r["s_q"], s_nu=r["s_nu"], check_every=check_every)
        if oracle_bounds:
            self.params.rho_max = min(self.rho_max, 1e300)
            self.params.rho_mid = self.rho_mid

    def desc(self):
        """Instance description for lbm_batch_create (FP32)."""
        p = L.lbm_params()
        ctypes_copy(p, self.params)
        p.precision = 32
        return dict(nx=self.nx, ny=self.ny, eos=self.geos, T=self.T, tau=self.tau, theta=self.theta, params=p)


def ctypes_copy(dst, src):
    for name, _ in src._fields_:
        setattr(dst, name, getattr(src, name))


class Pair(Case):
    """An oracle Sim and a GPU context with identical inputs."""

    def __init__(self, nx, ny, *, torch_state=False, stream=None, **kw):
        super().__init__(nx, ny, **kw)
        self.gpu = L.Lbm(nx, ny, self.geos, self.T, self.tau, theta=self.theta, walls=self.walls,
                         params=self.params, stream=stream, torch_state=torch_state)

    def set_rho(self, rho):
        self.orc.set_rho(rho)
        self.gpu.set_rho(rho)

    def set_f(self, f):
        self.orc.set_f(f)
        self.gpu.set_f(f)

    def step(self, n):
        so = self.orc.step(n)
        self.gpu.step(n)
        return so

    def close(self):
        self.gpu.close()
        self.orc.close()


def droplet_pair(w: I.Workload, precision=64, kernel=L.LBM_KERNEL_AUTO, **kw) -> Pair:
    p = Pair(w.nx, w.ny, t_over_tc=w.t_over_tc, tau=w.tau, theta=w.theta, rates=w.rates, precision=precision,
             kernel=kernel, eos=w.eos, A=w.A, kappa=w.kappa, **kw)
    p.set_rho(I.droplet_field(w.nx, w.ny, w.droplets, p.rho_v, p.rho_l, w.width))
    return p
