"""Workload -> liblbm arguments: the EOS, temperature, parameters and initial
density field of an ``inputs.Workload`` for lbm_create / lbm_batch_create.

Argument marshalling only; coexistence densities come from the library's own
host solver (lbm_coexistence)."""
from __future__ import annotations

from . import inputs as I
from . import lbm as L


def lib_eos(w: I.Workload):
    """(lbm_eos, T) of a workload."""
    e = w.eos
    if e["kind"] == "cs":
        eos = L.carnahan_starling(e["a"], e["b"], e["R"])
        return eos, w.t_over_tc * L.lbm_eos_critical(eos)[0]
    return L.piecewise(e["theta_v"], e["theta_m"], e["theta_l"], e["rho1"], e["rho2"]), 0.0


def lib_params(w: I.Workload, precision: int = 32, kernel: int = L.LBM_KERNEL_AUTO, check_every: int = 0):
    r = w.rates
    return L.lbm_params_default(precision=precision, kernel=kernel, check_every=check_every, A=w.A,
                                kappa=w.kappa, s_e=r.get("s_e", 0.0), s_eps=r.get("s_eps", 0.0),
                                s_j=r.get("s_j", 0.0), s_q=r.get("s_q", 0.0))


def initial_rho(w: I.Workload):
    """The workload's droplet field at the library's coexistence densities."""
    eos, T = lib_eos(w)
    rv, rl = L.lbm_coexistence(eos, T)
    return I.droplet_field(w.nx, w.ny, w.droplets, rv, rl, w.width)


def instance_desc(w: I.Workload) -> dict:
    """lbm_batch_create description of a workload (FP32)."""
    eos, T = lib_eos(w)
    return dict(nx=w.nx, ny=w.ny, eos=eos, T=T, tau=w.tau, theta=w.theta, params=lib_params(w))


def rho_mid(w: I.Workload) -> float:
    eos, T = lib_eos(w)
    rv, rl = L.lbm_coexistence(eos, T)
    return 0.5 * (rv + rl)
