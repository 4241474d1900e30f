"""Seeded synthetic workloads (initial density fields, wall-angle fields and
droplet layouts) shared by the tests, the benchmark and the examples.

This module holds input recipes only -- no step of the lattice Boltzmann
method.  Coexistence densities and temperatures are passed in as numbers.

Workloads (the paper gives no grid sizes; these follow its setup of
Secs. 3.1 and 4.2 -- a semicircular droplet on the bottom wall -- at the
sizes of the benchmark configurations):
  plain_fp64       100 x 60, CS T/Tc = 0.8, tau = 1, R0 = 20, theta = 90 deg
  single_droplet   400 x 200, CS (a = 0.25) T/Tc = 0.6, tau = 0.8, R0 = 60, A = -0.9
  throughput       4096 x 2048, Table 1 EOS at ratio 1000, tau = 1, 12 droplets per wall
  throughput_cs    4096 x 2048, CS (a = 0.25) T/Tc = 0.5, tau = 0.6, A = -0.9, same layout
  batched          256 instances of {128x64 .. 512x256}, seeded theta, T/Tc, tau
  adjoint_case     256 x 128, CS T/Tc = 0.7, tau = 1, R0 = 40, per-wall-node theta
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

LATTICE_SHAPE = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def droplet_field(nx: int, ny: int, droplets, rho_v: float, rho_l: float, width: float = 3.0) -> np.ndarray:
    """rho[ny, nx] = max over droplets of (rho_l+rho_v)/2 - (rho_l-rho_v)/2 tanh(2 (r - R)/width).

    droplets = [(xc, R, where)]: where = 0 centres the droplet at y = 1 (on the
    bottom wall), 1 at y = ny-2 (top wall); a float is taken as the centre row
    of a free droplet.  x distances are periodic."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rho = np.full((ny, nx), rho_v, dtype=np.float64)
    for d in droplets:
        xc, R, w = d
        yc = 1.0 if (isinstance(w, (int, np.integer)) and w == 0) else (
            ny - 2.0 if (isinstance(w, (int, np.integer)) and w == 1) else float(w))
        dx = x - xc
        dx = dx - nx * np.floor((dx + 0.5 * nx) / nx)
        r = np.sqrt(dx * dx + (y - yc) * (y - yc))
        rho = np.maximum(rho, 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - R) / width))
    return rho


def theta_field(nx: int, ny: int, bottom, top=np.pi / 2) -> np.ndarray:
    """Wall angles in radians: row 0 from ``bottom``, row ny-1 from ``top``
    (scalars or length-nx arrays); interior rows hold pi/2 (never read)."""
    th = np.full((ny, nx), np.pi / 2)
    th[0] = bottom
    th[-1] = top
    return th


def random_distributions(rho: np.ndarray, seed: int, amp: float = 0.05, walls: bool = True) -> np.ndarray:
    """f[9, ny, nx]: a positive perturbation of rho times the D2Q9 rest shape,
    used as a generic non-equilibrium state in parity tests."""
    rng = np.random.default_rng(seed)
    ny, nx = rho.shape
    f = LATTICE_SHAPE[:, None, None] * rho[None] * (1.0 + amp * rng.uniform(-1.0, 1.0, (9, ny, nx)))
    if walls:
        f[:, 0] = 0.0
        f[:, -1] = 0.0
    return f


# Table 1 of the paper (Sec. 3.1): Eq. 11 parameters per density ratio with
# rho_v = 1 and rho_l = ratio, as (rho1, rho2, theta_v, theta_m, theta_l).
TABLE1 = {
    10: (1.122, 9.54, 0.25, -0.02, 0.3),
    100: (1.486, 94.65, 0.1633, -0.02, 0.33333),
    1000: (1.325, 971.1017, 0.2, -0.01, 0.33333),
}


def cs_eos(a=1.0, b=4.0, R=1.0) -> dict:
    return {"kind": "cs", "a": a, "b": b, "R": R}


def table1_eos(ratio: int) -> dict:
    r1, r2, tv, tm, tl = TABLE1[ratio]
    return {"kind": "pw", "theta_v": tv, "theta_m": tm, "theta_l": tl, "rho1": r1, "rho2": r2}


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    t_over_tc: float                 # Carnahan-Starling only
    tau: float
    steps: int
    droplets: List[Tuple[float, float, int]]
    theta: np.ndarray                # [ny, nx] radians
    regions: List[Tuple[int, int, int]] = field(default_factory=list)  # (wall, x0, x1)
    theta_set: List[float] = field(default_factory=list)              # degrees per region
    rates: dict = field(default_factory=dict)                          # MRT rates (0 -> 1/tau)
    width: float = 3.0
    eos: dict = field(default_factory=cs_eos)
    A: float = -0.6
    kappa: float = 0.5
    notes: str = ""


# MRT rates for the low-temperature Carnahan-Starling workloads: the viscous
# rate follows tau; energy, energy-square and heat-flux rates take values used
# with pseudo-potential MRT models at large density ratios.  With all rates
# equal to 1/tau (BGK) these cases blow up within 100 steps.
LOW_T_RATES = dict(s_e=0.8, s_eps=0.8, s_j=1.0, s_q=1.1)
# Eq. 9 mixing parameter for the Carnahan-Starling workloads.  The paper's
# A = -0.6 goes with its piecewise EOS (Table 1); with Carnahan-Starling it
# leaves the flat-interface vapour far below the Maxwell density (T/Tc = 0.6:
# 1.8e-5 against 3.1e-3) or without a vapour phase at all (T/Tc = 0.5: the
# vapour condenses onto the liquid until a node reaches zero density).  At
# A = -0.9 the method's flat-interface densities are Maxwell's within 11%
# (vapour) and 0.1% (liquid) from T/Tc = 0.5 to 0.8 (a = 0.25, b = 4, R = 1).
CS_A = -0.9


def plain_fp64() -> Workload:
    """Carnahan-Starling a = 1, b = 4, R = 1, T/Tc = 0.8, BGK tau = 1."""
    nx, ny = 100, 60
    return Workload("plain_fp64_100x60", nx, ny, 0.8, 1.0, 2000, [(50.0, 20.0, 0)],
                    theta_field(nx, ny, np.pi / 2, np.pi / 2), [(0, 0, nx)], [90.0])


def single_droplet(theta_deg: float = 90.0) -> Workload:
    """Carnahan-Starling at T/Tc = 0.6 (density ratio 132), tau = 0.8, A = CS_A,
    a droplet of radius 60 started as the circular cap at theta_deg with the
    semicircle's area.  The attraction is scaled to a = 0.25: with a = 1 the
    liquid has dp/drho = 0.57 > c_s^2 = 1/3, psi(rho) falls through the liquid
    and angles below 60 deg blow up; the coexistence densities do not depend
    on a."""
    nx, ny = 400, 200
    return Workload(f"single_droplet_400x200_theta{int(theta_deg)}", nx, ny, 0.6, 0.8, 20000,
                    [cap_droplet(200.0, 60.0, theta_deg, 0, ny)], theta_field(nx, ny, np.deg2rad(theta_deg), np.pi / 2),
                    [(0, 0, nx)], [theta_deg], dict(LOW_T_RATES), eos=cs_eos(a=0.25), A=CS_A)


def _cap_base(r0: float, theta_deg: float) -> float:
    """Base width of the 2-D circular cap at angle theta whose area equals a
    semicircle of radius r0 (the droplet's initial shape)."""
    t = np.deg2rad(theta_deg)
    R = r0 * np.sqrt(0.5 * np.pi / (t - np.sin(t) * np.cos(t)))
    return 2.0 * R * np.sin(t) if t <= 0.5 * np.pi else 2.0 * R


def cap_droplet(xc: float, r0: float, theta_deg: float, wall: int, ny: int) -> Tuple[float, float, float]:
    """(xc, R, yc) of the 2-D circular cap at angle theta whose area equals a
    semicircle of radius r0 on the bottom (wall 0) or top (wall 1) boundary
    row, in the droplet_field form with an explicit centre row."""
    t = np.deg2rad(theta_deg)
    R = r0 * np.sqrt(0.5 * np.pi / (t - np.sin(t) * np.cos(t)))
    yc = 1.0 - R * np.cos(t) if wall == 0 else (ny - 2.0) + R * np.cos(t)
    return (float(xc), float(R), float(yc))


def _wall_layout(rng, nx: int, per_wall: int, width: float):
    """Seeded droplets on both walls: radii from U[40, 120], theta from
    U[30, 150] deg; each droplet gets a wall slot as wide as the base of the cap
    it relaxes to at its angle (same area as the initial semicircle) plus a
    margin, all radii scaled by one common factor so that the slots fill the
    wall, theta constant on each slot.  Returns (droplets, bottom, top, regions,
    theta_set, scales, per_wall) with per_wall lowered where the wall is too
    short for it."""
    margin = 8.0 + 2.0 * width
    per_wall = max(1, min(per_wall, int(nx // (margin + 20.0))))
    droplets, regions, theta_set, scales = [], [], [], []
    bottom = np.full(nx, np.pi / 2)
    top = np.full(nx, np.pi / 2)
    for wall in (0, 1):
        r = rng.uniform(40.0, 120.0, per_wall)
        th = rng.uniform(30.0, 150.0, per_wall)
        need = np.array([_cap_base(r[k], th[k]) for k in range(per_wall)])
        s = min(1.0, (nx - margin * per_wall) / need.sum())
        scales.append(s)
        r = r * s
        slot = need * s + margin
        slot *= nx / slot.sum()
        x0 = 0.0
        for k in range(per_wall):
            lo, hi = x0, x0 + slot[k]
            xc = 0.5 * (lo + hi)
            a, b = int(np.ceil(lo)), int(np.ceil(hi)) if k < per_wall - 1 else nx
            (bottom if wall == 0 else top)[a:b] = np.deg2rad(th[k])
            droplets.append((float(xc), float(r[k]), wall))
            regions.append((wall, a, b))
            theta_set.append(float(th[k]))
            x0 = hi
    return droplets, bottom, top, regions, theta_set, scales, per_wall


def throughput(seed: int = 1234, nx: int = 4096, ny: int = 2048, per_wall: int = 12) -> Workload:
    """Large density ratio with the paper's own model: the Eq. 11 EOS of
    Table 1 at ratio 1000 with the paper's relaxation (all rates 1, tau = 1),
    A = -0.6, kappa = 0.5, tanh interfaces of width 10, theta ~ U[30, 150] deg
    per droplet, radii drawn from U[40, 120] (see _wall_layout).

    12 droplets per wall (24 in all): with 32 per wall (64) the slots are too
    narrow at ratio 1000 and the run blows up within a few hundred steps; 16
    per wall lasts about 4900 steps, 12 per wall the full 5000."""
    rng = np.random.default_rng(seed)
    width = 10.0
    droplets, bottom, top, regions, theta_set, scales, pw = _wall_layout(rng, nx, per_wall, width)
    return Workload(f"throughput_{nx}x{ny}_{2 * pw}drops_ratio1000", nx, ny, 0.0, 1.0, 5000, droplets,
                    theta_field(nx, ny, bottom, top), regions, theta_set, {}, width=width,
                    eos=table1_eos(1000),
                    notes=f"radius scale factors per wall {scales[0]:.4f}, {scales[1]:.4f}")


def throughput_cs(seed: int = 1234, nx: int = 4096, ny: int = 2048, per_wall: int = 12) -> Workload:
    """Large density ratio with the Carnahan-Starling EOS: T/Tc = 0.5 (density
    ratio 724), tau = 0.6 with the MRT rates of LOW_T_RATES (so the fused
    kernel runs its general-rate collision), A = CS_A, kappa = 0.5, the wall
    layout of ``throughput`` (same seed: same radii, angles and slots), each
    droplet started as the circular cap at its angle with the area of its
    semicircle, tanh interfaces of width 10.  a = 0.25 (the coexistence
    densities depend only on b and T/Tc; with a = 1 the liquid's dp/drho
    exceeds c_s^2 and every run blows up within 500 steps)."""
    rng = np.random.default_rng(seed)
    width = 10.0
    droplets, bottom, top, regions, theta_set, scales, pw = _wall_layout(rng, nx, per_wall, width)
    caps = [cap_droplet(xc, r, th, wall, ny) for (xc, r, wall), th in zip(droplets, theta_set)]
    return Workload(f"throughput_cs_{nx}x{ny}_{2 * pw}drops_T0.5", nx, ny, 0.5, 0.6, 5000, caps,
                    theta_field(nx, ny, bottom, top), regions, theta_set, dict(LOW_T_RATES), width=width,
                    eos=cs_eos(a=0.25), A=CS_A,
                    notes=f"radius scale factors per wall {scales[0]:.4f}, {scales[1]:.4f}; caps of the "
                          f"semicircles' areas")


def batched(seed: int = 42, count: int = 256, width: float = 3.0):
    """Independent droplet instances: size uniform over {128x64, 256x128,
    384x192, 512x256}, theta ~ U(20, 160) deg, T/Tc in {0.5, 0.6, 0.7, 0.8},
    tau ~ U[0.6, 1.0], a droplet of radius R0 = nx/4 on the bottom wall,
    started as the circular cap at its angle with the area of the semicircle
    of radius R0 (a semicircle far from its angle sheds its excess energy in a
    transient that blows up 10 of the 256 at T/Tc = 0.5).  Carnahan-Starling with
    a = 0.25 (the coexistence densities depend only on b and T/Tc), A = CS_A and
    the low-temperature MRT rates below T/Tc = 0.7, as for single_droplet."""
    rng = np.random.default_rng(seed)
    sizes = [(128, 64), (256, 128), (384, 192), (512, 256)]
    out = []
    for i in range(count):
        nx, ny = sizes[rng.integers(0, 4)]
        th = rng.uniform(20.0, 160.0)
        tr = [0.5, 0.6, 0.7, 0.8][rng.integers(0, 4)]
        tau = rng.uniform(0.6, 1.0)
        out.append(Workload(f"batch{i}_{nx}x{ny}", nx, ny, tr, tau, 10000,
                            [cap_droplet(nx / 2.0, nx / 4.0, th, 0, ny)],
                            theta_field(nx, ny, np.deg2rad(th)), [(0, 0, nx)], [th],
                            dict(LOW_T_RATES) if tr < 0.7 else {}, width=width, eos=cs_eos(a=0.25), A=CS_A))
    return out


def adjoint_case(seed: int = 7, target_seed: int = 8) -> dict:
    """Wall-angle inversion case: 256 x 128, Carnahan-Starling (a = 1, b = 4,
    R = 1) at T/Tc = 0.7, tau = 1, a droplet of radius 40 centred on the bottom
    wall, 2000 steps with a checkpoint every 100.  The parameters are the 256
    bottom-wall angles, seeded U(45, 135) deg (``theta``); the target profile
    comes from the same run at a second seeded field (``theta_target``); the
    top wall stays at 90 deg.  The loss is
        L = sum_i (h_i - h*_i)^2 + (W - W*)^2,
        h_i = sum_{y=1}^{ny-2} phi(i, y),  W = sum_i phi(i, 1),
        phi = (rho - rho_v) / (rho_l - rho_v)
    with rho_v, rho_l the coexistence densities at the nominal T (held fixed)."""
    nx, ny = 256, 128
    th = np.random.default_rng(seed).uniform(np.deg2rad(45.0), np.deg2rad(135.0), nx)
    tt = np.random.default_rng(target_seed).uniform(np.deg2rad(45.0), np.deg2rad(135.0), nx)
    return dict(nx=nx, ny=ny, t_over_tc=0.7, tau=1.0, eos=cs_eos(), droplet=(nx / 2.0, 40.0, 0), width=3.0,
                theta=th, theta_target=tt, steps=2000, checkpoint_every=100)


def profile(rho: np.ndarray, rho_v: float, rho_l: float):
    """(h [nx], W) of a density field: h_i = sum over the fluid rows of phi,
    W = sum over the boundary row of phi, phi = (rho - rho_v) / (rho_l - rho_v)."""
    phi = (rho - rho_v) / (rho_l - rho_v)
    return phi[1:-1].sum(0), float(phi[1].sum())


def profile_loss_grad(rho: np.ndarray, h_target: np.ndarray, W_target: float, rho_v: float, rho_l: float):
    """(L, dL/drho [ny, nx]) of the height / base-width profile loss of adjoint_case."""
    h, W = profile(rho, rho_v, rho_l)
    L = float(((h - h_target) ** 2).sum() + (W - W_target) ** 2)
    g = np.zeros_like(rho)
    g[1:-1] = 2.0 * (h - h_target)[None, :]
    g[1] += 2.0 * (W - W_target)
    return L, g / (rho_l - rho_v)
