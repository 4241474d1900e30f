"""Seeded synthetic workloads (initial density fields, wall-angle fields and
droplet layouts) shared by the tests, the benchmark and the examples.

This module holds input recipes only -- no step of the lattice Boltzmann
method.  Coexistence densities and temperatures are passed in as numbers.

Workloads (the paper gives no grid sizes; these follow its setup of
Secs. 3.1 and 4.2 -- a semicircular droplet on the bottom wall -- at the
sizes of the benchmark configurations):
  plain_fp64       100 x 60, CS T/Tc = 0.8, tau = 1, R0 = 20, theta = 90 deg
  single_droplet   400 x 200, CS T/Tc = 0.6, tau = 0.8, R0 = 60, theta in {30..150}
  throughput       4096 x 2048, CS T/Tc = 0.5, tau = 0.6, 32 droplets per wall
  batched          256 instances of {128x64 .. 512x256}, seeded theta, T/Tc, tau
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


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    t_over_tc: float
    tau: float
    steps: int
    droplets: List[Tuple[float, float, int]]
    theta: np.ndarray                # [ny, nx] radians
    regions: List[Tuple[int, int, int]] = field(default_factory=list)  # (wall, x0, x1)
    theta_set: List[float] = field(default_factory=list)              # degrees per region
    rates: dict = field(default_factory=dict)                          # MRT rates (0 -> 1/tau)
    width: float = 3.0
    notes: str = ""


# MRT rates for the low-temperature workloads: the viscous rate follows tau;
# energy, energy-square and heat-flux rates take values used with
# pseudo-potential MRT models at large density ratios.  With all rates equal
# to 1/tau (BGK) these cases blow up within 100 steps.
LOW_T_RATES = dict(s_e=0.8, s_eps=0.8, s_j=1.0, s_q=1.1)


def plain_fp64() -> Workload:
    nx, ny = 100, 60
    return Workload("plain_fp64_100x60", nx, ny, 0.8, 1.0, 2000, [(50.0, 20.0, 0)],
                    theta_field(nx, ny, np.pi / 2, np.pi / 2), [(0, 0, nx)], [90.0])


def single_droplet(theta_deg: float = 90.0) -> Workload:
    nx, ny = 400, 200
    return Workload(f"single_droplet_400x200_theta{int(theta_deg)}", nx, ny, 0.6, 0.8, 20000,
                    [(200.0, 60.0, 0)], theta_field(nx, ny, np.deg2rad(theta_deg), np.pi / 2),
                    [(0, 0, nx)], [theta_deg], dict(LOW_T_RATES))


def throughput(seed: int = 1234, nx: int = 4096, ny: int = 2048, per_wall: int = 32) -> Workload:
    """Droplets on both walls.  64 droplets with radii U[40, 120] do not fit on
    one 4096-node wall (they need ~10^4 nodes), so each wall carries half of
    them, radii scaled by one common factor so that sum(2 r + 8) <= nx."""
    rng = np.random.default_rng(seed)
    droplets, regions, theta_set = [], [], []
    bottom = np.full(nx, np.pi / 2)
    top = np.full(nx, np.pi / 2)
    scales = []
    for wall in (0, 1):
        r = rng.uniform(40.0, 120.0, per_wall)
        s = min(1.0, (nx - 8.0 * per_wall) / (2.0 * r.sum()))
        scales.append(s)
        r = r * s
        free = nx - 2.0 * r.sum()
        gaps = rng.dirichlet(np.ones(per_wall)) * free
        th = rng.uniform(30.0, 150.0, per_wall)
        cursor = 0.0
        centres = []
        for k in range(per_wall):
            cursor += gaps[k]
            centres.append(cursor + r[k])
            cursor += 2.0 * r[k]
        centres = np.array(centres)
        # region bounds halfway between neighbouring droplets (periodic)
        bounds = []
        for k in range(per_wall):
            right_edge = centres[k] + r[k]
            nxt_left = centres[(k + 1) % per_wall] - r[(k + 1) % per_wall] + (nx if k == per_wall - 1 else 0)
            bounds.append(0.5 * (right_edge + nxt_left))
        for k in range(per_wall):
            lo = bounds[k - 1] - (nx if k == 0 else 0)
            hi = bounds[k]
            x0, x1 = int(np.ceil(lo)), int(np.ceil(hi))
            xs = np.arange(x0, x1) % nx
            (bottom if wall == 0 else top)[xs] = np.deg2rad(th[k])
            droplets.append((float(centres[k]), float(r[k]), wall))
            if x0 >= 0 and x1 <= nx:
                regions.append((wall, x0, x1))
                theta_set.append(float(th[k]))
    return Workload(f"throughput_{nx}x{ny}_{2 * per_wall}drops", nx, ny, 0.5, 0.6, 5000, droplets,
                    theta_field(nx, ny, bottom, top), regions, theta_set, dict(LOW_T_RATES),
                    notes=f"radius scale factors per wall {scales[0]:.4f}, {scales[1]:.4f}")


def batched(seed: int = 42, count: int = 256):
    """Independent instances: size uniform over four classes, theta ~ U(20, 160) deg,
    T/Tc in {0.5, 0.6, 0.7, 0.8}, tau ~ U[0.6, 1.0], R0 = nx/4."""
    rng = np.random.default_rng(seed)
    sizes = [(128, 64), (256, 128), (384, 192), (512, 256)]
    out = []
    for i in range(count):
        nx, ny = sizes[rng.integers(0, 4)]
        th = rng.uniform(20.0, 160.0)
        tr = [0.5, 0.6, 0.7, 0.8][rng.integers(0, 4)]
        tau = rng.uniform(0.6, 1.0)
        out.append(Workload(f"batch{i}_{nx}x{ny}", nx, ny, tr, tau, 10000, [(nx / 2.0, nx / 4.0, 0)],
                            theta_field(nx, ny, np.deg2rad(th)), [(0, 0, nx)], [th],
                            dict(LOW_T_RATES) if tr < 0.7 else {}))
    return out
