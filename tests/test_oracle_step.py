"""Pins for the oracle's full timestep: hand-computed steps on tiny grids,
conservation laws, lattice symmetries, the flat-wall invariance that Fig. 8
reports for the geometric method, and the stability flag."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O

E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
WEQ = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
WINT = [Fr(0)] + [Fr(1, 3)] * 4 + [Fr(1, 12)] * 4
BIG = np.finfo(np.float64).max
CS = O.carnahan_starling()
TC, _ = O.cs_critical(CS)


def _hand_step(f, nx, ny, walls, theta_v):
    """One step in exact rationals, written from the textbook BGK (tau = 1)
    collision with Guo forcing and the potential-form force (A = 1, kappa = 0,
    so F = -sum_a w_a U(x+e_a) e_a with U = p - rho/3 = (theta_v - 1/3) rho on
    the first EOS branch).  With theta = 90 deg the ghost row equals row 2
    (the boundary row's second neighbour), and populations leaving into a
    solid row return reversed (half-way bounce-back)."""
    fluid = [y for y in range(ny) if not (walls and y in (0, ny - 1))]
    rho = {(x, y): sum(f[a][y][x] for a in range(9)) for x in range(nx) for y in fluid}
    if walls:
        for x in range(nx):
            rho[(x, 0)] = rho[(x, 2)]
            rho[(x, ny - 1)] = rho[(x, ny - 3)]
    U = {k: (theta_v - Fr(1, 3)) * v for k, v in rho.items()}
    out = [[[Fr(0)] * nx for _ in range(ny)] for _ in range(9)]
    for y in fluid:
        for x in range(nx):
            Fx = Fy = Fr(0)
            for a in range(1, 9):
                ex, ey = E[a]
                u = U[((x + ex) % nx, (y + ey) % ny)]
                Fx -= WINT[a] * u * ex
                Fy -= WINT[a] * u * ey
            r = rho[(x, y)]
            jx = sum(f[a][y][x] * E[a][0] for a in range(9))
            jy = sum(f[a][y][x] * E[a][1] for a in range(9))
            vx, vy = (jx + Fx / 2) / r, (jy + Fy / 2) / r
            for a in range(9):
                ex, ey = E[a]
                ev = ex * vx + ey * vy
                feq = WEQ[a] * r * (1 + 3 * ev + Fr(9, 2) * ev * ev - Fr(3, 2) * (vx * vx + vy * vy))
                guo = WEQ[a] * (3 * ((ex - vx) * Fx + (ey - vy) * Fy) + 9 * ev * (ex * Fx + ey * Fy))
                fs = feq + guo / 2
                yt = (y + ey) % ny
                if walls and yt in (0, ny - 1):
                    out[OPP[a]][y][x] = fs
                else:
                    out[a][yt][(x + ex) % nx] = fs
    return out


@pytest.mark.parametrize("nx,ny,walls", [(4, 4, False), (4, 6, True), (5, 7, True)])
def test_hand_computed_single_step(nx, ny, walls):
    rng = np.random.default_rng(20 + nx + ny)
    f = [[[Fr(int(rng.integers(20, 60)), 997) for _ in range(nx)] for _ in range(ny)] for _ in range(9)]
    if walls:
        for a in range(9):
            f[a][0] = [Fr(0)] * nx
            f[a][ny - 1] = [Fr(0)] * nx
    theta_v = Fr(1, 4)
    eos = O.piecewise(0.25, -0.02, 0.3, 50.0, 60.0)
    s = O.Sim(nx, ny, eos, 0.0, tau=1.0, walls=walls, A=1.0, kappa=0.0, theta=np.pi / 2, rho_max_=BIG)
    s.set_f(np.array([[[float(v) for v in row] for row in plane] for plane in f]))
    assert s.step(1) == 0
    ref = _hand_step(f, nx, ny, walls, theta_v)
    ref = np.array([[[float(v) for v in row] for row in plane] for plane in ref])
    assert np.allclose(s.get_f(), ref, rtol=1e-13, atol=0)


def _droplet(nx, ny, xc, yc, R, rv, rl, W=3.0):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    dx = (x - xc + nx / 2) % nx - nx / 2
    r = np.hypot(dx, y - yc)
    return 0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2 * (r - R) / W)


def test_mass_conserved_with_walls():
    T = 0.8 * TC
    rv, rl = O.coexistence(CS, T)
    s = O.Sim(60, 40, CS, T, tau=1.0, walls=True, theta=np.deg2rad(60.0), rho_max_=O.rho_max(CS, T, rl))
    s.set_rho(_droplet(60, 40, 30, 1.0, 12, rv, rl))
    m0 = s.mass()
    assert s.step(300) == 0
    assert abs(s.mass() - m0) / m0 < 1e-13


def test_momentum_conserved_in_periodic_box():
    T = 0.8 * TC
    rv, rl = O.coexistence(CS, T)
    n = 32
    s = O.Sim(n, n, CS, T, tau=0.9, walls=False)
    s.set_rho(_droplet(n, n, 13.0, 17.0, 8, rv, rl))
    E_ = np.array(E, float)
    def mom():
        f = s.get_f()
        return np.einsum("ayx,ad->d", f, E_)
    p0 = mom()
    assert s.step(100) == 0
    # total force is zero in a periodic box, so sum_x (j + F) is unchanged
    assert np.abs(mom() - p0).max() < 1e-14 * s.mass()


PERM_ROT90 = [0, 2, 3, 4, 1, 6, 7, 8, 5]     # e_a rotated by +90 deg
PERM_FLIPX = [0, 3, 2, 1, 4, 6, 5, 8, 7]     # x -> -x
PERM_FLIPY = [0, 1, 4, 3, 2, 8, 7, 6, 5]     # y -> -y


def _rot90(f):
    n = f.shape[-1]
    out = np.empty_like(f)
    y, x = np.mgrid[0:n, 0:n]
    for a in range(9):
        out[PERM_ROT90[a]][x, (-y) % n] = f[a][y, x]
    return out


def _flipx(f):
    out = np.empty_like(f)
    for a in range(9):
        out[PERM_FLIPX[a]] = np.roll(f[a][:, ::-1], 1, axis=1)
    return out


def _flipy(f):
    out = np.empty_like(f)
    for a in range(9):
        out[PERM_FLIPY[a]] = f[a][::-1, :]
    return out


def _random_state(nx, ny, rv, rl, seed, walls):
    rng = np.random.default_rng(seed)
    base = _droplet(nx, ny, nx * 0.4, ny * 0.3 if not walls else 1.0, min(nx, ny) * 0.3, rv, rl)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = w[:, None, None] * base[None] * (1 + 0.05 * rng.uniform(-1, 1, (9, ny, nx)))
    if walls:
        f[:, 0] = 0
        f[:, -1] = 0
    return f


def test_rotation_equivariance_periodic():
    T = 0.8 * TC
    rv, rl = O.coexistence(CS, T)
    n = 20
    f0 = _random_state(n, n, rv, rl, 30, False)
    rates = dict(s_rho=0.0, s_e=1.1, s_eps=1.2, s_j=1.0, s_q=1.3, s_nu=1.4)
    a = O.Sim(n, n, CS, T, walls=False, rates=rates, kappa=0.6)
    b = O.Sim(n, n, CS, T, walls=False, rates=rates, kappa=0.6)
    a.set_f(f0)
    b.set_f(_rot90(f0))
    a.step(3)
    b.step(3)
    assert np.allclose(_rot90(a.get_f()), b.get_f(), rtol=1e-12, atol=1e-17)


@pytest.mark.parametrize("wetting", [O.GEOMETRIC, O.MARTYS_CHEN])
def test_reflection_equivariance_with_walls(wetting):
    T = 0.8 * TC
    rv, rl = O.coexistence(CS, T)
    nx, ny = 24, 14
    rng = np.random.default_rng(31)
    theta = np.deg2rad(rng.uniform(30, 150, (ny, nx)))
    f0 = _random_state(nx, ny, rv, rl, 32, True)
    kw = dict(walls=True, kappa=0.5, wetting=wetting, G_w=-0.8, rho_max_=O.rho_max(CS, T, rl))
    base = O.Sim(nx, ny, CS, T, theta=theta, **kw)
    base.set_f(f0)
    base.step(3)
    # x -> -x (theta field mirrored the same way)
    th_x = np.roll(theta[:, ::-1], 1, axis=1)
    mx = O.Sim(nx, ny, CS, T, theta=th_x, **kw)
    mx.set_f(_flipx(f0))
    mx.step(3)
    assert np.allclose(_flipx(base.get_f()), mx.get_f(), rtol=1e-12, atol=1e-17)
    # y -> -y swaps the two walls and their angles
    my = O.Sim(nx, ny, CS, T, theta=theta[::-1, :], **kw)
    my.set_f(_flipy(f0))
    my.step(3)
    assert np.allclose(_flipy(base.get_f()), my.get_f(), rtol=1e-12, atol=1e-17)


@pytest.mark.parametrize("theta_deg", [45.0, 135.0])
@pytest.mark.parametrize("phase", ["liquid", "vapour"])
def test_geometric_wall_keeps_bulk_flat(theta_deg, phase):
    """Fig. 8: with the geometric rule the density normal to the wall is flat.
    A uniform phase at rest between the walls is a fixed point for any theta."""
    T = 0.6 * TC
    rv, rl = O.coexistence(CS, T)
    r = rl if phase == "liquid" else rv
    s = O.Sim(16, 20, CS, T, tau=0.8, walls=True, theta=np.deg2rad(theta_deg), rho_max_=O.rho_max(CS, T, rl))
    s.set_rho(np.full((20, 16), r))
    assert s.step(200) == 0
    rho = s.rho()[1:-1]
    assert np.abs(rho - r).max() < 1e-13 * r


def test_martys_chen_distorts_near_wall_density():
    """Fig. 3: the fluid-solid force changes the density next to the wall."""
    T = 0.8 * TC
    rv, rl = O.coexistence(CS, T)
    s = O.Sim(16, 20, CS, T, tau=1.0, walls=True, wetting=O.MARTYS_CHEN, G_w=-0.5,
              rho_max_=O.rho_max(CS, T, rl))
    s.set_rho(np.full((20, 16), rl))
    assert s.step(400) == 0
    col = s.rho()[1:-1, 5]
    assert abs(col[0] - col[len(col) // 2]) > 1e-3 * rl


def test_instability_is_flagged():
    T = 0.8 * TC
    rv, rl = O.coexistence(CS, T)
    s = O.Sim(16, 12, CS, T, walls=True, rho_max_=O.rho_max(CS, T, rl))
    rho = np.full((12, 16), rl)
    rho[5, 7] = -0.1
    s.set_rho(rho)
    assert s.step(1) == -4


@pytest.mark.parametrize("rates", [None, dict(s_rho=0.0, s_e=0.8, s_eps=0.9, s_j=1.0, s_q=1.1, s_nu=1 / 0.9)])
def test_uniform_flow_is_a_fixed_point(rates):
    """A uniform density moving at a uniform velocity through a periodic box is
    a fixed point of the whole step: uniform psi and U give no force and no
    Eq. 16 source, the collision leaves the second-order equilibrium
    w_a rho [1 + 3 e.v + 9/2 (e.v)^2 - 3/2 v^2] unchanged at any rates, and
    streaming moves a uniform field onto itself -- which pins the
    velocity-dependent equilibrium moments (signs included)."""
    T = 0.8 * TC
    rv, _ = O.coexistence(CS, T)
    v = np.array([0.05, -0.03])
    e = np.array(E, float)
    w = np.array([float(x) for x in WEQ])
    ev = e @ v
    feq = w * rv * (1 + 3 * ev + 4.5 * ev ** 2 - 1.5 * (v @ v))
    nx, ny = 12, 8
    f0 = np.broadcast_to(feq[:, None, None], (9, ny, nx)).copy()
    kw = {} if rates is None else dict(rates=rates)
    s = O.Sim(nx, ny, CS, T, tau=0.9, walls=False, **kw)
    s.set_f(f0)
    assert s.step(3) == 0
    f = s.get_f()
    s.close()
    assert np.abs(f - f0).max() < 1e-14 * f0.max()
