"""Differentiable restatement of the oracle's timestep (FP64, PyTorch CPU ops),
used only by the tests as the reference for gradients: torch autograd through
this function gives the exact derivative of the step the C oracle computes.

TEST INFRASTRUCTURE ONLY -- like the rest of oracle/, nothing on the product
path imports it.  It shares no code with the CUDA library, and its forward is
pinned to the C oracle (tests/test_oracle_autodiff.py: equal distributions to
rounding on every model variant), so autograd here differentiates the same
function.

One step, in the order of Eq. 1 and Sec. 2 (the readings are those of the C
oracle):
  rho = sum_a f_a; U = p(rho) - rho/3, psi = sqrt(max(0, -2U))      Eqs. 10-11
  ghost rows: n_iter evaluations of Eq. 20 with the square root (Eq. 21),
              Eq. 19 for n_iter = 0, clamped to [0, ghost_max];
              psi = U = 0 at and above rho_max                     Eqs. 19-21
  F = -A sum w U(x+e) e - (1-A) G psi(x) sum w psi(x+e) e (G = -1)   Eq. 9
      (+ -G_w psi(x) sum w S(x+e) e for Martys-Chen)               Eq. 14
  Q = (kappa G/2) [(1-A) psi sum w (psi_a - psi) ee + (A/2) sum w (psi_a^2 - psi^2) ee]   Eq. 17
  MRT collision with Guo forcing and the Eq. 16 source             Eqs. 2-6, 15-16
  push streaming, x periodic, half-way bounce-back at solid rows  Eq. 1

Derivative conventions where the function has a kink: d sqrt(s)/ds := 0 at
s = 0 (psi of a node with U >= 0, and the Eq. 21 root when its argument
vanishes); d|a|/da := 0 at a = 0; clamped ghost densities pass no gradient.
"""
from __future__ import annotations

import math

import torch

EX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
EY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
OPP = (0, 3, 4, 1, 2, 7, 8, 5, 6)
WGT = (0.0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 1 / 12, 1 / 12, 1 / 12, 1 / 12)
G = -1.0

# MRT basis (rho, e, eps, jx, qx, jy, qy, pxx, pxy) as polynomials of (ex, ey)
def _basis():
    rows = []
    for ex, ey in zip(EX, EY):
        e2 = ex * ex + ey * ey
        rows.append([1, -4 + 3 * e2, 4 - 21 * e2 / 2 + 9 * e2 * e2 / 2, ex, (-5 + 3 * e2) * ex, ey,
                     (-5 + 3 * e2) * ey, ex * ex - ey * ey, ex * ey])
    return torch.tensor(rows, dtype=torch.float64).T.contiguous()  # [9 moments, 9 directions]


MB = _basis()
NORM = (MB * MB).sum(1)  # (9, 36, 36, 6, 12, 6, 12, 4, 4)


def _safe_sqrt(s):
    pos = s > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, s, torch.ones_like(s))), torch.zeros_like(s))


class Model:
    """Parameters of the step.  eos: ('cs', a, b, R) or ('pw', theta_v,
    theta_m, theta_l, rho1, rho2).  T: float or FP64 tensor (may require grad).  theta_bot,
    theta_top: [nx] tensors of wall angles in radians (may require grad).
    rates: s[9] in moment order.  walls: rows 0 and ny-1 solid."""

    def __init__(self, nx, ny, eos, T, theta_bot, theta_top, rates, A=-0.6, kappa=0.5, G_w=0.0, n_iter=4,
                 wetting=0, walls=True, rho_max=math.inf, ghost_max=None):
        self.nx, self.ny = nx, ny
        self.eos = eos
        self.T = torch.as_tensor(T, dtype=torch.float64)
        self.A, self.kappa, self.G_w, self.n_iter, self.wetting, self.walls = A, kappa, G_w, n_iter, wetting, walls
        self.s = torch.tensor(rates, dtype=torch.float64)
        self.rho_max = rho_max
        self.ghost_max = rho_max if ghost_max is None else ghost_max
        # Eqs. 19-21 use sin(pi/2 - theta) and tan(pi/2 - theta) of each wall node
        self.c = [torch.sin(math.pi / 2 - theta_bot), torch.sin(math.pi / 2 - theta_top)]
        self.cot = [torch.tan(math.pi / 2 - theta_bot), torch.tan(math.pi / 2 - theta_top)]
        fluid = torch.ones(ny, dtype=torch.float64)
        if walls:
            fluid[0] = 0.0
            fluid[-1] = 0.0
        self.fluid = fluid[:, None].expand(ny, nx)

    # ---- Eqs. 10-11 ----------------------------------------------------------
    def pressure(self, rho):
        e = self.eos
        if e[0] == "cs":
            a, b, R = e[1], e[2], e[3]
            eta = b * rho * 0.25
            return rho * R * self.T * (1 + eta + eta * eta - eta ** 3) / (1 - eta) ** 3 - a * rho * rho
        tv, tm, tl, r1, r2 = e[1:]
        return torch.where(rho <= r1, rho * tv,
                           torch.where(rho <= r2, r1 * tv + (rho - r1) * tm, r1 * tv + (r2 - r1) * tm + (rho - r2) * tl))

    def psi_U(self, rho):
        U = self.pressure(rho) - rho / 3.0
        return _safe_sqrt(-2.0 * U), U

    # ---- Eqs. 19-21 ------------------------------------------------------------
    def ghost(self, r1, r2, wall):
        a = torch.roll(r1, -1) - torch.roll(r1, 1)  # rho(i+1, 1) - rho(i-1, 1)
        if self.n_iter <= 0:
            g = r2 + self.cot[wall] * torch.abs(a)
        else:
            d = 2.0 * (r2 - r1)
            g = r2
            for _ in range(self.n_iter):
                g = r2 + self.c[wall] * _safe_sqrt(a * a + d * d)
                d = r2 - g
        g = torch.clamp(g, 0.0, self.ghost_max)
        psi, U = self.psi_U(g)
        top = g >= self.rho_max
        return g, torch.where(top, torch.zeros_like(psi), psi), torch.where(top, torch.zeros_like(U), U)

    def fields(self, f):
        rho = f.sum(0)
        psi, U = self.psi_U(rho)
        if not self.walls:
            return rho, psi, U
        rows_r, rows_p, rows_u = list(rho.unbind(0)), list(psi.unbind(0)), list(U.unbind(0))
        for wall, (yg, y1, y2) in enumerate(((0, 1, 2), (self.ny - 1, self.ny - 2, self.ny - 3))):
            if self.wetting == 1:
                z = torch.zeros(self.nx, dtype=torch.float64)
                rows_r[yg], rows_p[yg], rows_u[yg] = z, z, z
            else:
                rows_r[yg], rows_p[yg], rows_u[yg] = self.ghost(rho[y1], rho[y2], wall)
        return torch.stack(rows_r), torch.stack(rows_p), torch.stack(rows_u)

    # ---- Eqs. 9, 14, 17 ----------------------------------------------------------
    def force_Q(self, psi, U):
        def nb(arr, a):  # value at x + e_a
            return torch.roll(arr, shifts=(-EY[a], -EX[a]), dims=(0, 1))

        solid = 1.0 - self.fluid
        z = torch.zeros_like(psi)
        spx, spy, sUx, sUy, ssx, ssy = z, z, z, z, z, z
        q1 = [z, z, z]
        q2 = [z, z, z]
        for a in range(1, 9):
            w, ex, ey = WGT[a], EX[a], EY[a]
            pn, un, sn = nb(psi, a), nb(U, a), nb(solid, a)
            spx, spy = spx + w * pn * ex, spy + w * pn * ey
            sUx, sUy = sUx + w * un * ex, sUy + w * un * ey
            ssx, ssy = ssx + w * sn * ex, ssy + w * sn * ey
            t1, t2 = w * (pn - psi), w * (pn * pn - psi * psi)
            for k, e in enumerate((ex * ex, ey * ey, ex * ey)):
                q1[k] = q1[k] + e * t1
                q2[k] = q2[k] + e * t2
        cpsi = (1.0 - self.A) * G * psi
        Fx = -self.A * sUx - cpsi * spx
        Fy = -self.A * sUy - cpsi * spy
        if self.wetting == 1:
            Fx = Fx - self.G_w * psi * ssx
            Fy = Fy - self.G_w * psi * ssy
        pre = self.kappa * G * 0.5
        c1, c2 = (1.0 - self.A) * psi, self.A * 0.5
        Q = [pre * (c1 * q1[k] + c2 * q2[k]) for k in range(3)]
        return Fx, Fy, Q[0], Q[1], Q[2]

    # ---- Eqs. 2-6, 15-16 -----------------------------------------------------------
    def collide(self, f, rho, Fx, Fy, Qxx, Qyy, Qxy):
        s = self.s
        m = torch.einsum("ka,ayx->kyx", MB, f)
        vx = (m[3] + 0.5 * Fx) / rho
        vy = (m[5] + 0.5 * Fy) / rho
        v2 = vx * vx + vy * vy
        meq = torch.stack([rho, rho * (-2 + 3 * v2), rho * (1 - 3 * v2), rho * vx, -rho * vx, rho * vy, -rho * vy,
                           rho * (vx * vx - vy * vy), rho * vx * vy])
        vF = vx * Fx + vy * Fy
        S = torch.stack([torch.zeros_like(rho), 6 * vF, -6 * vF, Fx, -Fx, Fy, -Fy, 2 * (vx * Fx - vy * Fy),
                         vx * Fy + vy * Fx])
        z = torch.zeros_like(rho)
        C = torch.stack([z, 1.5 * s[1] * (Qxx + Qyy), z, z, z, z, z, -s[7] * (Qxx - Qyy), -s[8] * Qxy])
        ms = m - s[:, None, None] * (m - meq) + (1 - 0.5 * s[:, None, None]) * S + C
        return torch.einsum("ka,kyx->ayx", MB, ms / NORM[:, None, None])

    # ---- Eq. 1 (streaming) -------------------------------------------------------
    def stream(self, fs):
        fl = self.fluid
        out = [torch.zeros_like(fs[0]) for _ in range(9)]
        for a in range(9):
            tgt_fluid = torch.roll(fl, shifts=-EY[a], dims=0) if self.walls else torch.ones_like(fl)
            go = fs[a] * fl * tgt_fluid
            out[a] = out[a] + torch.roll(go, shifts=(EY[a], EX[a]), dims=(0, 1))
            out[OPP[a]] = out[OPP[a]] + fs[a] * fl * (1.0 - tgt_fluid)
        return torch.stack(out)

    def step(self, f):
        rho, psi, U = self.fields(f)
        Fx, Fy, Qxx, Qyy, Qxy = self.force_Q(psi, U)
        rho_safe = torch.where(self.fluid > 0, rho, torch.ones_like(rho))
        fs = self.collide(f, rho_safe, Fx, Fy, Qxx, Qyy, Qxy) * self.fluid
        return self.stream(fs)

    def run(self, f, nsteps):
        for _ in range(nsteps):
            f = self.step(f)
        return f
