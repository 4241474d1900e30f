// lbm_ref_node.cuh -- per-node arithmetic of the canonical-order reference
// step (model constants, EOS, Eq. 9 / Eq. 17 stencil, MRT collision), shared
// by the reference kernels (lbm_ref.cu) and the adjoint kernels
// (lbm_adjoint.cu), which recompute the forward quantities of a step.  Both
// translation units are compiled with -fmad=false.
#pragma once

#include <math.h>

#include "lbm_internal.h"

namespace lbm_ref {

// D2Q9 velocities, opposite directions, the moment basis (rho, e, eps, jx, qx,
// jy, qy, pxx, pxy) and its row norms.  Kept as local tables so that fully
// unrolled loops fold every coefficient into the instruction stream.
__device__ __forceinline__ int EX(int a) {
  const int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  return t[a];
}
__device__ __forceinline__ int EY(int a) {
  const int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  return t[a];
}
__device__ __forceinline__ int OPP(int a) {
  const int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  return t[a];
}
__device__ __forceinline__ double MC(int k, int a) {
  const double t[9][9] = {
      {1, 1, 1, 1, 1, 1, 1, 1, 1},     {-4, -1, -1, -1, -1, 2, 2, 2, 2}, {4, -2, -2, -2, -2, 1, 1, 1, 1},
      {0, 1, 0, -1, 0, 1, -1, -1, 1},  {0, -2, 0, 2, 0, 1, -1, -1, 1},   {0, 0, 1, 0, -1, 1, 1, -1, -1},
      {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
  return t[k][a];
}
__device__ __forceinline__ double NRM(int k) {
  const double t[9] = {9, 36, 36, 6, 12, 6, 12, 4, 4};
  return t[k];
}

template <typename R>
struct Mdl {
  int nx, ny, walls, kind, n_iter, wetting;
  R a, b, Rg, T, thv, thm, thl, r1, r2, A, kappa, Gw, rho_max, ghost_max;
  R s[9];
  __device__ explicit Mdl(const lbm_dev_params &P)
      : nx(P.nx), ny(P.ny), walls(P.walls), kind(P.eos_kind), n_iter(P.n_iter), wetting(P.wetting),
        a((R)P.a), b((R)P.b), Rg((R)P.R), T((R)P.T), thv((R)P.thv), thm((R)P.thm), thl((R)P.thl),
        r1((R)P.r1), r2((R)P.r2), A((R)P.A), kappa((R)P.kappa), Gw((R)P.Gw), rho_max((R)P.rho_max),
        ghost_max((R)P.ghost_max) {
    for (int k = 0; k < 9; ++k) s[k] = (R)P.s[k];
  }
  __device__ bool solid_row(int y) const { return walls && (y == 0 || y == ny - 1); }
  __device__ int wx(int x) const { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }
  __device__ int wy(int y) const { return y < 0 ? y + ny : (y >= ny ? y - ny : y); }
};

// Carnahan-Starling or Eq. 11 pressure.
template <typename R>
__device__ R pressure(const Mdl<R> &m, R rho) {
  if (m.kind == LBM_EOS_CARNAHAN_STARLING) {
    R eta = (m.b * rho) * (R)0.25;
    R num = (((R)1 + eta) + eta * eta) - (eta * eta) * eta;
    R den = (((R)1 - eta) * ((R)1 - eta)) * ((R)1 - eta);
    return (((rho * m.Rg) * m.T) * num) / den - (m.a * rho) * rho;
  }
  if (rho <= m.r1) return rho * m.thv;
  if (rho <= m.r2) return m.r1 * m.thv + (rho - m.r1) * m.thm;
  return (m.r1 * m.thv + (m.r2 - m.r1) * m.thm) + (rho - m.r2) * m.thl;
}

// Eq. 10 with c = 1, G = -1: U = p - rho/3, psi = sqrt(max(0, -2U)).
template <typename R>
__device__ void psi_U(const Mdl<R> &m, R rho, R &psi, R &U) {
  R u = pressure(m, rho) - rho / (R)3;
  U = u;
  psi = sqrt(fmax((R)0, (R)-2 * u));
}

template <typename R>
__device__ __forceinline__ R wgt(int a) { return a <= 4 ? (R)1 / (R)3 : (R)1 / (R)12; }

// Eq. 9 force (+ Eq. 14) and Eq. 17 tensor at fluid node (x, y).
template <typename R>
__device__ void force_Q(const Mdl<R> &m, const R *__restrict__ fields, int y, int x, R &Fx, R &Fy, R &Qxx,
                        R &Qyy, R &Qxy) {
  size_t n = (size_t)m.nx * m.ny;
  const R *psi = fields + n, *U = fields + 2 * n;
  R psi0 = psi[(size_t)y * m.nx + x];
  R spx = 0, spy = 0, sUx = 0, sUy = 0, ssx = 0, ssy = 0;
  R qxx1 = 0, qyy1 = 0, qxy1 = 0, qxx2 = 0, qyy2 = 0, qxy2 = 0;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    int yn = m.wy(y + EY(a)), xn = m.wx(x + EX(a));
    size_t j = (size_t)yn * m.nx + xn;
    R pn = psi[j], un = U[j];
    R w = wgt<R>(a);
    R solid = m.solid_row(yn) ? (R)1 : (R)0;
    if (EX(a) != 0) {
      R tp = w * pn, tu = w * un, ts = w * solid;
      if (EX(a) > 0) { spx = spx + tp; sUx = sUx + tu; ssx = ssx + ts; }
      else { spx = spx - tp; sUx = sUx - tu; ssx = ssx - ts; }
    }
    if (EY(a) != 0) {
      R tp = w * pn, tu = w * un, ts = w * solid;
      if (EY(a) > 0) { spy = spy + tp; sUy = sUy + tu; ssy = ssy + ts; }
      else { spy = spy - tp; sUy = sUy - tu; ssy = ssy - ts; }
    }
    R t1 = w * (pn - psi0);
    R t2 = w * (pn * pn - psi0 * psi0);
    int exx = EX(a) * EX(a), eyy = EY(a) * EY(a), exy = EX(a) * EY(a);
    if (exx) { qxx1 = qxx1 + t1; qxx2 = qxx2 + t2; }
    if (eyy) { qyy1 = qyy1 + t1; qyy2 = qyy2 + t2; }
    if (exy > 0) { qxy1 = qxy1 + t1; qxy2 = qxy2 + t2; }
    if (exy < 0) { qxy1 = qxy1 - t1; qxy2 = qxy2 - t2; }
  }
  const R G = (R)-1;
  R cpsi = (((R)1 - m.A) * G) * psi0;
  R fx = -(m.A * sUx) - cpsi * spx;
  R fy = -(m.A * sUy) - cpsi * spy;
  if (m.wetting == LBM_WET_MARTYS_CHEN) {
    R gp = m.Gw * psi0;
    fx = fx + (-(gp * ssx));
    fy = fy + (-(gp * ssy));
  }
  R pre = m.kappa * (G * (R)0.5);
  R c1 = ((R)1 - m.A) * psi0, c2 = m.A * (R)0.5;
  Fx = fx;
  Fy = fy;
  Qxx = pre * ((c1 * qxx1) + (c2 * qxx2));
  Qyy = pre * ((c1 * qyy1) + (c2 * qyy2));
  Qxy = pre * ((c1 * qxy1) + (c2 * qxy2));
}

// MRT collision with forcing (Eqs. 4, 6, 15 with the Eq. 16 source).
template <typename R>
__device__ void collide(const Mdl<R> &m, const R *f, R rho, R Fx, R Fy, R Qxx, R Qyy, R Qxy, R *fs) {
  R mm[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    R acc = (R)0;
#pragma unroll
    for (int a = 0; a < 9; ++a)
      if (MC(k, a) != 0.0) acc = acc + (R)MC(k, a) * f[a];
    mm[k] = acc;
  }
  R vx = (mm[3] + (R)0.5 * Fx) / rho;
  R vy = (mm[5] + (R)0.5 * Fy) / rho;
  R v2 = vx * vx + vy * vy;
  R meq[9], S[9], C[9];
  meq[0] = rho;
  meq[1] = rho * ((R)-2 + (R)3 * v2);
  meq[2] = rho * ((R)1 - (R)3 * v2);
  meq[3] = rho * vx;
  meq[4] = -(rho * vx);
  meq[5] = rho * vy;
  meq[6] = -(rho * vy);
  meq[7] = rho * (vx * vx - vy * vy);
  meq[8] = rho * (vx * vy);
  R vF = vx * Fx + vy * Fy;
  S[0] = 0;
  S[1] = (R)6 * vF;
  S[2] = -((R)6 * vF);
  S[3] = Fx;
  S[4] = -Fx;
  S[5] = Fy;
  S[6] = -Fy;
  S[7] = (R)2 * (vx * Fx - vy * Fy);
  S[8] = vx * Fy + vy * Fx;
#pragma unroll
  for (int k = 0; k < 9; ++k) C[k] = 0;
  C[1] = ((R)1.5 * m.s[1]) * (Qxx + Qyy);
  C[7] = -(m.s[7] * (Qxx - Qyy));
  C[8] = -(m.s[8] * Qxy);
  R r[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    R ms = ((mm[k] - m.s[k] * (mm[k] - meq[k])) + ((R)1 - (R)0.5 * m.s[k]) * S[k]) + C[k];
    r[k] = ms / (R)NRM(k);
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    R acc = (R)0;
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (MC(k, a) != 0.0) acc = acc + (R)MC(k, a) * r[k];
    fs[a] = acc;
  }
}

}  // namespace lbm_ref
