// lbm_adjoint.cu -- discrete adjoint (reverse-time) of the reference step.
//
// Forward step n -> n+1 (lbm_ref.cu): rho, psi, U (Eqs. 1, 10-11); ghost rows
// (Eqs. 19-21); per fluid node the force F (Eq. 9 [+ Eq. 14]) and tensor Q
// (Eq. 17) from the 3x3 stencil of (psi, U); the MRT collision with Guo
// forcing and the Eq. 16 source (Eqs. 4-6, 15); push streaming with half-way
// bounce-back.  Given lam = dL/df^{n+1}, one reverse step computes
// dL/df^n and adds this step's part of dL/dtheta (per wall node, through
// c = sin(pi/2 - theta) of Eq. 21 or cot of Eq. 19) and dL/dT (through the
// EOS), in four kernels:
//
//   k_adj_collide  per fluid node: pull lam back through the streaming
//                  (bounce-back included), recompute F, Q and the collision,
//                  and transpose it: dL/df through the moments, velocity,
//                  equilibrium and forcing, plus dL/dF and dL/dQ (5 values).
//   k_adj_psi      per node (ghost rows too): gather dL/dpsi and dL/dU from
//                  the dL/dF, dL/dQ of the fluid nodes whose stencil holds it
//                  (its own included), map them to dL/drho through the EOS
//                  (psi = sqrt(-2U): dpsi/dU = -1/psi, 0 where psi = 0) and
//                  add the node's dL/dT.
//   k_adj_ghost    per wall node: back through the clamp and the n_iter
//                  iterations of Eq. 20 (or Eq. 19) to the densities of the
//                  boundary row (x-1, x, x+1) and the second row, and to theta.
//   k_adj_finish   per fluid node: dL/df^n_a = collision part + dL/drho for
//                  every a (rho = sum_a f_a), the ghost-rule parts gathered
//                  from the neighbouring wall nodes.
//
// Kinks follow the oracle's convention: d sqrt(s)/ds = 0 at s = 0, d|a|/da = 0
// at a = 0, clamped ghost densities pass nothing.  Gathers instead of atomics
// keep every sum in a fixed order (the result is reproducible bit for bit).
//
// Recording: lbm_adjoint_record runs the steps with the context's own step
// kernel and keeps the state every `checkpoint_every` steps;
// lbm_adjoint_backward replays each segment forward with the same kernel into
// a segment buffer and then walks it back (the canonical fields of each
// state, ghost rows included, are recomputed first).
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "lbm_internal.h"
#include "lbm_ref_node.cuh"

using namespace lbm_ref;

struct lbm_tape {
  int nsteps, every, nseg;
  size_t state_bytes;            // one [9][ny][nx] array
  std::vector<void *> ckpt;      // state at the start of each segment
  void *seg;                     // (every + 1) states of the segment being reversed
  void *lam[2];                  // adjoint fields
  void *aux;                     // 5 planes: dL/dFx, dL/dFy, dL/dQxx, dL/dQyy, dL/dQxy
  void *rhob;                    // dL/drho per node (ghost rows: of the ghost density)
  double *tacc;                  // per-node dL/dT, accumulated over the steps
  double *gpart;                 // [2 walls][4][nx]: ghost-rule partials
  double *dtheta;                // [2][nx]
  double *red;                   // reduction output
  // captured graphs (contexts with a non-NULL stream): the recorded forward of
  // one full segment per starting array, and the replay + reverse sweep of one
  // full segment per starting adjoint buffer
  cudaGraphExec_t fwd_graph[2], bwd_graph[2];
  unsigned long long fwd_launches, bwd_launches;  // kernels per replay
};

namespace {

constexpr int kMaxIter = 64;

template <typename R>
__device__ void eos_derivs(const Mdl<R> &m, R rho, R &dp_drho, R &dp_dT) {
  if (m.kind == LBM_EOS_CARNAHAN_STARLING) {
    // p = rho R T Z(eta) - a rho^2, Z = N/D, N = 1 + eta + eta^2 - eta^3, D = (1 - eta)^3, eta = b rho/4:
    // dp/drho = R T (Z + eta dZ/deta) - 2 a rho,  dZ/deta = N'/D + 3 N/(1 - eta)^4
    R eta = (m.b * rho) * (R)0.25;
    R om = (R)1 - eta;
    R num = (((R)1 + eta) + eta * eta) - (eta * eta) * eta;
    R dnum = ((R)1 + (R)2 * eta) - (R)3 * (eta * eta);
    R den = (om * om) * om;
    R Z = num / den;
    R dZ = dnum / den + ((R)3 * num) / (den * om);
    dp_drho = (m.Rg * m.T) * (Z + eta * dZ) - (R)2 * (m.a * rho);
    dp_dT = (rho * m.Rg) * Z;
  } else {
    dp_dT = (R)0;
    dp_drho = rho <= m.r1 ? m.thv : (rho <= m.r2 ? m.thm : m.thl);
  }
}

template <typename R>
__global__ void k_adj_collide(lbm_dev_params P, const R *__restrict__ f, const R *__restrict__ fields,
                              const R *__restrict__ lam_in, R *__restrict__ lam_out, R *__restrict__ aux) {
  Mdl<R> m(P);
  size_t n = (size_t)m.nx * m.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / m.nx), x = (int)(i - (size_t)y * m.nx);
  if (m.solid_row(y)) return;
  // adjoint of the post-collision populations (transpose of the push streaming)
  R ls[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    int yt = m.wy(y + EY(a));
    ls[a] = m.solid_row(yt) ? lam_in[OPP(a) * n + i] : lam_in[a * n + (size_t)yt * m.nx + m.wx(x + EX(a))];
  }
  R Fx, Fy, Qxx, Qyy, Qxy;
  force_Q(m, fields, y, x, Fx, Fy, Qxx, Qyy, Qxy);
  const R rho = fields[i];
  R mm[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    R acc = (R)0;
#pragma unroll
    for (int a = 0; a < 9; ++a)
      if (MC(k, a) != 0.0) acc = acc + (R)MC(k, a) * f[a * n + i];
    mm[k] = acc;
  }
  const R vx = (mm[3] + (R)0.5 * Fx) / rho, vy = (mm[5] + (R)0.5 * Fy) / rho;
  const R v2 = vx * vx + vy * vy;
  // f* = M^T diag(1/N) m*  ->  dL/dm*_k = sum_a M_ka ls_a / N_k
  R msb[9], mb[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    R acc = (R)0;
#pragma unroll
    for (int a = 0; a < 9; ++a)
      if (MC(k, a) != 0.0) acc = acc + (R)MC(k, a) * ls[a];
    msb[k] = acc / (R)NRM(k);
  }
  // m*_k = m_k - s_k (m_k - meq_k) + (1 - s_k/2) S_k + C_k
  R meqb[9], Sb[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    mb[k] = ((R)1 - m.s[k]) * msb[k];
    meqb[k] = m.s[k] * msb[k];
    Sb[k] = ((R)1 - (R)0.5 * m.s[k]) * msb[k];
  }
  // C_1 = 1.5 s_1 (Qxx + Qyy), C_7 = -s_7 (Qxx - Qyy), C_8 = -s_8 Qxy
  const R Qxxb = ((R)1.5 * m.s[1]) * msb[1] - m.s[7] * msb[7];
  const R Qyyb = ((R)1.5 * m.s[1]) * msb[1] + m.s[7] * msb[7];
  const R Qxyb = -(m.s[8] * msb[8]);
  // S = (0, 6 vF, -6 vF, Fx, -Fx, Fy, -Fy, 2 (vx Fx - vy Fy), vx Fy + vy Fx), vF = v.F
  const R vFb = (R)6 * (Sb[1] - Sb[2]);
  R Fxb = (Sb[3] - Sb[4]) + (R)2 * vx * Sb[7] + vy * Sb[8] + vx * vFb;
  R Fyb = (Sb[5] - Sb[6]) - (R)2 * vy * Sb[7] + vx * Sb[8] + vy * vFb;
  R vxb = (R)2 * Fx * Sb[7] + Fy * Sb[8] + Fx * vFb;
  R vyb = -((R)2 * Fy * Sb[7]) + Fx * Sb[8] + Fy * vFb;
  // meq = rho (1, -2 + 3 v2, 1 - 3 v2, vx, -vx, vy, -vy, vx^2 - vy^2, vx vy)
  R rhob = meqb[0] + meqb[1] * ((R)-2 + (R)3 * v2) + meqb[2] * ((R)1 - (R)3 * v2) + (meqb[3] - meqb[4]) * vx +
           (meqb[5] - meqb[6]) * vy + meqb[7] * (vx * vx - vy * vy) + meqb[8] * (vx * vy);
  const R v2b = (R)3 * rho * (meqb[1] - meqb[2]);
  vxb = vxb + (R)2 * vx * v2b + rho * (meqb[3] - meqb[4]) + (R)2 * rho * vx * meqb[7] + rho * vy * meqb[8];
  vyb = vyb + (R)2 * vy * v2b + rho * (meqb[5] - meqb[6]) - (R)2 * rho * vy * meqb[7] + rho * vx * meqb[8];
  // v = (j + F/2) / rho
  mb[3] = mb[3] + vxb / rho;
  mb[5] = mb[5] + vyb / rho;
  Fxb = Fxb + (R)0.5 * vxb / rho;
  Fyb = Fyb + (R)0.5 * vyb / rho;
  rhob = rhob - (vxb * vx + vyb * vy) / rho;
  // m = M f and rho = sum_a f_a
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    R acc = rhob;
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (MC(k, a) != 0.0) acc = acc + (R)MC(k, a) * mb[k];
    lam_out[a * n + i] = acc;
  }
  aux[i] = Fxb;
  aux[n + i] = Fyb;
  aux[2 * n + i] = Qxxb;
  aux[3 * n + i] = Qyyb;
  aux[4 * n + i] = Qxyb;
}

template <typename R>
__global__ void k_adj_psi(lbm_dev_params P, const R *__restrict__ fields, const R *__restrict__ aux,
                          R *__restrict__ rhob_out, double *__restrict__ tacc) {
  Mdl<R> m(P);
  size_t n = (size_t)m.nx * m.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / m.nx), x = (int)(i - (size_t)y * m.nx);
  const R *psi = fields + n, *U = fields + 2 * n;
  const R G = (R)-1;
  const R pre = m.kappa * (G * (R)0.5);
  const R omA = (R)1 - m.A;
  const R psi_p = psi[i];
  R pb = (R)0, ub = (R)0;
  // fluid nodes q = p - e_a hold p in their stencil in direction a:
  //   dF(q)/dpsi_p = (1-A) psi_q w_a e_a,  dF(q)/dU_p = -A w_a e_a,
  //   dQ_ij(q)/dpsi_p = pre w_a e_ai e_aj ((1-A) psi_q + A psi_p)
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    int yq = y - EY(a);
    if (m.walls && (yq < 0 || yq >= m.ny)) continue;
    yq = m.wy(yq);
    if (m.solid_row(yq)) continue;
    size_t j = (size_t)yq * m.nx + m.wx(x - EX(a));
    const R w = wgt<R>(a);
    const R eF = aux[j] * (R)EX(a) + aux[n + j] * (R)EY(a);
    const R eQ = aux[2 * n + j] * (R)(EX(a) * EX(a)) + aux[3 * n + j] * (R)(EY(a) * EY(a)) +
                 aux[4 * n + j] * (R)(EX(a) * EY(a));
    const R psi_q = psi[j];
    pb = pb + (omA * psi_q) * w * eF + pre * w * eQ * (omA * psi_q + m.A * psi_p);
    ub = ub - m.A * w * eF;
  }
  const bool fluid = !m.solid_row(y);
  if (fluid) {
    // own terms: dF/dpsi_0 = (1-A) s_psi (+ Eq. 14), dQ_ii/dpsi_0 = pre ((1-A) q1_ii - psi_0),
    // dQ_xy/dpsi_0 = pre (1-A) q1_xy
    R spx = 0, spy = 0, ssx = 0, ssy = 0, qxx1 = 0, qyy1 = 0, qxy1 = 0;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      int yn = m.wy(y + EY(a)), xn = m.wx(x + EX(a));
      size_t j = (size_t)yn * m.nx + xn;
      const R w = wgt<R>(a);
      const R pn = psi[j];
      const R sol = m.solid_row(yn) ? (R)1 : (R)0;
      spx = spx + w * pn * (R)EX(a);
      spy = spy + w * pn * (R)EY(a);
      ssx = ssx + w * sol * (R)EX(a);
      ssy = ssy + w * sol * (R)EY(a);
      const R t1 = w * (pn - psi_p);
      qxx1 = qxx1 + t1 * (R)(EX(a) * EX(a));
      qyy1 = qyy1 + t1 * (R)(EY(a) * EY(a));
      qxy1 = qxy1 + t1 * (R)(EX(a) * EY(a));
    }
    const R Fxb = aux[i], Fyb = aux[n + i];
    pb = pb + omA * (Fxb * spx + Fyb * spy);
    if (m.wetting == LBM_WET_MARTYS_CHEN) pb = pb - m.Gw * (Fxb * ssx + Fyb * ssy);
    pb = pb + pre * (omA * (aux[2 * n + i] * qxx1 + aux[3 * n + i] * qyy1 + aux[4 * n + i] * qxy1) -
                     psi_p * (aux[2 * n + i] + aux[3 * n + i]));
  }
  // to dL/drho (and dL/dT) through U = p(rho) - rho/3 and psi = sqrt(-2U)
  R rb = (R)0;
  double tb = 0.0;
  const R rho = fields[i];
  const bool ghost = !fluid && m.wetting == LBM_WET_GEOMETRIC;
  if (fluid || (ghost && rho < m.rho_max)) {
    R dp, dpT;
    eos_derivs(m, rho, dp, dpT);
    const R ut = ub - (psi_p > (R)0 ? pb / psi_p : (R)0);
    rb = ut * (dp - (R)1 / (R)3);
    tb = (double)(ut * dpT);
  }
  rhob_out[i] = rb;
  tacc[i] += tb;
}

template <typename R>
__global__ void k_adj_ghost(lbm_dev_params P, const R *__restrict__ fields, const double *__restrict__ coef,
                            const double *__restrict__ dcoef, const R *__restrict__ rhob,
                            double *__restrict__ gpart, double *__restrict__ dtheta) {
  Mdl<R> m(P);
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * m.nx) return;
  int w = t / m.nx, x = t - w * m.nx;
  int yg = w == 0 ? 0 : m.ny - 1, y1 = w == 0 ? 1 : m.ny - 2, y2 = w == 0 ? 2 : m.ny - 3;
  double *gp = gpart + (size_t)w * 4 * m.nx;
  const R *rho = fields;
  R rim1 = rho[(size_t)y1 * m.nx + m.wx(x - 1)];
  R rip1 = rho[(size_t)y1 * m.nx + m.wx(x + 1)];
  R ri1 = rho[(size_t)y1 * m.nx + x];
  R ri2 = rho[(size_t)y2 * m.nx + x];
  R c = (R)coef[w * m.nx + x];
  R cot = (R)coef[2 * m.nx + w * m.nx + x];
  R a = rip1 - rim1;
  // forward again, keeping the iterates
  R d[kMaxIter];
  R g;
  const int nit = m.n_iter < kMaxIter ? m.n_iter : kMaxIter;
  if (nit <= 0) {
    g = ri2 + cot * fabs(a);
  } else {
    d[0] = (R)2 * (ri2 - ri1);
    g = ri2;
    for (int k = 0; k < nit; ++k) {
      R s = a * a + d[k] * d[k];
      g = ri2 + c * sqrt(s);
      if (k + 1 < nit) d[k + 1] = ri2 - g;
    }
  }
  R gb = rhob[(size_t)yg * m.nx + x];
  if (!(g > (R)0 && g < m.ghost_max)) gb = (R)0;  // clamped: no gradient
  R ab = 0, ri1b = 0, ri2b = 0, cb = 0, cotb = 0;
  if (nit <= 0) {
    ri2b = gb;
    cotb = gb * fabs(a);
    ab = a > (R)0 ? gb * cot : (a < (R)0 ? -(gb * cot) : (R)0);
  } else {
    R gbar = gb;
    for (int k = nit - 1; k >= 0; --k) {
      // g_{k+1} = ri2 + c sqrt(a^2 + d_k^2)
      R s = a * a + d[k] * d[k];
      R sq = sqrt(s);
      ri2b = ri2b + gbar;
      cb = cb + gbar * sq;
      R sb = s > (R)0 ? (gbar * c) * (R)0.5 / sq : (R)0;
      ab = ab + sb * (R)2 * a;
      R db = sb * (R)2 * d[k];
      if (k >= 1) {  // d_k = ri2 - g_k
        ri2b = ri2b + db;
        gbar = -db;
      } else {  // d_0 = 2 (ri2 - ri1)
        ri2b = ri2b + (R)2 * db;
        ri1b = ri1b - (R)2 * db;
      }
    }
  }
  gp[x] = -(double)ab;                // to rho(x-1, boundary row)
  gp[m.nx + x] = (double)ab;          // to rho(x+1, boundary row)
  gp[2 * m.nx + x] = (double)ri1b;    // to rho(x, boundary row)
  gp[3 * m.nx + x] = (double)ri2b;    // to rho(x, second row)
  dtheta[w * m.nx + x] += (double)cb * dcoef[w * m.nx + x] + (double)cotb * dcoef[2 * m.nx + w * m.nx + x];
}

template <typename R>
__global__ void k_adj_finish(lbm_dev_params P, R *__restrict__ lam, const R *__restrict__ rhob,
                             const double *__restrict__ gpart, int geo) {
  Mdl<R> m(P);
  size_t n = (size_t)m.nx * m.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / m.nx), x = (int)(i - (size_t)y * m.nx);
  if (m.solid_row(y)) {
#pragma unroll
    for (int a = 0; a < 9; ++a) lam[a * n + i] = (R)0;
    return;
  }
  double r = (double)rhob[i];
  if (geo) {
    const int xm = m.wx(x - 1), xp = m.wx(x + 1);
    for (int w = 0; w < 2; ++w) {
      const double *gp = gpart + (size_t)w * 4 * m.nx;
      const int y1 = w == 0 ? 1 : m.ny - 2, y2 = w == 0 ? 2 : m.ny - 3;
      // boundary row: this node is x-1 of wall node x+1, x+1 of wall node x-1, and x of wall node x
      if (y == y1) r += gp[xp] + gp[m.nx + xm] + gp[2 * m.nx + x];
      if (y == y2) r += gp[3 * m.nx + x];
    }
  }
  const R rr = (R)r;
#pragma unroll
  for (int a = 0; a < 9; ++a) lam[a * n + i] = lam[a * n + i] + rr;
}

template <typename R>
__global__ void k_adj_init(lbm_dev_params P, const double *__restrict__ dl_drho, R *__restrict__ lam) {
  size_t n = (size_t)P.nx * P.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / P.nx);
  const bool solid = P.walls && (y == 0 || y == P.ny - 1);
  const R v = solid ? (R)0 : (R)dl_drho[i];
#pragma unroll
  for (int a = 0; a < 9; ++a) lam[a * n + i] = v;
}

// Deterministic sum of n doubles by one block.
__global__ void k_sum(const double *__restrict__ v, size_t n, double *__restrict__ out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

template <typename R>
__global__ void k_to_double(const R *__restrict__ in, double *__restrict__ out, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

#define ACK(x)                          \
  do {                                  \
    if ((x) != cudaSuccess) {           \
      cudaGetLastError();               \
      return LBM_ECUDA;                 \
    }                                   \
  } while (0)

size_t rsize(const lbm_ctx *C) { return C->precision == 64 ? sizeof(double) : sizeof(float); }

// One forward step src -> dst with the context's own step kernel: the fused
// FP32 kernel where the context runs it (so the recorded forward advances
// exactly like lbm_step), else the canonical reference kernels.  The reverse
// kernels transpose the canonical step at the states this produces.
int fwd_step(lbm_ctx *C, const void *src, void *dst) {
  if (C->kernel_in_use == LBM_KERNEL_FUSED) {
    ACK(lbm_fused_step_between(C, src, dst, &C->launches));
    return LBM_OK;
  }
  ACK(lbm_ref_fields(C, src, C->d_fields, &C->launches));
  ACK(lbm_ref_collide(C, src, dst, C->d_fields, &C->launches));
  return LBM_OK;
}

template <typename R>
int reverse_step(lbm_ctx *C, lbm_tape *T, const void *f, int lin) {
  const size_t n = (size_t)C->nx * C->ny;
  const int B = 256;
  const unsigned g = (unsigned)((n + B - 1) / B), gw = (unsigned)((2 * C->nx + B - 1) / B);
  const lbm_dev_params &P = C->dp;
  const R *fields = (const R *)C->d_fields;
  ACK(lbm_ref_fields(C, f, C->d_fields, &C->launches));
  R *lam_in = (R *)T->lam[lin], *lam_out = (R *)T->lam[lin ^ 1];
  k_adj_collide<R><<<g, B, 0, C->stream>>>(P, (const R *)f, fields, lam_in, lam_out, (R *)T->aux);
  k_adj_psi<R><<<g, B, 0, C->stream>>>(P, fields, (const R *)T->aux, (R *)T->rhob, T->tacc);
  C->launches += 2;
  const int geo = C->walls && P.wetting == LBM_WET_GEOMETRIC;
  if (geo) {
    k_adj_ghost<R><<<gw, B, 0, C->stream>>>(P, fields, C->d_coef, C->d_dcoef, (const R *)T->rhob, T->gpart,
                                            T->dtheta);
    ++C->launches;
  }
  k_adj_finish<R><<<g, B, 0, C->stream>>>(P, lam_out, (const R *)T->rhob, T->gpart, geo);
  ++C->launches;
  ACK(cudaGetLastError());
  return LBM_OK;
}

// Capture the work that fn() enqueues on the context stream into *out; the
// kernels it launches are counted into *launches (not into the context).
template <typename Fn>
int capture(lbm_ctx *C, cudaGraphExec_t *out, unsigned long long *launches, Fn fn) {
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  const unsigned long long l0 = C->launches;
  int st = fn();
  *launches = C->launches - l0;
  C->launches = l0;
  cudaError_t e = cudaStreamEndCapture(C->stream, &graph);
  if (st == LBM_OK && e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (st == LBM_OK && e != cudaSuccess) st = LBM_ECUDA;
  if (st != LBM_OK) {
    cudaGetLastError();
    *out = nullptr;
  }
  return st;
}

// Replay of a segment from seg[0] (len states) and its reverse sweep, adjoint
// starting in lam[lin]; returns the status and leaves the final buffer in *lin.
template <typename R>
int segment_reverse(lbm_ctx *C, lbm_tape *T, int len, int *lin) {
  char *seg = (char *)T->seg;
  int st = LBM_OK;
  for (int k = 0; k + 1 < len && st == LBM_OK; ++k)
    st = fwd_step(C, seg + (size_t)k * T->state_bytes, seg + (size_t)(k + 1) * T->state_bytes);
  for (int k = len - 1; k >= 0 && st == LBM_OK; --k) {
    st = reverse_step<R>(C, T, seg + (size_t)k * T->state_bytes, *lin);
    *lin ^= 1;
  }
  return st;
}

template <typename R>
int backward(lbm_ctx *C, lbm_tape *T, const double *dl_drho, double *dl_dtheta, double *dl_dT, double *dl_df0) {
  const size_t n = (size_t)C->nx * C->ny;
  const int B = 256;
  double *h = nullptr;
  ACK(cudaMalloc(&h, n * sizeof(double)));
  cudaError_t e = cudaMemcpyAsync(h, dl_drho, n * sizeof(double), cudaMemcpyHostToDevice, C->stream);
  if (e == cudaSuccess) {
    k_adj_init<R><<<(unsigned)((n + B - 1) / B), B, 0, C->stream>>>(C->dp, h, (R *)T->lam[0]);
    ++C->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(T->tacc, 0, n * sizeof(double), C->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(T->dtheta, 0, 2 * (size_t)C->nx * sizeof(double), C->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(T->gpart, 0, 8 * (size_t)C->nx * sizeof(double), C->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h);
    return LBM_ECUDA;
  }
  int lin = 0;
  int st = LBM_OK;
  for (int sgi = T->nseg - 1; sgi >= 0 && st == LBM_OK; --sgi) {
    const int s0 = sgi * T->every, len = (sgi == T->nseg - 1) ? T->nsteps - s0 : T->every;
    // replay the segment: states s0 .. s0 + len - 1 into the segment buffer
    if (cudaMemcpyAsync(T->seg, T->ckpt[sgi], T->state_bytes, cudaMemcpyDeviceToDevice, C->stream) != cudaSuccess) {
      st = LBM_ECUDA;
      break;
    }
    if (C->stream && len == T->every) {
      const int l0 = lin;
      if (!T->bwd_graph[l0]) {
        st = capture(C, &T->bwd_graph[l0], &T->bwd_launches, [&]() {
          int l = l0;
          return segment_reverse<R>(C, T, len, &l);
        });
        if (st) break;
      }
      if (cudaGraphLaunch(T->bwd_graph[l0], C->stream) != cudaSuccess) {
        cudaGetLastError();
        st = LBM_ECUDA;
        break;
      }
      C->launches += T->bwd_launches;
      lin ^= len & 1;
    } else {
      st = segment_reverse<R>(C, T, len, &lin);
    }
  }
  if (st == LBM_OK) {
    // dL/dT: deterministic sum of the per-node parts; dL/dtheta; dL/df0
    k_sum<<<1, 1024, 0, C->stream>>>(T->tacc, n, T->red);
    ++C->launches;
    e = cudaGetLastError();
    if (e == cudaSuccess && dl_dT)
      e = cudaMemcpyAsync(dl_dT, T->red, sizeof(double), cudaMemcpyDeviceToHost, C->stream);
    if (e == cudaSuccess && dl_dtheta)
      e = cudaMemcpyAsync(dl_dtheta, T->dtheta, 2 * (size_t)C->nx * sizeof(double), cudaMemcpyDeviceToHost,
                          C->stream);
    if (e == cudaSuccess && dl_df0) {
      double *tmp = nullptr;
      e = cudaMalloc(&tmp, 9 * n * sizeof(double));
      if (e == cudaSuccess) {
        k_to_double<R><<<(unsigned)((9 * n + B - 1) / B), B, 0, C->stream>>>((const R *)T->lam[lin], tmp, 9 * n);
        ++C->launches;
        e = cudaGetLastError();
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(dl_df0, tmp, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, C->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(C->stream);
        cudaFree(tmp);
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(C->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st = LBM_ECUDA;
    }
  }
  cudaStreamSynchronize(C->stream);
  cudaFree(h);
  return st;
}

}  // namespace

void lbm_adjoint_free_tape(lbm_ctx *C) {
  if (!C || !C->tape) return;
  lbm_tape *T = C->tape;
  cudaStreamSynchronize(C->stream);
  for (void *p : T->ckpt) cudaFree(p);
  cudaFree(T->seg);
  cudaFree(T->lam[0]);
  cudaFree(T->lam[1]);
  cudaFree(T->aux);
  cudaFree(T->rhob);
  cudaFree(T->tacc);
  cudaFree(T->gpart);
  cudaFree(T->dtheta);
  cudaFree(T->red);
  for (int p = 0; p < 2; ++p) {
    if (T->fwd_graph[p]) cudaGraphExecDestroy(T->fwd_graph[p]);
    if (T->bwd_graph[p]) cudaGraphExecDestroy(T->bwd_graph[p]);
  }
  cudaGetLastError();
  delete T;
  C->tape = nullptr;
}

extern "C" {

int lbm_adjoint_record(lbm_ctx *C, int nsteps, int checkpoint_every) {
  LbmRange nvtx_range("lbm_adjoint_record");
  if (!C || nsteps < 1 || checkpoint_every < 1) return LBM_EINVAL;
  if (C->status) return C->status;
  if (C->dp.n_iter > kMaxIter) return LBM_EUNSUPPORTED;
  lbm_adjoint_free_tape(C);
  lbm_tape *T = new (std::nothrow) lbm_tape();
  if (!T) return LBM_ENOMEM;
  C->tape = T;
  const size_t n = (size_t)C->nx * C->ny, rs = rsize(C);
  T->nsteps = nsteps;
  T->every = checkpoint_every < nsteps ? checkpoint_every : nsteps;
  T->nseg = (nsteps + T->every - 1) / T->every;
  T->state_bytes = 9 * n * rs;
  T->ckpt.assign(T->nseg, nullptr);
  bool ok = true;
  for (int k = 0; k < T->nseg && ok; ++k) ok = cudaMalloc(&T->ckpt[k], T->state_bytes) == cudaSuccess;
  ok = ok && cudaMalloc(&T->seg, (size_t)T->every * T->state_bytes) == cudaSuccess &&
       cudaMalloc(&T->lam[0], T->state_bytes) == cudaSuccess && cudaMalloc(&T->lam[1], T->state_bytes) == cudaSuccess &&
       cudaMalloc(&T->aux, 5 * n * rs) == cudaSuccess && cudaMalloc(&T->rhob, n * rs) == cudaSuccess &&
       cudaMalloc(&T->tacc, n * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&T->gpart, 8 * (size_t)C->nx * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&T->dtheta, 2 * (size_t)C->nx * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&T->red, sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_adjoint_free_tape(C);
    return LBM_ENOMEM;
  }
  if (!C->d_fields && cudaMalloc(&C->d_fields, 3 * n * rs) != cudaSuccess) {
    cudaGetLastError();
    lbm_adjoint_free_tape(C);
    return LBM_ENOMEM;
  }
  // run the steps, keeping the state at each segment start
  for (int sg = 0; sg < T->nseg; ++sg) {
    const int len = sg == T->nseg - 1 ? nsteps - sg * T->every : T->every;
    int st = LBM_OK;
    if (cudaMemcpyAsync(T->ckpt[sg], C->f[C->cur], T->state_bytes, cudaMemcpyDeviceToDevice, C->stream) !=
        cudaSuccess) {
      cudaGetLastError();
      st = LBM_ECUDA;
    }
    auto steps = [&](int count, int cur) {
      int r = LBM_OK;
      for (int k = 0; k < count && r == LBM_OK; ++k) r = fwd_step(C, C->f[cur ^ (k & 1)], C->f[cur ^ (k & 1) ^ 1]);
      return r;
    };
    if (st == LBM_OK && C->stream && len == T->every) {
      const int p = C->cur;
      if (!T->fwd_graph[p]) st = capture(C, &T->fwd_graph[p], &T->fwd_launches, [&]() { return steps(len, p); });
      if (st == LBM_OK) {
        if (cudaGraphLaunch(T->fwd_graph[p], C->stream) != cudaSuccess) {
          cudaGetLastError();
          st = LBM_ECUDA;
        } else {
          C->launches += T->fwd_launches;
        }
      }
    } else if (st == LBM_OK) {
      st = steps(len, C->cur);
    }
    if (st) {
      lbm_adjoint_free_tape(C);
      C->status = st;
      return st;
    }
    C->cur ^= len & 1;
    C->steps += len;
  }
  if (cudaStreamSynchronize(C->stream) != cudaSuccess) {
    cudaGetLastError();
    lbm_adjoint_free_tape(C);
    return LBM_ECUDA;
  }
  return lbm_status(C);
}

int lbm_adjoint_backward(lbm_ctx *C, const double *dl_drho, double *dl_dtheta, double *dl_dT, double *dl_df0) {
  LbmRange nvtx_range("lbm_adjoint_backward");
  if (!C || !dl_drho) return LBM_EINVAL;
  if (!C->tape) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  return C->precision == 64 ? backward<double>(C, C->tape, dl_drho, dl_dtheta, dl_dT, dl_df0)
                            : backward<float>(C, C->tape, dl_drho, dl_dtheta, dl_dT, dl_df0);
}

int lbm_adjoint_release(lbm_ctx *C) {
  if (!C) return LBM_EINVAL;
  lbm_adjoint_free_tape(C);
  return LBM_OK;
}

}  // extern "C"
