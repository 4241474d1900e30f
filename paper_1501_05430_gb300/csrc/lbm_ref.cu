// lbm_ref.cu -- unfused reference kernels of the pseudo-potential D2Q9 step,
// written in the canonical evaluation order (sums left to right in index
// order, integer moment coefficients applied as multiplications) and compiled
// with -fmad=false, so that the double instantiation is bit-identical to any
// IEEE FP64 evaluation of the step in the same order.
//
// One step = lbm_ref_fields (rho, psi, U; Eqs. 1, 10, 11 -- and on the solid
// rows the ghost values of Eqs. 19-21 or the Martys-Chen zero potential) ->
// lbm_ref_collide (Eq. 9 [+ Eq. 14], Eqs. 16-17, collision Eqs. 4-6 and 15,
// streaming of Eq. 1 with half-way bounce-back).  The fused FP32 kernel (lbm_fused.cu) computes the
// same step in one pass; these kernels also serve the macroscopic getters.
#include <math.h>
#include <stdint.h>

#include "lbm_internal.h"
#include "lbm_ref_node.cuh"

namespace {

using namespace lbm_ref;

// rho at node i: f_0 + f_1 + ... + f_8, left to right.
template <typename R>
__device__ __forceinline__ R node_rho(const R *__restrict__ f, size_t n, size_t i) {
  R r = (R)0;
#pragma unroll
  for (int a = 0; a < 9; ++a) r = r + f[a * n + i];
  return r;
}

// rho, psi, U at every node.  A solid-row node carries its wall's ghost
// values: Eqs. 19-21 (geometric) from the densities of rows 1-2 (ny-2, ny-3),
// which the thread sums itself in the same order as their own threads do, or
// the zero potential (Martys-Chen).
template <typename R>
__global__ void k_fields(lbm_dev_params P, const R *__restrict__ f, const double *__restrict__ coef,
                         R *__restrict__ fields, int *flag) {
  Mdl<R> m(P);
  size_t n = (size_t)m.nx * m.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / m.nx);
  if (m.solid_row(y)) {
    const int x = (int)(i - (size_t)y * m.nx);
    R g = (R)0, psi = (R)0, U = (R)0;
    if (m.wetting != LBM_WET_MARTYS_CHEN) {
      const int w = y == 0 ? 0 : 1, y1 = w == 0 ? 1 : m.ny - 2, y2 = w == 0 ? 2 : m.ny - 3;
      const R rim1 = node_rho(f, n, (size_t)y1 * m.nx + m.wx(x - 1));
      const R rip1 = node_rho(f, n, (size_t)y1 * m.nx + m.wx(x + 1));
      const R ri1 = node_rho(f, n, (size_t)y1 * m.nx + x);
      const R ri2 = node_rho(f, n, (size_t)y2 * m.nx + x);
      const R c = (R)coef[w * m.nx + x];
      const R cot = (R)coef[2 * m.nx + w * m.nx + x];
      const R a = rip1 - rim1;
      if (m.n_iter <= 0) {
        g = ri2 + cot * fabs(a);
      } else {
        R d = (R)2 * (ri2 - ri1);
        g = ri2;
        for (int k = 0; k < m.n_iter; ++k) {
          R s = a * a + d * d;
          g = ri2 + c * sqrt(s);
          d = ri2 - g;
        }
      }
      g = fmin(fmax(g, (R)0), m.ghost_max);
      // at rho_max (the root of U, Eq. 10) psi and U take their exact value 0
      if (g < m.rho_max) psi_U(m, g, psi, U);
    }
    fields[i] = g;
    fields[n + i] = psi;
    fields[2 * n + i] = U;
    return;
  }
  const R r = node_rho(f, n, i);
  R psi, U;
  psi_U(m, r, psi, U);
  fields[i] = r;
  fields[n + i] = psi;
  fields[2 * n + i] = U;
  if (!(r > (R)0) || r > m.rho_max) atomicOr(flag, 1);
}

template <typename R>
__global__ void k_collide(lbm_dev_params P, const R *__restrict__ fin, R *__restrict__ fout,
                          const R *__restrict__ fields) {
  Mdl<R> m(P);
  size_t n = (size_t)m.nx * m.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / m.nx), x = (int)(i - (size_t)y * m.nx);
  if (m.solid_row(y)) return;
  R Fx, Fy, Qxx, Qyy, Qxy;
  force_Q(m, fields, y, x, Fx, Fy, Qxx, Qyy, Qxy);
  R fl[9], fs[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) fl[a] = fin[a * n + i];
  collide(m, fl, fields[i], Fx, Fy, Qxx, Qyy, Qxy, fs);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    int yt = m.wy(y + EY(a));
    if (m.solid_row(yt)) {
      fout[OPP(a) * n + i] = fs[a];
    } else {
      fout[a * n + (size_t)yt * m.nx + m.wx(x + EX(a))] = fs[a];
    }
  }
}

// Macroscopic outputs at every node: out7 = {ux, uy, Fx, Fy, Qxx, Qyy, Qxy}
// (zero on the solid rows).
template <typename R>
__global__ void k_macro(lbm_dev_params P, const R *__restrict__ f, const R *__restrict__ fields,
                        double *__restrict__ out7) {
  Mdl<R> m(P);
  size_t n = (size_t)m.nx * m.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / m.nx), x = (int)(i - (size_t)y * m.nx);
  if (m.solid_row(y)) {
    for (int k = 0; k < 7; ++k) out7[k * n + i] = 0.0;
    return;
  }
  R Fx, Fy, Qxx, Qyy, Qxy;
  force_Q(m, fields, y, x, Fx, Fy, Qxx, Qyy, Qxy);
  R jx = 0, jy = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    if (MC(3, a) != 0.0) jx = jx + (R)MC(3, a) * f[a * n + i];
    if (MC(5, a) != 0.0) jy = jy + (R)MC(5, a) * f[a * n + i];
  }
  R r = fields[i];
  out7[i] = (double)((jx + (R)0.5 * Fx) / r);
  out7[n + i] = (double)((jy + (R)0.5 * Fy) / r);
  out7[2 * n + i] = (double)Fx;
  out7[3 * n + i] = (double)Fy;
  out7[4 * n + i] = (double)Qxx;
  out7[5 * n + i] = (double)Qyy;
  out7[6 * n + i] = (double)Qxy;
}

// A density a state may start from: finite and > 0.  Tested on the bits
// (0 < bits < the bits of +infinity), without FP64 instructions.
__device__ __forceinline__ bool rho_ok(double r) {
  const long long b = __double_as_longlong(r);
  return b > 0 && b < 0x7ff0000000000000ll;
}

// f := M^-1 m_eq(rho, 0).  The double instantiation evaluates it in the
// canonical order; the float one uses its closed form rho * (4/9, 1/9 x4,
// 1/36 x4) in double and rounds once (the same values up to the last bit of
// double, without nine double divisions per node).  rho may be device memory
// or mapped (pinned) host memory; with bad != NULL, *bad |= 1 for a fluid
// density that fails rho_ok (the nodes are written all the same).
template <typename R>
__global__ void k_set_rho(lbm_dev_params P, const double *__restrict__ rho, R *__restrict__ f, int *bad) {
  size_t n = (size_t)P.nx * P.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / P.nx);
  if (P.walls && (y == 0 || y == P.ny - 1)) {
    for (int a = 0; a < 9; ++a) f[a * n + i] = (R)0;
    return;
  }
  double r = rho[i], vx = 0.0, vy = 0.0;
  if (bad && !rho_ok(r)) atomicOr(bad, 1);
  if (sizeof(R) == sizeof(float)) {
    const double w0 = 4.0 / 9.0, w1 = 1.0 / 9.0, w2 = 1.0 / 36.0;
    f[i] = (R)(r * w0);
#pragma unroll
    for (int a = 1; a < 5; ++a) f[a * n + i] = (R)(r * w1);
#pragma unroll
    for (int a = 5; a < 9; ++a) f[a * n + i] = (R)(r * w2);
    return;
  }
  double v2 = vx * vx + vy * vy;
  double meq[9] = {r, r * (-2.0 + 3.0 * v2), r * (1.0 - 3.0 * v2), r * vx, -(r * vx),
                   r * vy, -(r * vy), r * (vx * vx - vy * vy), r * (vx * vy)};
  double q[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k] = meq[k] / NRM(k);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (MC(k, a) != 0.0) acc = acc + MC(k, a) * q[k];
    f[a * n + i] = (R)acc;
  }
}

// The float closed form for nx % 4 == 0: four consecutive nodes of one row
// per thread (two 16-byte loads of rho, one 16-byte store per plane).
__global__ void k_set_rho_x4(int nx, int ny, int walls, const double2 *__restrict__ rho, float4 *__restrict__ f,
                             int *bad) {
  const size_t n4 = (size_t)nx * ny / 4;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const int y = (int)((4 * i) / nx);
  float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0, q2 = q0;
  if (!(walls && (y == 0 || y == ny - 1))) {
    const double2 a = rho[2 * i], b = rho[2 * i + 1];
    if (bad && !(rho_ok(a.x) && rho_ok(a.y) && rho_ok(b.x) && rho_ok(b.y))) atomicOr(bad, 1);
    const double w0 = 4.0 / 9.0, w1 = 1.0 / 9.0, w2 = 1.0 / 36.0;
    q0 = make_float4((float)(a.x * w0), (float)(a.y * w0), (float)(b.x * w0), (float)(b.y * w0));
    q1 = make_float4((float)(a.x * w1), (float)(a.y * w1), (float)(b.x * w1), (float)(b.y * w1));
    q2 = make_float4((float)(a.x * w2), (float)(a.y * w2), (float)(b.x * w2), (float)(b.y * w2));
  }
  f[i] = q0;
#pragma unroll
  for (int k = 1; k < 5; ++k) f[k * n4 + i] = q1;
#pragma unroll
  for (int k = 5; k < 9; ++k) f[k * n4 + i] = q2;
}

// Droplet density field: max over droplets of the tanh profile.
__global__ void k_droplets(lbm_dev_params P, int nd, const double *__restrict__ drop, double width, double rho_v,
                           double rho_l, double *__restrict__ rho) {
  size_t n = (size_t)P.nx * P.ny;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int y = (int)(i / P.nx), x = (int)(i - (size_t)y * P.nx);
  double best = rho_v;
  for (int k = 0; k < nd; ++k) {
    double xc = drop[3 * k], R0 = drop[3 * k + 1];
    double yc = drop[3 * k + 2] == 0.0 ? 1.0 : (double)(P.ny - 2);
    double dx = (double)x - xc;
    double half = 0.5 * P.nx;
    dx = dx - P.nx * floor((dx + half) / P.nx);
    double r = sqrt(dx * dx + ((double)y - yc) * ((double)y - yc));
    double v = 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * tanh(2.0 * (r - R0) / width);
    best = fmax(best, v);
  }
  rho[i] = best;
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t lbm_ref_fields(const lbm_ctx *C, const void *f, void *fields, unsigned long long *launches) {
  size_t n = (size_t)C->nx * C->ny;
  if (C->precision == 64)
    k_fields<double><<<nblk(n, 256), 256, 0, C->stream>>>(C->dp, (const double *)f, C->d_coef, (double *)fields,
                                                          C->d_flag);
  else
    k_fields<float><<<nblk(n, 256), 256, 0, C->stream>>>(C->dp, (const float *)f, C->d_coef, (float *)fields,
                                                         C->d_flag);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t lbm_ref_collide(const lbm_ctx *C, const void *fin, void *fout, const void *fields,
                            unsigned long long *launches) {
  size_t n = (size_t)C->nx * C->ny;
  if (C->precision == 64)
    k_collide<double><<<nblk(n, 128), 128, 0, C->stream>>>(C->dp, (const double *)fin, (double *)fout,
                                                           (const double *)fields);
  else
    k_collide<float><<<nblk(n, 128), 128, 0, C->stream>>>(C->dp, (const float *)fin, (float *)fout,
                                                          (const float *)fields);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t lbm_ref_macro(const lbm_ctx *C, const void *f, const void *fields, double *out7,
                          unsigned long long *launches) {
  size_t n = (size_t)C->nx * C->ny;
  if (C->precision == 64)
    k_macro<double><<<nblk(n, 128), 128, 0, C->stream>>>(C->dp, (const double *)f, (const double *)fields, out7);
  else
    k_macro<float><<<nblk(n, 128), 128, 0, C->stream>>>(C->dp, (const float *)f, (const float *)fields, out7);
  ++*launches;
  return cudaGetLastError();
}

// Input check of lbm_set_rho: every fluid-node density finite and > 0.
cudaError_t lbm_ref_set_rho(const lbm_ctx *C, const double *rho, void *f, int *bad, unsigned long long *launches) {
  size_t n = (size_t)C->nx * C->ny;
  if (C->precision == 64)
    k_set_rho<double><<<nblk(n, 256), 256, 0, C->stream>>>(C->dp, rho, (double *)f, bad);
  else if (C->nx % 4 == 0 && ((uintptr_t)rho & 15) == 0 && ((uintptr_t)f & 15) == 0)
    k_set_rho_x4<<<nblk(n / 4, 256), 256, 0, C->stream>>>(C->nx, C->ny, C->walls, (const double2 *)rho,
                                                          (float4 *)f, bad);
  else
    k_set_rho<float><<<nblk(n, 256), 256, 0, C->stream>>>(C->dp, rho, (float *)f, bad);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t lbm_ref_droplets(const lbm_ctx *C, int nd, const double *drop, double width, double *rho,
                             unsigned long long *launches) {
  size_t n = (size_t)C->nx * C->ny;
  k_droplets<<<nblk(n, 256), 256, 0, C->stream>>>(C->dp, nd, drop, width, C->rho_v, C->rho_l, rho);
  ++*launches;
  return cudaGetLastError();
}
