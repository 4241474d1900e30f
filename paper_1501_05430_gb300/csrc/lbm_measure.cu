// lbm_measure.cu -- density field, reductions and the apparent contact-angle
// measurement (the paper reports "measured" angles in Secs. 4.2.1-4.2.2
// without a procedure; the one implemented here is documented in lbm.h).
// Compiled with -fmad=false: with an FP64 state the column sums, crossings
// and heights are bit-identical to a sequential FP64 evaluation.
#include <float.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace {

// The left-to-right double sum (((0 + f_0) + f_1) + ...) + f_8 of nine
// floats, bit for bit, mostly without FP64 instructions (GB300 issues FP64 at
// a small fraction of its FP32 rate).  When the nonzero terms span at most 26
// binades (exponents emin..emin+25), each term is an integer multiple of
// u = 2^(emin - 150) below 2^49 u, so every partial sum is a multiple of u
// below 9 * 2^49 u < 2^53 u: exactly representable in double.  The double
// additions are then exact, and the sum is the integer total S times u,
// assembled directly as a double (exact cancellation gives +0, as the double
// additions starting from +0 do).  Wider spans and subnormal, infinite or NaN
// terms take the double additions.
__device__ __forceinline__ double sum9(const float (&v)[9]) {
  int emin = 255, emax = 0;
  bool plain = true;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const unsigned u = __float_as_uint(v[a]);
    const int e = (int)((u >> 23) & 255u);
    plain &= e != 255 && (e != 0 || (u & 0x7fffffu) == 0u);
    if (e != 0) {
      emin = min(emin, e);
      emax = max(emax, e);
    }
  }
  if (plain && emax - emin <= 25) {
    long long S = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const unsigned u = __float_as_uint(v[a]);
      const int e = (int)((u >> 23) & 255u);
      if (e != 0) {
        const long long m = (long long)((u & 0x7fffffu) | 0x800000u) << (e - emin);
        S += (u >> 31) ? -m : m;
      }
    }
    if (S == 0) return 0.0;
    const unsigned long long A = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
    const int p = 63 - __clzll((long long)A);  // p <= 52
    const unsigned long long bits = ((unsigned long long)(S < 0) << 63) |
                                    ((unsigned long long)(p + emin - 150 + 1023) << 52) |
                                    ((A << (52 - p)) & 0xfffffffffffffull);
    return __longlong_as_double((long long)bits);
  }
  double r = 0.0;
#pragma unroll
  for (int a = 0; a < 9; ++a) r = r + (double)v[a];
  return r;
}

// rho = sum_a f_a accumulated in double, left to right, at fluid nodes; 0 on
// the solid rows; nodes [i0, i1) of the field.
template <typename R>
__global__ void k_rho64(int nx, int ny, int walls, const R *__restrict__ f, double *__restrict__ rho, size_t i0,
                        size_t i1) {
  size_t n = (size_t)nx * ny;
  size_t i = i0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= i1) return;
  int y = (int)(i / nx);
  if (walls && (y == 0 || y == ny - 1)) {
    rho[i] = 0.0;
    return;
  }
  if (sizeof(R) == sizeof(float)) {
    float v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = (float)f[a * n + i];
    rho[i] = sum9(v);
    return;
  }
  double r = 0.0;
#pragma unroll
  for (int a = 0; a < 9; ++a) r = r + (double)f[a * n + i];
  rho[i] = r;
}

// The same for FP32 states with nx % 4 == 0: four consecutive nodes of one
// row per thread (16-byte loads of each plane, 2 x 16-byte stores); groups of
// four [q0, q1).
__global__ void k_rho64_x4(int nx, int ny, int walls, const float4 *__restrict__ f, double2 *__restrict__ rho,
                           size_t q0, size_t q1) {
  const size_t n4 = (size_t)nx * ny / 4;
  const size_t i = q0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q1) return;
  const int y = (int)((4 * i) / nx);
  double2 lo = make_double2(0.0, 0.0), hi = lo;
  if (!(walls && (y == 0 || y == ny - 1))) {
    float v0[9], v1[9], v2[9], v3[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float4 v = f[a * n4 + i];
      v0[a] = v.x;
      v1[a] = v.y;
      v2[a] = v.z;
      v3[a] = v.w;
    }
    lo = make_double2(sum9(v0), sum9(v1));
    hi = make_double2(sum9(v2), sum9(v3));
  }
  rho[2 * i] = lo;
  rho[2 * i + 1] = hi;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Stage 1: block b sums the fluid part of a fixed contiguous chunk; stage 2:
// one block sums the partials.  Both stages use a fixed tree, so the result
// does not depend on scheduling.
__global__ void k_sum_partial(const double *__restrict__ v, size_t n, size_t y0, size_t y1, int nx,
                              double *__restrict__ partial) {
  __shared__ double sh[32];
  size_t lo = y0 * nx, hi = y1 * nx;
  size_t len = hi - lo, chunk = (len + gridDim.x - 1) / gridDim.x;
  size_t b0 = lo + blockIdx.x * chunk, b1 = min(hi, b0 + chunk);
  double s = 0.0;
  for (size_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += v[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

__global__ void k_sum_final(const double *__restrict__ partial, int np, double *__restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[0] = t;
  }
}

__global__ void k_speed_partial(const double *__restrict__ ux, const double *__restrict__ uy, size_t y0, size_t y1,
                                int nx, double *__restrict__ partial) {
  __shared__ double sh[32];
  size_t lo = y0 * nx, hi = y1 * nx;
  size_t len = hi - lo, chunk = (len + gridDim.x - 1) / gridDim.x;
  size_t b0 = lo + blockIdx.x * chunk, b1 = min(hi, b0 + chunk);
  double m = 0.0;
  for (size_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) m = fmax(m, sqrt(ux[i] * ux[i] + uy[i] * uy[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_max(t);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

__global__ void k_max_final(const double *__restrict__ partial, int np, double *__restrict__ out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) m = fmax(m, partial[i]);
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_max(t);
    if (threadIdx.x == 0) out[0] = t;
  }
}

// Block-wide reductions of one int / one (value, index) pair.
__device__ int block_reduce_int(int v, bool is_max, int *sh) {
  for (int o = 16; o > 0; o >>= 1) {
    int u = __shfl_down_sync(0xffffffffu, v, o);
    v = is_max ? max(v, u) : min(v, u);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int nw = blockDim.x >> 5;
    int t = threadIdx.x < nw ? sh[threadIdx.x] : (is_max ? INT_MIN : INT_MAX);
    for (int o = 16; o > 0; o >>= 1) {
      int u = __shfl_down_sync(0xffffffffu, t, o);
      t = is_max ? max(t, u) : min(t, u);
    }
    if (threadIdx.x == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// One block per call.  res = {theta, H, L, xc, status}.
__global__ void k_angle(const double *__restrict__ rho, int nx, int ny, int wall, int x0, int x1, double rho_mid,
                        double *__restrict__ res) {
  __shared__ double shv[33];
  __shared__ int shi[33];
  int ylo = wall == 0 ? 1 : ny / 2, yhi = wall == 0 ? ny / 2 : ny - 1;
  int base = wall == 0 ? 1 : ny - 2, dir = wall == 0 ? 1 : -1;
  // column sums over the wall's half, each summed bottom to top
  double best = -DBL_MAX;
  int bx = INT_MAX;
  for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
    double s = 0.0;
    for (int y = ylo; y < yhi; ++y) s = s + rho[(size_t)y * nx + x];
    if (s > best || (s == best && x < bx)) { best = s; bx = x; }
  }
  // argmax, ties to the lowest column
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, best, o);
    int ox = __shfl_down_sync(0xffffffffu, bx, o);
    if (ov > best || (ov == best && ox < bx)) { best = ov; bx = ox; }
  }
  if ((threadIdx.x & 31) == 0) { shv[threadIdx.x >> 5] = best; shi[threadIdx.x >> 5] = bx; }
  __syncthreads();
  if (threadIdx.x < 32) {
    int nw = blockDim.x >> 5;
    double v = threadIdx.x < nw ? shv[threadIdx.x] : -DBL_MAX;
    int xx = threadIdx.x < nw ? shi[threadIdx.x] : INT_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, v, o);
      int ox = __shfl_down_sync(0xffffffffu, xx, o);
      if (ov > v || (ov == v && ox < xx)) { v = ov; xx = ox; }
    }
    if (threadIdx.x == 0) shi[32] = xx;
  }
  __syncthreads();
  int xc = shi[32];
  const double *row = rho + (size_t)base * nx;
  // liquid run of the boundary row containing xc
  int jl = INT_MIN, jr = INT_MAX;
  for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
    bool vap = !(row[x] >= rho_mid);
    if (vap && x < xc) jl = max(jl, x);
    if (vap && x > xc) jr = min(jr, x);
  }
  __shared__ int shr[33];
  jl = block_reduce_int(jl, true, shr);
  jr = block_reduce_int(jr, false, shr);
  // first vapour node walking away from the wall along xc
  int ymax = wall == 0 ? yhi : ylo - 1;
  int kmin = INT_MAX;
  int nwalk = wall == 0 ? (ymax - base - 1) : (base - ymax - 1);
  for (int k = 1 + threadIdx.x; k <= nwalk; k += blockDim.x) {
    int y = base + k * dir;
    if (!(rho[(size_t)y * nx + xc] >= rho_mid)) kmin = min(kmin, k);
  }
  kmin = block_reduce_int(kmin, false, shr);
  if (threadIdx.x != 0) return;
  res[3] = (double)xc;
  if (!(row[xc] >= rho_mid) || jl == INT_MIN || jr == INT_MAX || kmin == INT_MAX) {
    res[4] = (double)LBM_ENOCONTACT;
    return;
  }
  int xl = jl + 1, xr = jr - 1;
  double xleft = (double)(xl - 1) + (rho_mid - row[xl - 1]) / (row[xl] - row[xl - 1]);
  double xright = (double)xr + (row[xr] - rho_mid) / (row[xr] - row[xr + 1]);
  int steps = kmin - 1;
  int y = base + steps * dir;
  double ra = rho[(size_t)y * nx + xc], rb = rho[(size_t)(y + dir) * nx + xc];
  double h = (double)steps + (ra - rho_mid) / (ra - rb);
  double L = xright - xleft;
  res[0] = 2.0 * atan2(2.0 * h, L);
  res[1] = h;
  res[2] = L;
  res[4] = 0.0;
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t lbm_rho64_rows(const lbm_ctx *C, const void *f, double *rho, int row0, int row1,
                           unsigned long long *launches) {
  const size_t i0 = (size_t)row0 * C->nx, i1 = (size_t)row1 * C->nx;
  if (i1 <= i0) return cudaSuccess;
  if (C->precision == 64)
    k_rho64<double><<<nblk(i1 - i0, 256), 256, 0, C->stream>>>(C->nx, C->ny, C->walls, (const double *)f, rho, i0,
                                                                i1);
  else if (C->nx % 4 == 0 && ((uintptr_t)f & 15) == 0 && ((uintptr_t)rho & 15) == 0)
    k_rho64_x4<<<nblk((i1 - i0) / 4, 256), 256, 0, C->stream>>>(C->nx, C->ny, C->walls, (const float4 *)f,
                                                                 (double2 *)rho, i0 / 4, i1 / 4);
  else
    k_rho64<float><<<nblk(i1 - i0, 256), 256, 0, C->stream>>>(C->nx, C->ny, C->walls, (const float *)f, rho, i0, i1);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t lbm_rho64(const lbm_ctx *C, const void *f, double *rho, unsigned long long *launches) {
  return lbm_rho64_rows(C, f, rho, 0, C->ny, launches);
}

cudaError_t lbm_reduce_mass(const lbm_ctx *C, const double *rho, double *partial, int npart, double *res,
                            unsigned long long *launches) {
  size_t y0 = C->walls ? 1 : 0, y1 = C->walls ? C->ny - 1 : C->ny;
  k_sum_partial<<<npart, 256, 0, C->stream>>>(rho, (size_t)C->nx * C->ny, y0, y1, C->nx, partial);
  k_sum_final<<<1, 1024, 0, C->stream>>>(partial, npart, res);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t lbm_reduce_max_speed(const lbm_ctx *C, const double *ux, const double *uy, double *partial, int npart,
                                 double *res, unsigned long long *launches) {
  size_t y0 = C->walls ? 1 : 0, y1 = C->walls ? C->ny - 1 : C->ny;
  k_speed_partial<<<npart, 256, 0, C->stream>>>(ux, uy, y0, y1, C->nx, partial);
  k_max_final<<<1, 1024, 0, C->stream>>>(partial, npart, res);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t lbm_angle(const lbm_ctx *C, const double *rho, int wall, int x0, int x1, double rho_mid, double *res,
                      unsigned long long *launches) {
  k_angle<<<1, 1024, 0, C->stream>>>(rho, C->nx, C->ny, wall, x0, x1, rho_mid, res);
  ++*launches;
  return cudaGetLastError();
}
