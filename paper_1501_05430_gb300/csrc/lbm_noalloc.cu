// lbm_noalloc.cu -- lbm_mass_noalloc: the total-mass reduction for callers that
// cannot allocate device memory.
//
// lbm_mass computes rho per node into a context-owned scratch field and sums it
// through a context-owned array of block partials.  This variant takes the
// caller's distribution-function array directly, forms rho on the fly and keeps
// its block partials in a fixed file-scope device array, so a call allocates
// nothing.  Host code must not pass the array's name to a kernel (in host code
// it names a host-side stand-in); the device address is looked up once per
// device with cudaGetSymbolAddress and cached here.
#include <mutex>

#include "lbm_internal.h"

namespace {

constexpr int kPartials = LBM_NOALLOC_MAX_PARTIALS;  // 1024 doubles = 8 KiB per device

// Shared by every call on a device; each call overwrites the slots it uses
// before reading them, so nothing needs clearing between calls.
__device__ __align__(256) double g_mass_partials[kPartials];

template <typename R>
__global__ void k_mass_partial_noalloc(const R *__restrict__ f, int nx, int ny, int walls, double *partials) {
  __shared__ double sh[32];
  const size_t n = (size_t)nx * ny;
  const size_t lo = walls ? (size_t)nx : 0, hi = walls ? n - nx : n;
  const size_t len = hi - lo, chunk = (len + gridDim.x - 1) / gridDim.x;
  const size_t b0 = lo + blockIdx.x * chunk, b1 = min(hi, b0 + chunk);
  double s = 0.0;
  for (size_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    double r = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) r = r + (double)f[a * n + i];
    s += r;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

__global__ void k_mass_final_noalloc(const double *partials, int np, double *out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partials[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) out[0] = t;
  }
}

// Device address of g_mass_partials, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_ptr[kMaxDevices] = {};

int partials_ptr(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return LBM_ECUDA;
    }
    g_ptr[dev] = (double *)p;
  }
  *out = g_ptr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_mass_noalloc(const void *f, int nx, int ny, int precision, int walls, double *mass,
                                void *stream) {
  if (!f || !mass || nx < 1 || (precision != 32 && precision != 64) || (walls != 0 && walls != 1))
    return LBM_EINVAL;
  if (ny < (walls ? 3 : 1)) return LBM_EINVAL;
  if ((size_t)nx * (size_t)ny > (size_t)LBM_NOALLOC_MAX_NODES) return LBM_EINVAL;
  double *partials = nullptr;
  int st = partials_ptr(&partials);
  if (st != LBM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t fluid = (size_t)nx * (size_t)(ny - (walls ? 2 : 0));
  int blocks = (int)((fluid + 255) / 256);
  if (blocks > kPartials) blocks = kPartials;
  if (blocks < 1) blocks = 1;
  if (precision == 64)
    k_mass_partial_noalloc<double><<<blocks, 256, 0, s>>>((const double *)f, nx, ny, walls, partials);
  else
    k_mass_partial_noalloc<float><<<blocks, 256, 0, s>>>((const float *)f, nx, ny, walls, partials);
  k_mass_final_noalloc<<<1, 1024, 0, s>>>(partials, blocks, mass);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
