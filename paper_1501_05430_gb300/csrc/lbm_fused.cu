// lbm_fused.cu -- the single-pass FP32 timestep for sm_103a.
//
// One kernel launch performs the whole step of the pseudo-potential D2Q9 model
// (Eqs. 1-6, 9-11, 14-17, 19-21):
//
//  * Work split: the grid is cut into strips of W = 128 columns; a "unit" is
//    one fluid row of one strip.  The launch is persistent (a few CTAs per
//    SM) and each CTA sweeps one contiguous, equally sized range of units,
//    bottom to top inside each strip.
//  * Loads: one elected thread streams the rows of the CTA's range into a
//    ring of shared-memory stages with TMA (cp.async.bulk.tensor, a 3-D
//    tensor map over [9][ny][nx] with a box of W columns x 1 row x 9 planes),
//    plus two 4-column halo boxes for the periodic x neighbours.  Completion is
//    tracked with mbarriers; every wait is bounded in time and a timeout sets a
//    device flag (LBM_ETIMEOUT) instead of hanging.
//  * Per row: each thread owns one column, sums its 9 populations (rho), maps
//    rho to U and psi (Eq. 10 with the Carnahan-Starling or Eq. 11 EOS) and
//    writes them into a 4-row window; the ghost rows of Eqs. 19-21 are formed
//    in the same window as soon as rows 1-2 (or ny-2, ny-3) are present.
//    With the window holding rows y-1..y+1, row y is collided: Eq. 9 force,
//    Eq. 17 tensor, MRT collision with the Eq. 6 forcing and Eq. 16 source,
//    and the post-collision populations are pushed to the neighbours in the
//    second distribution array (half-way bounce-back on the solid rows).
//  * Bytes: every population is read once from HBM and written once (72 B per
//    node); halo columns and the two extra rows at range ends are re-read
//    mostly from L2.  psi and U never go to HBM.
#include <cuda.h>
#include <math.h>

#include "lbm_internal.h"

namespace {

constexpr int W = 128;             // columns per strip = consumer threads
constexpr int NTHREADS = W + 32;   // + one producer / halo warp
constexpr int HB = 4;              // halo box width (16 bytes of floats)
constexpr int WIN = W + 4;         // window columns: c = -2 .. W+1 at index c+2
constexpr int NSLOT = 4;           // window rows (ring)
constexpr int MAIN_BYTES = 9 * W * 4;
constexpr int HALO_BYTES = 9 * HB * 4;
constexpr int HALO_PAD = 256;
constexpr int STAGE_BYTES = MAIN_BYTES + 2 * HALO_PAD;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per bounded wait

struct FusedArgs {
  int nx, ny, walls, wetting, n_iter, kind;
  int nstrips, nrows, y0;
  long long total;
  int stages;
  float b4, RT, a, thv, thm, thl, r1, r2, p2;  // EOS constants (b/4, R*T, ...)
  float A, omA, pre, halfA, rho_max, ghost_max; // force / Q constants, bounds
  float se, seps, sq, snu;                      // rates
  float he, heps, hq, hnu;                      // 1 - s/2
  float Gw;
  const double *coef;
  float *fout;
  int *flag;
};

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: false after kWaitNs without completion.
__device__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  unsigned long long t0 = gtimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 0 && gtimer() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load3(unsigned dst, const CUtensorMap *map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// The row stream of one CTA: maximal runs ("segments") of its unit range that
// lie in one strip, each visited as virtual rows ya-1 .. yb (the halo rows
// included).  Virtual rows that are solid carry no load.
struct Seq {
  long long u, u1;
  int strip, v, vend, ya, yb;
  bool has;
  __device__ void start(const FusedArgs &P) {
    if (u >= u1) { has = false; return; }
    strip = (int)(u / P.nrows);
    int r0 = (int)(u - (long long)strip * P.nrows);
    long long left = u1 - u;
    int cnt = (int)min(left, (long long)(P.nrows - r0));
    ya = P.y0 + r0;
    yb = ya + cnt;
    v = ya - 1;
    vend = yb;
    u += cnt;
    has = true;
  }
  __device__ void init(const FusedArgs &P, long long a, long long b) { u = a; u1 = b; start(P); }
  __device__ void next(const FusedArgs &P) {
    if (v < vend) ++v; else start(P);
  }
  __device__ bool solid(const FusedArgs &P) const { return P.walls && (v == 0 || v == P.ny - 1); }
};

__device__ __forceinline__ void eos_psiU(const FusedArgs &P, float rho, float &psi, float &U) {
  float p;
  if (P.kind == LBM_EOS_CARNAHAN_STARLING) {
    float e = P.b4 * rho;
    float om = 1.0f - e;
    float num = fmaf(e, fmaf(e, 1.0f - e, 1.0f), 1.0f);
    float den = om * om * om;
    p = rho * P.RT * num * __frcp_rn(den) - P.a * rho * rho;
  } else {
    if (rho <= P.r1) p = rho * P.thv;
    else if (rho <= P.r2) p = fmaf(rho - P.r1, P.thm, P.r1 * P.thv);
    else p = fmaf(rho - P.r2, P.thl, P.p2);
  }
  U = fmaf(rho, -1.0f / 3.0f, p);
  psi = sqrtf(fmaxf(0.0f, -2.0f * U));
}

__global__ void __launch_bounds__(NTHREADS) k_fused(const __grid_constant__ CUtensorMap tm_main,
                                                    const __grid_constant__ CUtensorMap tm_halo, FusedArgs P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned in shared memory
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int S = P.stages;
  unsigned char *stage_base = smem;
  unsigned long long *bars = (unsigned long long *)(smem + (size_t)S * STAGE_BYTES);
  float *win = (float *)(bars + S);  // [NSLOT][3][WIN]: rho, psi, U
  volatile int &s_abort = *(volatile int *)(win + NSLOT * 3 * WIN);

  const int tid = threadIdx.x;
  const bool consumer = tid < W;
  const int lane = tid & 31;
  const bool producer = tid == W;  // lane 0 of the last warp
  const long long G = gridDim.x;
  const long long u0 = (long long)blockIdx.x * P.total / G;
  const long long u1 = (long long)(blockIdx.x + 1) * P.total / G;
  const size_t n = (size_t)P.nx * P.ny;

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  // ---- producer state -----------------------------------------------------
  Seq ps{};
  long long issued = 0;
  auto issue_until = [&](long long limit) {
    while (ps.has && issued < limit) {
      if (!ps.solid(P)) {
        int s = (int)(issued % S);
        unsigned bar = smem_u32(&bars[s]);
        unsigned char *st = stage_base + (size_t)s * STAGE_BYTES;
        int x0 = ps.strip * W;
        int wr = min(W, P.nx - x0);
        int y = ps.v < 0 ? ps.v + P.ny : (ps.v >= P.ny ? ps.v - P.ny : ps.v);
        int xl = x0 - HB < 0 ? x0 - HB + P.nx : x0 - HB;
        int xr = x0 + wr >= P.nx ? x0 + wr - P.nx : x0 + wr;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(MAIN_BYTES + 2 * HALO_BYTES)
                     : "memory");
        tma_load3(smem_u32(st), &tm_main, x0, y, 0, bar);
        tma_load3(smem_u32(st + MAIN_BYTES), &tm_halo, xl, y, 0, bar);
        tma_load3(smem_u32(st + MAIN_BYTES + HALO_PAD), &tm_halo, xr, y, 0, bar);
        ++issued;
      }
      ps.next(P);
    }
  };
  if (producer) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tm_main) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tm_halo) : "memory");
    ps.init(P, u0, u1);
    issue_until(S);
  }

  // ---- consumer / halo state ------------------------------------------------
  Seq cs;
  cs.init(P, u0, u1);
  long long consumed = 0;
  long long it = 0;
  float fcur[9], fnext[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) fcur[a] = fnext[a] = 0.0f;
  bool bad = false;
  const float w1 = 1.0f / 3.0f, w2 = 1.0f / 12.0f;

  while (cs.has) {
    const int v = cs.v;
    const int x0 = cs.strip * W;
    const int wr = min(W, P.nx - x0);
    const int slot = (int)(it & 3);
    float *wrho = win + (size_t)slot * 3 * WIN;
    const bool geo = P.wetting == LBM_WET_GEOMETRIC;
    // column handled by this thread in the row phase
    int c = consumer ? tid : (lane == 0 ? -1 : lane == 1 ? wr : lane == 2 ? -2 : lane == 3 ? wr + 1 : -100);
    bool need2 = P.walls && geo && ((v == 1 && cs.ya == 1) || (v == P.ny - 2 && cs.yb == P.ny - 1));
    bool active = consumer ? (c < wr) : (lane < 2 || (lane < 4 && need2));
    if (!cs.solid(P)) {
      int s = (int)(consumed % S);
      unsigned parity = (unsigned)((consumed / S) & 1);
      unsigned bar = smem_u32(&bars[s]);
      if (!mbar_wait(bar, parity)) {
        s_abort = 1;
        atomicOr(P.flag + 1, 1);
      }
      const float *st = (const float *)(stage_base + (size_t)s * STAGE_BYTES);
      if (active) {
        const float *src;
        int stride;
        if (c >= 0 && c < wr) { src = st + c; stride = W; }
        else if (c < 0) { src = st + MAIN_BYTES / 4 + (HB + c); stride = HB; }
        else { src = st + (MAIN_BYTES + HALO_PAD) / 4 + (c - wr); stride = HB; }
        float f[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) f[a] = src[a * stride];
        float rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        float psi, U;
        eos_psiU(P, rho, psi, U);
        wrho[c + 2] = rho;
        wrho[WIN + c + 2] = psi;
        wrho[2 * WIN + c + 2] = U;
        if (!(rho > 0.0f) || rho > P.rho_max) bad = true;
        if (consumer) {
#pragma unroll
          for (int a = 0; a < 9; ++a) fnext[a] = f[a];
        }
      }
      ++consumed;
      // bottom ghost row (Eqs. 19-21): rows 1 and 2 are now in the window
      if (P.walls && geo && cs.ya == 1 && v == 2 && (consumer ? c < wr : lane < 2)) {
        const float *r1w = win + (size_t)((it - 1) & 3) * 3 * WIN;  // row 1
        float *gw = win + (size_t)((it - 2) & 3) * 3 * WIN;         // row 0
        int gx = x0 + c;
        gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
        float cc = (float)P.coef[gx], cot = (float)P.coef[2 * P.nx + gx];
        float rl = r1w[c + 1], rr = r1w[c + 3], ri1 = r1w[c + 2], ri2 = wrho[c + 2];
        float aa = rr - rl, g;
        if (P.n_iter <= 0) {
          g = fmaf(cot, fabsf(aa), ri2);
        } else {
          float d = 2.0f * (ri2 - ri1);
          g = ri2;
          for (int k = 0; k < P.n_iter; ++k) {
            g = fmaf(cc, sqrtf(fmaf(aa, aa, d * d)), ri2);
            d = ri2 - g;
          }
        }
        g = fminf(fmaxf(g, 0.0f), P.ghost_max);
        float psi = 0.0f, U = 0.0f;  // exact values at the clamp rho_max (root of U)
        if (g < P.rho_max) eos_psiU(P, g, psi, U);
        gw[c + 2] = g;
        gw[WIN + c + 2] = psi;
        gw[2 * WIN + c + 2] = U;
      }
    } else if (v == 0) {
      // bottom solid row: Martys-Chen carries zero potential there; the
      // geometric ghost values are written once rows 1 and 2 are known
      if (!geo && (consumer ? c < wr : lane < 2)) {
        wrho[c + 2] = 0.0f;
        wrho[WIN + c + 2] = 0.0f;
        wrho[2 * WIN + c + 2] = 0.0f;
      }
    } else {
      // top solid row: ghost from rows ny-2 (previous slot) and ny-3
      if (consumer ? c < wr : lane < 2) {
        if (geo) {
          const float *r1w = win + (size_t)((it - 1) & 3) * 3 * WIN;  // row ny-2
          const float *r2w = win + (size_t)((it - 2) & 3) * 3 * WIN;  // row ny-3
          int gx = x0 + c;
          gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
          float cc = (float)P.coef[P.nx + gx], cot = (float)P.coef[3 * P.nx + gx];
          float rl = r1w[c + 1], rr = r1w[c + 3], ri1 = r1w[c + 2], ri2 = r2w[c + 2];
          float aa = rr - rl, g;
          if (P.n_iter <= 0) {
            g = fmaf(cot, fabsf(aa), ri2);
          } else {
            float d = 2.0f * (ri2 - ri1);
            g = ri2;
            for (int k = 0; k < P.n_iter; ++k) {
              g = fmaf(cc, sqrtf(fmaf(aa, aa, d * d)), ri2);
              d = ri2 - g;
            }
          }
          g = fminf(fmaxf(g, 0.0f), P.ghost_max);
          float psi = 0.0f, U = 0.0f;  // exact values at the clamp rho_max (root of U)
          if (g < P.rho_max) eos_psiU(P, g, psi, U);
          wrho[c + 2] = g;
          wrho[WIN + c + 2] = psi;
          wrho[2 * WIN + c + 2] = U;
        } else {
          wrho[c + 2] = 0.0f;
          wrho[WIN + c + 2] = 0.0f;
          wrho[2 * WIN + c + 2] = 0.0f;
        }
      }
    }
    __syncthreads();
    if (s_abort) break;

    // ---- collide row v-1 --------------------------------------------------
    if (consumer && c < wr && v >= cs.ya + 1 && v <= cs.yb) {
      const int y = v - 1;
      const float *wm = win + (size_t)((it - 2) & 3) * 3 * WIN;  // row y-1
      const float *w0 = win + (size_t)((it - 1) & 3) * 3 * WIN;  // row y
      const float *wp = wrho;                                      // row y+1
      const int i0 = c + 2;
      float psi0 = w0[WIN + i0];
      float rho = w0[i0];
      // neighbour potentials, e1..e8
      float p1 = w0[WIN + i0 + 1], p3 = w0[WIN + i0 - 1];
      float p2 = wp[WIN + i0], p4 = wm[WIN + i0];
      float p5 = wp[WIN + i0 + 1], p6 = wp[WIN + i0 - 1];
      float p7 = wm[WIN + i0 - 1], p8 = wm[WIN + i0 + 1];
      float u1 = w0[2 * WIN + i0 + 1], u3 = w0[2 * WIN + i0 - 1];
      float u2 = wp[2 * WIN + i0], u4 = wm[2 * WIN + i0];
      float u5 = wp[2 * WIN + i0 + 1], u6 = wp[2 * WIN + i0 - 1];
      float u7 = wm[2 * WIN + i0 - 1], u8 = wm[2 * WIN + i0 + 1];
      // Eq. 9
      float spx = fmaf(w1, p1 - p3, w2 * ((p5 - p6) + (p8 - p7)));
      float spy = fmaf(w1, p2 - p4, w2 * ((p5 + p6) - (p7 + p8)));
      float sux = fmaf(w1, u1 - u3, w2 * ((u5 - u6) + (u8 - u7)));
      float suy = fmaf(w1, u2 - u4, w2 * ((u5 + u6) - (u7 + u8)));
      // F = -A sum w U e - (1-A) G psi sum w psi e with G = -1
      float cpsi = P.omA * psi0;  // (1 - A) psi
      float Fx = fmaf(cpsi, spx, -P.A * sux);
      float Fy = fmaf(cpsi, spy, -P.A * suy);
      if (P.wetting == LBM_WET_MARTYS_CHEN && P.walls) {
        // Eq. 14 for flat solid rows: sum_a w_a S e_a = (0, -1/2) below, (0, 1/2) above
        float ssy = (y == 1 ? -0.5f : 0.0f) + (y == P.ny - 2 ? 0.5f : 0.0f);
        Fy = fmaf(-P.Gw * psi0, ssy, Fy);
      }
      // Eq. 17 (with its G/2 prefactor)
      float sd = (p5 + p6) + (p7 + p8);
      float q0 = 4.0f * psi0;
      float qxx1 = fmaf(w1, (p1 + p3) - 0.5f * q0, w2 * (sd - q0));
      float qyy1 = fmaf(w1, (p2 + p4) - 0.5f * q0, w2 * (sd - q0));
      float qxy1 = w2 * ((p5 + p7) - (p6 + p8));
      float s0 = psi0 * psi0;
      float t1 = p1 * p1, t2 = p2 * p2, t3 = p3 * p3, t4 = p4 * p4;
      float t5 = p5 * p5, t6 = p6 * p6, t7 = p7 * p7, t8 = p8 * p8;
      float td = (t5 + t6) + (t7 + t8);
      float qxx2 = fmaf(w1, (t1 + t3) - 2.0f * s0, w2 * (td - 4.0f * s0));
      float qyy2 = fmaf(w1, (t2 + t4) - 2.0f * s0, w2 * (td - 4.0f * s0));
      float qxy2 = w2 * ((t5 + t7) - (t6 + t8));
      float c1 = P.omA * psi0;
      float Qxx = P.pre * fmaf(c1, qxx1, P.halfA * qxx2);
      float Qyy = P.pre * fmaf(c1, qyy1, P.halfA * qyy2);
      float Qxy = P.pre * fmaf(c1, qxy1, P.halfA * qxy2);
      // moments of f (Eq. 4 ordering)
      const float *f = fcur;
      float a13 = f[1] + f[3], s13 = f[1] - f[3];
      float a24 = f[2] + f[4], s24 = f[2] - f[4];
      float d57 = f[5] - f[7], d86 = f[8] - f[6];
      float ax = a13 + a24, dg = (f[5] + f[6]) + (f[7] + f[8]);
      float jx = s13 + d57 + d86;
      float jy = s24 + d57 - d86;
      float me = fmaf(-4.0f, f[0], fmaf(2.0f, dg, -ax));
      float meps = fmaf(4.0f, f[0], fmaf(-2.0f, ax, dg));
      float mqx = fmaf(-2.0f, s13, d57 + d86);
      float mqy = fmaf(-2.0f, s24, d57 - d86);
      float mpxx = a13 - a24;
      float mpxy = (f[5] + f[7]) - (f[6] + f[8]);
      // velocity with the half-force shift
      float ir = __frcp_rn(rho);
      float vx = fmaf(0.5f, Fx, jx) * ir, vy = fmaf(0.5f, Fy, jy) * ir;
      float v2 = fmaf(vx, vx, vy * vy);
      float vF = fmaf(vx, Fx, vy * Fy);
      // relaxation (Eq. 15) with forcing S (Eq. 6) and source C (Eq. 16)
      float e_eq = rho * fmaf(3.0f, v2, -2.0f);
      float eps_eq = rho * fmaf(-3.0f, v2, 1.0f);
      float es = fmaf(-P.se, me - e_eq, me) + P.he * 6.0f * vF + 1.5f * P.se * (Qxx + Qyy);
      float epss = fmaf(-P.seps, meps - eps_eq, meps) - P.heps * 6.0f * vF;
      float qxs = fmaf(-P.sq, mqx + rho * vx, mqx) - P.hq * Fx;
      float qys = fmaf(-P.sq, mqy + rho * vy, mqy) - P.hq * Fy;
      float pxxs = fmaf(-P.snu, mpxx - rho * (vx * vx - vy * vy), mpxx) +
                   P.hnu * 2.0f * (vx * Fx - vy * Fy) - P.snu * (Qxx - Qyy);
      float pxys = fmaf(-P.snu, mpxy - rho * vx * vy, mpxy) + P.hnu * fmaf(vx, Fy, vy * Fx) - P.snu * Qxy;
      float jxs = jx + Fx, jys = jy + Fy;
      // back to populations: f* = M^T diag(1/N) m*
      // rho/9 correctly rounded: a biased 1/9 constant would leak mass every step
      float r0 = __fdiv_rn(rho, 9.0f), r1 = es * (1.0f / 36.0f), r2 = epss * (1.0f / 36.0f);
      float r3 = jxs * (1.0f / 6.0f), r4 = qxs * (1.0f / 12.0f), r5 = jys * (1.0f / 6.0f),
            r6 = qys * (1.0f / 12.0f);
      float r7 = pxxs * 0.25f, r8 = pxys * 0.25f;
      float fs[9];
      fs[0] = fmaf(4.0f, r2 - r1, r0);
      float Aax = fmaf(-2.0f, r2, r0 - r1);
      float Bdg = fmaf(2.0f, r1, r0 + r2);
      float X1 = fmaf(-2.0f, r4, r3), Y1 = fmaf(-2.0f, r6, r5);
      fs[1] = (Aax + X1) + r7;
      fs[3] = (Aax - X1) + r7;
      fs[2] = (Aax + Y1) - r7;
      fs[4] = (Aax - Y1) - r7;
      float X2 = r3 + r4, Y2 = r5 + r6;
      fs[5] = (Bdg + X2) + (Y2 + r8);
      fs[6] = (Bdg - X2) + (Y2 - r8);
      fs[7] = (Bdg - X2) - (Y2 - r8);
      fs[8] = (Bdg + X2) - (Y2 + r8);
      // streaming with half-way bounce-back
      const int x = x0 + c;
      const int xm = x == 0 ? P.nx - 1 : x - 1, xp = x == P.nx - 1 ? 0 : x + 1;
      const int ym = y == 0 ? P.ny - 1 : y - 1, yp = y == P.ny - 1 ? 0 : y + 1;
      const bool wall_dn = P.walls && y == 1, wall_up = P.walls && y == P.ny - 2;
      float *out = P.fout;
      const size_t ry = (size_t)y * P.nx, rym = (size_t)ym * P.nx, ryp = (size_t)yp * P.nx;
      out[0 * n + ry + x] = fs[0];
      out[1 * n + ry + xp] = fs[1];
      out[3 * n + ry + xm] = fs[3];
      if (wall_up) {
        out[4 * n + ry + x] = fs[2];
        out[7 * n + ry + x] = fs[5];
        out[8 * n + ry + x] = fs[6];
      } else {
        out[2 * n + ryp + x] = fs[2];
        out[5 * n + ryp + xp] = fs[5];
        out[6 * n + ryp + xm] = fs[6];
      }
      if (wall_dn) {
        out[2 * n + ry + x] = fs[4];
        out[5 * n + ry + x] = fs[7];
        out[6 * n + ry + x] = fs[8];
      } else {
        out[4 * n + rym + x] = fs[4];
        out[7 * n + rym + xm] = fs[7];
        out[8 * n + rym + xp] = fs[8];
      }
    }
    if (consumer) {
#pragma unroll
      for (int a = 0; a < 9; ++a) fcur[a] = fnext[a];
    }
    if (producer) issue_until(consumed + S);
    ++it;
    cs.next(P);
  }

  if (s_abort && producer) {
    // drain the loads still in flight (bounded) before the CTA exits
    for (long long k = consumed - 1; k < issued; ++k) {
      int s = (int)(k % S);
      mbar_wait(smem_u32(&bars[s]), (unsigned)((k / S) & 1));
    }
  }
  if (bad) atomicOr(P.flag, 1);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encoder() {
  static EncodeTiledFn fn = nullptr;
  if (fn) return fn;
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  fn = (EncodeTiledFn)p;
  return fn;
}

bool encode(CUtensorMap *m, void *base, int nx, int ny, int boxw) {
  EncodeTiledFn enc = get_encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
  cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  cuuint32_t box[3] = {(cuuint32_t)boxw, 1, 9};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t smem_bytes(int stages) {
  return 128 + (size_t)stages * STAGE_BYTES + (size_t)stages * 8 + (size_t)NSLOT * 3 * WIN * sizeof(float) + 16;
}

}  // namespace

int lbm_fused_plan(lbm_ctx *C) {
  C->fused_ok = 0;
  if (C->precision != 32 || (C->nx % 4) != 0) return 0;
  static_assert(sizeof(CUtensorMap) <= sizeof(C->tmaps[0]), "tensor map storage");
  for (int b = 0; b < 2; ++b) {
    if (!encode((CUtensorMap *)C->tmaps[2 * b], C->f[b], C->nx, C->ny, W)) return 0;
    if (!encode((CUtensorMap *)C->tmaps[2 * b + 1], C->f[b], C->nx, C->ny, HB)) return 0;
  }
  int stages = 6;
  size_t smem = smem_bytes(stages);
  if (cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused, NTHREADS, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return 0;
  }
  int nstrips = (C->nx + W - 1) / W;
  int nrows = C->walls ? C->ny - 2 : C->ny;
  long long total = (long long)nstrips * nrows;
  long long blocks = (long long)nsm * occ;
  if (blocks > total) blocks = total;
  C->tile_w = W;
  C->tile_stages = stages;
  C->tile_blocks = (int)blocks;
  C->fused_smem = (int)smem;
  C->fused_ok = 1;
  return 1;
}

cudaError_t lbm_fused_step(lbm_ctx *C, int src, unsigned long long *launches) {
  FusedArgs P;
  const lbm_dev_params &D = C->dp;
  P.nx = C->nx;
  P.ny = C->ny;
  P.walls = C->walls;
  P.wetting = D.wetting;
  P.n_iter = D.n_iter;
  P.kind = D.eos_kind;
  P.nstrips = (C->nx + W - 1) / W;
  P.nrows = C->walls ? C->ny - 2 : C->ny;
  P.y0 = C->walls ? 1 : 0;
  P.total = (long long)P.nstrips * P.nrows;
  P.stages = C->tile_stages;
  P.b4 = (float)(0.25 * D.b);
  P.RT = (float)(D.R * D.T);
  P.a = (float)D.a;
  P.thv = (float)D.thv;
  P.thm = (float)D.thm;
  P.thl = (float)D.thl;
  P.r1 = (float)D.r1;
  P.r2 = (float)D.r2;
  P.p2 = (float)(D.r1 * D.thv + (D.r2 - D.r1) * D.thm);
  P.A = (float)D.A;
  P.omA = (float)(1.0 - D.A);
  P.pre = (float)(-0.5 * D.kappa);
  P.halfA = (float)(0.5 * D.A);
  P.rho_max = (float)fmin(D.rho_max, 3.0e38);
  P.ghost_max = (float)fmin(D.ghost_max, 3.0e38);
  P.se = (float)D.s[1];
  P.seps = (float)D.s[2];
  P.sq = (float)D.s[4];
  P.snu = (float)D.s[7];
  P.he = (float)(1.0 - 0.5 * D.s[1]);
  P.heps = (float)(1.0 - 0.5 * D.s[2]);
  P.hq = (float)(1.0 - 0.5 * D.s[4]);
  P.hnu = (float)(1.0 - 0.5 * D.s[7]);
  P.Gw = (float)D.Gw;
  P.coef = C->d_coef;
  P.fout = (float *)C->f[src ^ 1];
  P.flag = C->d_flag;
  const CUtensorMap *tm = (const CUtensorMap *)C->tmaps[2 * src];
  const CUtensorMap *th = (const CUtensorMap *)C->tmaps[2 * src + 1];
  k_fused<<<C->tile_blocks, NTHREADS, C->fused_smem, C->stream>>>(*tm, *th, P);
  ++*launches;
  return cudaGetLastError();
}
