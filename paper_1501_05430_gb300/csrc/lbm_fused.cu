// lbm_fused.cu -- the single-pass FP32 timestep for sm_103a.
//
// One kernel launch performs the whole step of the pseudo-potential D2Q9 model
// (Eqs. 1-6, 9-11, 14-17, 19-21):
//
//  * Work split: the grid is cut into strips of W = 256 columns; a "unit" is
//    one fluid row of one strip.  The launch is persistent (4 CTAs of 128
//    threads per SM) and each CTA sweeps one contiguous, equally sized range
//    of units, bottom to top inside each strip.
//  * Loads: one elected thread streams the rows of the CTA's range into a
//    ring of shared-memory stages with TMA (cp.async.bulk.tensor, a 3-D
//    tensor map over [9][ny][nx] with a box of W columns x 1 row x 9 planes),
//    plus two 4-column halo boxes for the periodic x neighbours.  Completion is
//    tracked with mbarriers; every wait is bounded in time and a timeout sets a
//    device flag (LBM_ETIMEOUT) instead of hanging.
//  * Per row: each thread owns columns t and t + 128 as one lane pair, keeps
//    their 9 populations in registers, sums rho for both with packed FP32
//    adds, maps rho to psi and psi^2 (Eq. 10 with the Carnahan-Starling or
//    Eq. 11 EOS) and writes them into a 4-row window laid out in lane pairs;
//    the ghost rows of Eqs. 19-21 are formed in the same window as soon as
//    rows 1-2 (or ny-2, ny-3) are present.  With the window holding rows
//    y-1..y+1, row y is collided, both columns per packed instruction: Eq. 9
//    force, Eq. 17 tensor, MRT collision with the Eq. 6 forcing and Eq. 16
//    source, and the post-collision populations are pushed to the neighbours
//    in the second distribution array (half-way bounce-back on the solid rows).
//  * Bytes: every population is read once from HBM and written once (72 B per
//    node); halo columns and the two extra rows at range ends are re-read
//    mostly from L2.  psi and U never go to HBM.
#include <cuda.h>
#include <math.h>
#include <stdlib.h>

#include "lbm_internal.h"
#include "lbm_node.cuh"

namespace {

using lbm_node::add2;
using lbm_node::collide_node2;
using lbm_node::eos_node;
using lbm_node::eos_node2;
using lbm_node::ghost_node;
using lbm_node::sqrt0;

constexpr int NCONS = 128;               // threads per CTA (4 warps)
constexpr int HB = 4;                    // halo box width (16 bytes of floats)
constexpr int NSLOT = 4;                 // window rows (ring)
constexpr int HALO_BYTES = 9 * HB * 4;
constexpr int HALO_PAD = 256;

// Launch shape for NC columns per thread: strips of W = 128 NC columns.
template <int NC>
struct Cfg {
  static constexpr int W = NC * NCONS;                          // columns per strip
  static constexpr int WIN = W + 4;                             // window columns c = -2 .. W+1
  static constexpr int WP = NCONS + 4;                          // paired window entries i = -2 .. NCONS+1
  static constexpr int MAIN_BYTES = 9 * W * 4;                  // 9 planes x W floats
  static constexpr int STAGE_BYTES = MAIN_BYTES + 2 * HALO_PAD;
  static constexpr int MIN_CTAS = 4;                            // register budget per thread
};
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per bounded wait

struct FusedArgs {
  int nx, ny, walls, wetting, n_iter, kind;
  int nstrips, nrows, y0;
  long long total;
  int stages;
  float b4, RT2, a2, r1, r2, pc0, pc1, pc2;    // EOS constants (b/4, -2RT, 2a; Eq. 11 break-
                                                // points and slopes folded into -2U)
  float A, omA, pre, halfA, rho_max, ghost_max; // force / Q constants, bounds
  lbm_node::RateK k;                            // relaxation constants
  float Gw;
  long long eoff[9];  // byte offset of plane a's destination from (row y, column x) of plane 0 for an
                      // interior node: 4 (a n + e_ay nx + e_ax) (streaming without wrap or bounce-back)
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

// Test an mbarrier phase; a thread that finds it incomplete is suspended by
// the hardware for up to ~0.5 ms (the suspend-time hint) or until the phase
// completes, instead of spinning through issue slots.
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(500000u)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: false after kWaitNs without completion.
__device__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  unsigned long long t0 = gtimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (gtimer() - t0 > kWaitNs) return false;
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

template <bool UNIT, int NC, int MCW, int KIND>
__global__ void __launch_bounds__(NCONS, Cfg<NC>::MIN_CTAS)
    k_fused(const __grid_constant__ CUtensorMap tm_main, const __grid_constant__ CUtensorMap tm_halo, FusedArgs P) {
  static_assert(NC == 2, "two columns per thread: one lane pair");
  constexpr int W = Cfg<NC>::W, WIN = Cfg<NC>::WIN, WP = Cfg<NC>::WP, MAIN_BYTES = Cfg<NC>::MAIN_BYTES;
  constexpr int STAGE_BYTES = Cfg<NC>::STAGE_BYTES;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned in shared memory
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int S = P.stages;
  unsigned char *stage_base = smem;
  // window rows: psi and psi^2 in lane pairs -- entry i holds columns i and
  // i + NCONS, i in [-2, NCONS + 1] at index i + 2 -- so that a thread's two
  // columns (t, t + NCONS) and their x neighbours are one 64-bit load each;
  // rho in column order (column c at c + 2, c in [-2, W + 1])
  float2 *wpsi = (float2 *)(smem + (size_t)S * STAGE_BYTES);  // [NSLOT][WP]
  float2 *wsq = wpsi + NSLOT * WP;                            // [NSLOT][WP]
  float *winr = (float *)(wsq + NSLOT * WP);                  // [NSLOT][WIN]
  unsigned long long *bars = (unsigned long long *)(winr + NSLOT * WIN);
  volatile int &s_abort = *(volatile int *)(bars + S);

  const int tid = threadIdx.x;
  const bool producer = tid == 0;
  // the four top lanes of the last warp also form the halo columns:
  // -1 and wr (always), -2 and wr+1 (rows whose ghost needs them)
  const int hidx = tid - (NCONS - 4);
  const long long G = gridDim.x;
  const long long u0 = (long long)blockIdx.x * P.total / G;
  const long long u1 = (long long)(blockIdx.x + 1) * P.total / G;
  const size_t n = (size_t)P.nx * P.ny;
  const bool geo = P.wetting == LBM_WET_GEOMETRIC;

  // Programmatic dependent launch: the next step's grid may be scheduled once
  // every CTA of this one has started (all of them are resident: the grid is
  // one wave), so its CTAs take the slots of this grid's first finishers and
  // do their set-up there; before touching global memory every thread waits
  // until the previous grid has completed and its stores are visible (a
  // no-op for a launch without a programmatic dependency).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tm_main) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tm_halo) : "memory");
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();

  // ---- producer -------------------------------------------------------------
  Seq ps{};
  int issued = 0, put_stage = 0;  // loads issued; ring slot of the next load
  auto issue_until = [&](int limit) {
    if (ps.has && issued < limit) {
      // order the generic-proxy reads of the stages being refilled before
      // the asynchronous-proxy writes of the new loads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    while (ps.has && issued < limit) {
      if (!ps.solid(P)) {
        const int s = put_stage;
        put_stage = put_stage + 1 == S ? 0 : put_stage + 1;
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
    ps.init(P, u0, u1);
    issue_until(S);
  }

  // ---- row sweep --------------------------------------------------------------
  // A stage is read once, when its row enters the window (iteration i): each
  // thread keeps the populations of its two columns in registers (lane pairs)
  // until the row is collided in iteration i+1.  The stage is free after the
  // barrier of iteration i, so the producer refills up to (loads consumed) +
  // S.  Two register sets alternate between the "entering" and the
  // "colliding" row (the loop body is instantiated twice with the sets
  // swapped).
  Seq cs;
  cs.init(P, u0, u1);
  int consumed = 0;                             // loads consumed
  int get_stage = 0;                            // ring slot of the next load to consume
  unsigned get_phase = 0;                       // its mbarrier phase parity
  int it = 0;
  bool bad = false;
  // thread t owns columns t and t + NCONS: unit-stride shared-memory and
  // global accesses across the warp for each of them
  float2 fA[9], fB[9];
  // (psi, psi^2) of column c into a window row pair: lane 0 of entry c and/or
  // lane 1 of entry c - NCONS
  auto put = [&](float2 *ps, float2 *sq, int c, float p, float q) {
    if (c <= NCONS + 1) {
      ps[c + 2].x = p;
      sq[c + 2].x = q;
    }
    if (c >= NCONS - 2) {
      ps[c - NCONS + 2].y = p;
      sq[c - NCONS + 2].y = q;
    }
  };

  auto body = [&](float2 (&fin)[9], const float2 (&fcol)[9]) -> bool {
    const int v = cs.v;
    const int x0 = cs.strip * W;
    const int wr = min(W, P.nx - x0);
    float2 *pcur = wpsi + (size_t)(it & 3) * WP, *qcur = wsq + (size_t)(it & 3) * WP;
    float *rcur = winr + (size_t)(it & 3) * WIN;
    const bool need2 = P.walls && geo && ((v == 1 && cs.ya == 1) || (v == P.ny - 2 && cs.yb == P.ny - 1));
    const int hc = hidx == 0 ? -1 : hidx == 1 ? wr : hidx == 2 ? -2 : wr + 1;
    const bool hact = hidx >= 0 && (hidx < 2 || need2);
    const bool hact2 = hidx >= 0 && hidx < 2;  // halo columns that get a ghost value
    const int c0 = tid, c1 = tid + NCONS;
    const bool act0 = c0 < wr, act1 = c1 < wr;  // act1 implies act0
    if (!cs.solid(P)) {
      const int s = get_stage;
      const unsigned ph = get_phase;
      if (++get_stage == S) {
        get_stage = 0;
        get_phase ^= 1u;
      }
      if (!mbar_wait(smem_u32(&bars[s]), ph)) {
        s_abort = 1;
        atomicOr(P.flag + 1, 1);
      }
      const float *st = (const float *)(stage_base + (size_t)s * STAGE_BYTES);
      if (act0) {
        const float *q0 = st + c0, *q1 = st + (act1 ? c1 : c0);
#pragma unroll
        for (int a = 0; a < 9; ++a) fin[a] = make_float2(q0[a * W], q1[a * W]);
        // rho of both columns, summed in the same order for each
        const float2 r = add2(add2(add2(add2(fin[0], fin[1]), add2(fin[2], fin[3])),
                                   add2(add2(fin[4], fin[5]), add2(fin[6], fin[7]))),
                              fin[8]);
        float2 ps, ps2;
        eos_node2<KIND>(P, r, ps, ps2);
        // unstable unless 0 < rho <= rho_max, tested on the bits: positive
        // floats order like their bit patterns, and -0, negatives, +inf and
        // NaN all land at or above rho_max's pattern after the decrement
        const unsigned mx = __float_as_uint(P.rho_max);
        if (act1) {
          // both columns: window entry c0 + 2 is the pair (c0, c1), one
          // 64-bit store per quantity; the periodic copies as in put()
          pcur[c0 + 2] = ps;
          qcur[c0 + 2] = ps2;
          if (c0 >= NCONS - 2) {
            pcur[c0 - NCONS + 2].y = ps.x;
            qcur[c0 - NCONS + 2].y = ps2.x;
          }
          if (c1 <= NCONS + 1) {
            pcur[c1 + 2].x = ps.y;
            qcur[c1 + 2].x = ps2.y;
          }
          rcur[c0 + 2] = r.x;
          rcur[c1 + 2] = r.y;
          bad |= (__float_as_uint(r.x) - 1u >= mx) | (__float_as_uint(r.y) - 1u >= mx);
        } else {
          rcur[c0 + 2] = r.x;
          put(pcur, qcur, c0, ps.x, ps2.x);
          bad |= __float_as_uint(r.x) - 1u >= mx;
        }
      }
      if (hact) {
        const float *src = hc < 0 ? st + MAIN_BYTES / 4 + (HB + hc) : st + (MAIN_BYTES + HALO_PAD) / 4 + (hc - wr);
        float r = (((src[0] + src[HB]) + (src[2 * HB] + src[3 * HB])) +
                   ((src[4 * HB] + src[5 * HB]) + (src[6 * HB] + src[7 * HB]))) +
                  src[8 * HB];
        const float4 e = eos_node<KIND>(P, r);
        rcur[hc + 2] = r;
        put(pcur, qcur, hc, e.y, e.z);
      }
      ++consumed;
      // bottom ghost row (Eqs. 19-21): rows 1 and 2 are now in the window
      if (P.walls && geo && cs.ya == 1 && v == 2) {
        const float *r1w = winr + (size_t)((it - 1) & 3) * WIN;  // row 1 densities
        float2 *gp = wpsi + (size_t)((it - 2) & 3) * WP;         // row 0
        float2 *gq = wsq + (size_t)((it - 2) & 3) * WP;
        float *gr = winr + (size_t)((it - 2) & 3) * WIN;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const int c = tid + j * NCONS;
          if (c < wr) {
            const float4 e = ghost_node<KIND>(P, r1w, rcur, c, x0 + c, 0);
            gr[c + 2] = e.x;
            put(gp, gq, c, e.y, e.z);
          }
        }
        if (hact2) {
          int gx = x0 + hc;
          gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
          const float4 e = ghost_node<KIND>(P, r1w, rcur, hc, gx, 0);
          gr[hc + 2] = e.x;
          put(gp, gq, hc, e.y, e.z);
        }
      }
    } else {
      // solid row: zero potential (Martys-Chen), or the top ghost row from rows
      // ny-2 and ny-3 (the bottom ghost row is filled at v == 2)
      const bool top = v != 0;
      const float *r1w = winr + (size_t)((it - 1) & 3) * WIN;
      const float *r2w = winr + (size_t)((it - 2) & 3) * WIN;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const int c = tid + j * NCONS;
        if (c < wr) {
          if (!geo) {
            rcur[c + 2] = 0.0f;
            put(pcur, qcur, c, 0.0f, 0.0f);
          } else if (top) {
            const float4 e = ghost_node<KIND>(P, r1w, r2w, c, x0 + c, 1);
            rcur[c + 2] = e.x;
            put(pcur, qcur, c, e.y, e.z);
          }
        }
      }
      if (hact2) {
        if (!geo) {
          rcur[hc + 2] = 0.0f;
          put(pcur, qcur, hc, 0.0f, 0.0f);
        } else if (top) {
          int gx = x0 + hc;
          gx = gx < 0 ? gx + P.nx : (gx >= P.nx ? gx - P.nx : gx);
          const float4 e = ghost_node<KIND>(P, r1w, r2w, hc, gx, 1);
          rcur[hc + 2] = e.x;
          put(pcur, qcur, hc, e.y, e.z);
        }
      }
    }
    __syncthreads();
    if (s_abort) return false;

    // ---- collide row v-1 (its populations are in registers since the last iteration) ----
    if (act0 && v >= cs.ya + 1 && v <= cs.yb) {
      const int y = v - 1;
      const float2 *pm = wpsi + (size_t)((it - 2) & 3) * WP, *qm = wsq + (size_t)((it - 2) & 3) * WP;  // row y-1
      const float2 *p0 = wpsi + (size_t)((it - 1) & 3) * WP, *q0 = wsq + (size_t)((it - 1) & 3) * WP;  // row y
      const float2 *pp = pcur, *qp = qcur;                                                               // row y+1
      const float *r0w = winr + (size_t)((it - 1) & 3) * WIN;
      const int ym = y == 0 ? P.ny - 1 : y - 1, yp = y == P.ny - 1 ? 0 : y + 1;
      const bool wall_dn = P.walls && y == 1, wall_up = P.walls && y == P.ny - 2;
      // per-plane output pointers are warp-uniform; each store adds one 32-bit
      // element offset (9 nx ny < 2^31 is checked at creation)
      float *const o0p = P.fout, *const o1p = o0p + n, *const o2p = o1p + n, *const o3p = o2p + n;
      float *const o4p = o3p + n, *const o5p = o4p + n, *const o6p = o5p + n, *const o7p = o6p + n;
      float *const o8p = o7p + n;
      const unsigned ry = (unsigned)y * P.nx, rym = (unsigned)ym * P.nx, ryp = (unsigned)yp * P.nx;
      // streaming with half-way bounce-back of node x's post-collision populations
      auto push = [&](int x, float f0, float f1, float f2, float f3, float f4, float f5, float f6, float f7,
                      float f8) {
        const unsigned xm = x == 0 ? P.nx - 1 : x - 1, xp = x == P.nx - 1 ? 0 : x + 1;
        o0p[ry + x] = f0;
        o1p[ry + xp] = f1;
        o3p[ry + xm] = f3;
        if (wall_up) {
          o4p[ry + x] = f2;
          o7p[ry + x] = f5;
          o8p[ry + x] = f6;
        } else {
          o2p[ryp + x] = f2;
          o5p[ryp + xp] = f5;
          o6p[ryp + xm] = f6;
        }
        if (wall_dn) {
          o2p[ry + x] = f4;
          o5p[ry + x] = f7;
          o6p[ry + x] = f8;
        } else {
          o4p[rym + x] = f4;
          o7p[rym + xm] = f7;
          o8p[rym + xp] = f8;
        }
      };
      // both columns at once with the packed FP32 instructions (the second
      // lane is computed even past a ragged strip end; it is not stored)
      const int i = tid + 2;
      float2 pn[9], qn[9], fs2[9];
      pn[0] = p0[i];
      qn[0] = q0[i];
      pn[1] = p0[i + 1];
      qn[1] = q0[i + 1];
      pn[2] = pp[i];
      qn[2] = qp[i];
      pn[3] = p0[i - 1];
      qn[3] = q0[i - 1];
      pn[4] = pm[i];
      qn[4] = qm[i];
      pn[5] = pp[i + 1];
      qn[5] = qp[i + 1];
      pn[6] = pp[i - 1];
      qn[6] = qp[i - 1];
      pn[7] = pm[i - 1];
      qn[7] = qm[i - 1];
      pn[8] = pm[i + 1];
      qn[8] = qm[i + 1];
      collide_node2<UNIT, MCW>(P, fcol, pn, qn, make_float2(r0w[c0 + 2], r0w[c1 + 2]), y, fs2);
      if (!UNIT && !wall_dn && !wall_up && y >= 1 && y <= P.ny - 2 && x0 >= 1 && x0 + W <= P.nx - 1) {
        // a row away from the walls and the y wrap, in a strip away from the x wrap:
        // every destination is a fixed offset from the node, and column c1
        // is NCONS floats after column c0, so one address per plane serves both
        // (measured at 4096 x 2048: general-rate step 112.2 -> 111.2 us; the
        // unit-rate step ran slower with it, 104.5 -> 107.2 us, and keeps push)
        char *const a = (char *)(P.fout + ((size_t)ry + (size_t)(x0 + c0)));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          float *const d = (float *)(a + P.eoff[k]);
          d[0] = fs2[k].x;
          d[NCONS] = fs2[k].y;
        }
      } else {
        push(x0 + c0, fs2[0].x, fs2[1].x, fs2[2].x, fs2[3].x, fs2[4].x, fs2[5].x, fs2[6].x, fs2[7].x, fs2[8].x);
        if (act1)
          push(x0 + c1, fs2[0].y, fs2[1].y, fs2[2].y, fs2[3].y, fs2[4].y, fs2[5].y, fs2[6].y, fs2[7].y, fs2[8].y);
      }
    }
    if (producer) issue_until(consumed + S);
    ++it;
    cs.next(P);
    return cs.has;
  };
  if (cs.has) {  // (every range holds a unit: the grid has at most `total` CTAs)
    while (body(fA, fB) && body(fB, fA)) {
    }
  }

  if (s_abort && producer) {
    // drain the loads still in flight (bounded) before the CTA exits
    for (int k = max(consumed - 1, 0); k < issued; ++k) mbar_wait(smem_u32(&bars[k % S]), (unsigned)((k / S) & 1));
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

constexpr int kNC = 2;  // columns per thread

size_t smem_bytes(int stages) {
  using C = Cfg<kNC>;
  return 128 + (size_t)stages * C::STAGE_BYTES + (size_t)NSLOT * C::WP * 2 * sizeof(float2) +
         (size_t)NSLOT * C::WIN * sizeof(float) + (size_t)stages * 8 + 16;
}

// the eight specialisations: collision (unit or general rates) x wetting
// rule (geometric or Martys-Chen) x EOS (Carnahan-Starling or Eq. 11), each
// fixed at compile time so that no branch is left in the per-node arithmetic
typedef void (*FusedKernel)(CUtensorMap, CUtensorMap, FusedArgs);
template <bool UNIT, int MCW>
FusedKernel pick_kind(int kind) {
  return kind == LBM_EOS_CARNAHAN_STARLING ? (FusedKernel)k_fused<UNIT, kNC, MCW, LBM_EOS_CARNAHAN_STARLING>
                                           : (FusedKernel)k_fused<UNIT, kNC, MCW, LBM_EOS_PIECEWISE>;
}
FusedKernel kernel_ptr(bool unit, bool mc, int kind) {
  if (mc) return unit ? pick_kind<true, 1>(kind) : pick_kind<false, 1>(kind);
  return unit ? pick_kind<true, 0>(kind) : pick_kind<false, 0>(kind);
}

}  // namespace

int lbm_fused_plan(lbm_ctx *C) {
  C->fused_ok = 0;
  if (C->precision != 32 || (C->nx % 4) != 0) return 0;
  static_assert(sizeof(CUtensorMap) <= sizeof(C->tmaps[0]), "tensor map storage");
  // tuning knobs (defaults measured on GB300): TMA ring depth and CTAs per SM
  const int nc = kNC;
  int stages = 3;
  if (const char *e = getenv("LBM_FUSED_STAGES")) stages = atoi(e);
  if (stages < 3 || stages > 12) stages = 3;
  const int W = nc * NCONS;
  for (int b = 0; b < 2; ++b) {
    if (!encode((CUtensorMap *)C->tmaps[2 * b], C->f[b], C->nx, C->ny, W)) return 0;
    if (!encode((CUtensorMap *)C->tmaps[2 * b + 1], C->f[b], C->nx, C->ny, HB)) return 0;
  }
  size_t smem = smem_bytes(stages);
  // the diag(0,1,...,1) relaxation of Sec. 3.1 takes the specialised collision
  const lbm_dev_params &D = C->dp;
  C->fused_unit = D.s[1] == 1.0 && D.s[2] == 1.0 && D.s[4] == 1.0 && D.s[7] == 1.0;
  const void *kern = (const void *)kernel_ptr(C->fused_unit, D.wetting == LBM_WET_MARTYS_CHEN, D.eos_kind);
  int dev = 0, nsm = 0, occ = 0, optin = 0;
  cudaGetDevice(&dev);
  // the attribute is per kernel, not per context: allow the device maximum so
  // that contexts planned with different ring depths coexist
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int dyn_max = optin - (int)fa.sharedSizeBytes;  // static + dynamic <= the opt-in limit
  if ((int)smem > dyn_max ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NCONS, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return 0;
  }
  int nstrips = (C->nx + W - 1) / W;
  int nrows = C->walls ? C->ny - 2 : C->ny;
  long long total = (long long)nstrips * nrows;
  if (const char *e = getenv("LBM_FUSED_CTAS_PER_SM")) {
    int want = atoi(e);
    if (want >= 1 && want < occ) occ = want;
  }
  long long blocks = (long long)nsm * occ;
  if (blocks > total) blocks = total;
  C->fused_cols = nc;
  C->tile_w = W;
  C->tile_stages = stages;
  C->tile_blocks = (int)blocks;
  C->fused_smem = (int)smem;
  C->fused_ok = 1;
  return 1;
}

namespace {

// Launch arguments of a context's step (all but the destination array).
FusedArgs fused_args(const lbm_ctx *C) {
  FusedArgs P;
  const lbm_dev_params &D = C->dp;
  const int W = C->tile_w;
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
  P.RT2 = (float)(-2.0 * D.R * D.T);
  P.a2 = (float)(2.0 * D.a);
  P.r1 = (float)D.r1;
  P.r2 = (float)D.r2;
  P.pc0 = (float)(-2.0 * (D.thv - 1.0 / 3.0));
  P.pc1 = (float)(-2.0 * (D.thm - D.thv));
  P.pc2 = (float)(-2.0 * (D.thl - D.thm));
  P.A = (float)D.A;
  P.omA = (float)(1.0 - D.A);
  P.pre = (float)(-0.5 * D.kappa);
  P.halfA = (float)(0.5 * D.A);
  P.rho_max = (float)fmin(D.rho_max, 3.0e38);
  P.ghost_max = (float)fmin(D.ghost_max, 3.0e38);
  P.k = lbm_node::rate_consts(D.s);
  P.Gw = (float)D.Gw;
  {
    const long long n = (long long)C->nx * C->ny, nx = C->nx;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int k = 0; k < 9; ++k) P.eoff[k] = 4 * (k * n + ey[k] * nx + ex[k]);
  }
  P.coef = C->d_coef;
  P.fout = nullptr;
  P.flag = C->d_flag;
  return P;
}

// Launched with programmatic stream serialisation (the kernel orders its own
// global accesses after the previous grid with griddepcontrol.wait), so that
// back-to-back steps overlap one grid's tail with the next grid's launch and
// set-up; LBM_FUSED_PDL=0 turns it off.
cudaError_t launch_fused(lbm_ctx *C, const CUtensorMap &tm, const CUtensorMap &th, const FusedArgs &P,
                         unsigned long long *launches) {
  static const int pdl = [] {
    const char *e = getenv("LBM_FUSED_PDL");
    return e && atoi(e) == 0 ? 0 : 1;
  }();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C->tile_blocks);
  cfg.blockDim = dim3(NCONS);
  cfg.dynamicSmemBytes = (size_t)C->fused_smem;
  cfg.stream = C->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl;
  const FusedKernel kern = kernel_ptr(C->fused_unit, C->dp.wetting == LBM_WET_MARTYS_CHEN, C->dp.eos_kind);
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, tm, th, P);
  ++*launches;
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t lbm_fused_step(lbm_ctx *C, int src, unsigned long long *launches) {
  FusedArgs P = fused_args(C);
  P.fout = (float *)C->f[src ^ 1];
  return launch_fused(C, *(const CUtensorMap *)C->tmaps[2 * src], *(const CUtensorMap *)C->tmaps[2 * src + 1], P,
                      launches);
}

cudaError_t lbm_fused_step_between(lbm_ctx *C, const void *src, void *dst, unsigned long long *launches) {
  CUtensorMap tm, th;
  if (!encode(&tm, const_cast<void *>(src), C->nx, C->ny, C->tile_w) ||
      !encode(&th, const_cast<void *>(src), C->nx, C->ny, HB))
    return cudaErrorInvalidValue;
  FusedArgs P = fused_args(C);
  P.fout = (float *)dst;
  return launch_fused(C, tm, th, P, launches);
}
