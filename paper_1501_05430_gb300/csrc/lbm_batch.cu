// lbm_batch.cu -- many independent droplet instances (uneven nx, ny, EOS
// temperature, tau, wall angles) advanced together by one persistent launch.
//
// Work list: every instance is cut into "items", bands of whole fluid rows
// (full width, so the periodic x neighbours are in the CTA's own window).  The
// items of all instances form one list, ordered by instance and row.  A launch
// runs `steps` timesteps as the sequence (step, item) = (0, 0), (0, 1), ...,
// (1, 0), ...; every CTA of the persistent grid takes the next entry from a
// global counter, so the work balances itself and steps overlap across
// instances.  Before an item of step s the CTA waits until every item of the
// same instance has finished step s-1: a per-instance arrival counter,
// released with a fence + atomic add, acquired with a bounded spin on
// %globaltimer.  Entries are taken in order and every CTA is resident
// (cooperative launch), so the entries a wait depends on are always finished or
// in progress.  A wait that runs out sets a per-instance timeout bit and a
// batch abort word, and every CTA leaves at its next entry.  Instances never
// wait on each other.
//
// Rows are streamed through a ring of shared-memory slots by one-dimensional
// bulk copies (cp.async.bulk, 9 per row, one per plane) that one thread
// issues, completing on an mbarrier per slot; the ring's memory (S rows of the
// widest instance) is repacked for each item into as many rows of that
// instance's width as fit (at most 16), so narrow instances keep more rows in
// flight.  After acquiring an instance's barrier that thread orders the
// previous step's generic stores (of this and other CTAs) before its
// asynchronous-proxy reads with fence.proxy.async.
// Thread t < h = nx/2 owns columns t and t + h as one lane pair (every lane
// busy whatever the width; warps past h skip the row work): rho of both with
// packed adds, psi and psi^2 written to a window laid out in lane pairs, and
// the node arithmetic of lbm_node.cuh in its packed two-node form -- the same
// per-node operations as the single-domain fused kernel, so a batch instance
// and a lone context produce the same bits: rho, EOS, ghost rows (Eqs. 19-21),
// force (Eq. 9, Eq. 14), Eq. 17 tensor, MRT collision with the Eq. 6 forcing
// and Eq. 16 source, push streaming with half-way bounce-back.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "lbm_internal.h"
#include "lbm_node.cuh"

namespace {

using lbm_node::add2;
using lbm_node::collide_node2;
using lbm_node::eos_node;
using lbm_node::eos_node2;
using lbm_node::ghost_value;

// Threads per CTA NT (a template parameter): thread t < nx/2 owns columns t
// and t + nx/2 (one lane pair), so an instance is at most 2 NT wide.  The
// default shape runs every instance in 256-thread CTAs; the split shape runs
// the instances up to 256 wide in a launch of their own with 128-thread CTAs,
// where a 256-wide row keeps every thread busy (in a 256-thread CTA half the
// warps would wait at each row's barrier).
constexpr int kMaxNx = 512;      // widest instance
constexpr int kSlots = 4;        // window rows (ring)
constexpr int kMaxRing = 16;     // row slots (and mbarriers) of the copy ring at most

// Per-instance block: the node-function fields (same names as the fused
// kernel's) and the batch bookkeeping.
struct BInst {
  int kind, wetting, walls, nx, ny, n_iter;
  float b4, RT2, a2, r1, r2, pc0, pc1, pc2;
  float A, omA, pre, halfA, rho_max, ghost_max;
  lbm_node::RateK k;
  float Gw;
  const double *coef;
  int unit;    // all non-conserved rates are 1
  int items;   // items of this instance = barrier arrivals per step
  int first;   // index of its first item
  int pad;
  float *f[2];
  int *flag;   // the instance context's flags: [0] unstable, [1] timeout
};

struct BItem {
  int inst, y0, y1, pad;  // fluid rows [y0, y1)
};

struct BatchArgs {
  const BInst *inst;
  const BItem *items;
  int nitems;
  unsigned *bar;           // [ninst] arrivals in this launch, [ninst]: next entry (zeroed before it)
  unsigned *next;
  int *abort;              // [0]: a barrier wait ran out
  int *iflag;              // [ninst] bit 0 unstable, bit 1 timeout
  unsigned long long *work;  // [ninst] fluid-node updates computed (frozen instances add none)
  const int *cur;          // [ninst] array index holding the state at phase 0
  int steps, phase;        // steps in this launch; parity of its first step
  int nxs, stages;         // stage row stride (floats), ring depth
  unsigned long long wait_ns;
  int hold;                // testing aid: this instance's first item never arrives (-1: none)
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Test an mbarrier phase; a thread that finds it incomplete is suspended for
// up to ~0.5 ms (the suspend-time hint) or until the phase completes.
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

// Bounded wait on an mbarrier phase: false after limit ns without completion.
__device__ bool mbar_wait(unsigned bar, unsigned parity, unsigned long long limit) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (gtimer() - t0 > limit) return false;
  }
}

// One-dimensional bulk copy global -> shared, completion counted in bytes on an mbarrier.
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Bounded wait until *p >= target.  False if the batch aborted or the wait ran out.
__device__ bool wait_ge(const unsigned *p, unsigned target, const int *abort, unsigned long long limit) {
  if (ld_acquire(p) >= target) return true;
  const unsigned long long t0 = gtimer();
  for (;;) {
    __nanosleep(200);
    if (ld_acquire(p) >= target) return true;
    if (*(volatile const int *)abort) return false;
    if (gtimer() - t0 > limit) return false;
  }
}

// Shared memory of a CTA (dynamic part, 128-byte aligned base).
struct Smem {
  float *stage;              // S x 9 x nxs floats: rows loaded by bulk copies (K slots of 9 x nx per item)
  float2 *wpsi, *wsq;        // [kSlots][NT + 2]: psi and psi^2 in lane pairs (entry e = columns e, e + nx/2)
  float *wrho;               // [nxs + 2]: boundary-row densities, column c at c + 1 (periodic copies at 0, nx + 1)
  unsigned long long *bars;  // [kMaxRing]: one mbarrier per row slot
};

// Row loads of the CTA.  The ring is empty between items, so each item
// repacks the stage memory into K = min(kMaxRing, S nxs / nx) row slots
// (narrow instances keep more rows in flight); load k of the item goes to
// slot k % K.  Bit s of wph is the phase parity of the next completion of
// mbarrier s (every thread keeps the same copy).
struct Ring {
  unsigned issued, consumed;  // loads of the current item
  unsigned wph;
  int K;
  int islot, cslot;           // slots of the next load and of the next row to consume (issued, consumed mod K)
};

// One item of one step: stream virtual rows y0-1 .. y1 (halo and solid rows
// included), fill the window, collide rows y0 .. y1-1 into dst.  Rows come in
// by bulk copies that one thread issues (9 per row, one per plane) into a ring
// of S stages; a stage is read when its row arrives (rho) and again when the
// row is collided one iteration later, then refilled.
// Returns false if a wait on a row ran out (the CTA then aborts).
// NX: the instance width when fixed at compile time (0: read from P), so that
// every plane and lane-pair offset is an immediate.
template <bool UNIT, int NT, int KIND, int MCW, int NX = 0>
__device__ bool sweep(const BInst &P, const BItem &it, const float *__restrict__ src, float *__restrict__ dst,
                      const Smem &M, int nxs, int S, Ring &rg, unsigned long long wait_ns, bool &bad) {
  constexpr int kWP = NT + 2;  // paired window entries e = -1 .. nx/2 at index e + 1
  const int tid = threadIdx.x;
  const int nx = NX > 0 ? NX : P.nx, ny = P.ny;
  const size_t n = (size_t)nx * ny;
  const int R = it.y1 - it.y0 + 2;
  const bool geo = MCW < 0 ? P.wetting == LBM_WET_GEOMETRIC : MCW == 0;
  const unsigned row_bytes = (unsigned)nx * 4u;
  const int K = min(kMaxRing, S * nxs / nx);  // row slots of 9 x nx floats (plane stride nx)
  rg.issued = rg.consumed = 0u;
  rg.islot = rg.cslot = 0;
  rg.K = K;
  const int h = nx >> 1;  // lane-pair offset (nx is a multiple of 4)
  const int c0 = tid, c1 = tid + h;
  const bool act0 = tid < h, act1 = act0;  // c1 < nx exactly when c0 < h

  int jn = 0;  // next row to load (meaningful in thread 0 only)
  // a stage stays in use until its row is collided (read in the iteration the
  // row arrives and in the next one): rows consumed before the previous
  // iteration are released
  unsigned released = 0u, start_prev = 0u;
  auto issue = [&]() {
    // after the generic-proxy reads of the slots being refilled
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    while (jn < R && rg.issued - released < (unsigned)K) {
      const int v = it.y0 - 1 + jn;
      ++jn;
      if (v <= 0 || v >= ny - 1) continue;  // solid rows are not loaded
      const int s = rg.islot;
      if (++rg.islot == K) rg.islot = 0;
      const unsigned bar = smem_u32(&M.bars[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(9u * row_bytes)
                   : "memory");
      float *st = M.stage + (size_t)s * 9 * nx;
      const float *row = src + (size_t)v * nx;
#pragma unroll
      for (int a = 0; a < 9; ++a) bulk_g2s(smem_u32(st + a * nx), row + a * n, row_bytes, bar);
      ++rg.issued;
    }
  };
  if (tid == 0) issue();

  // (psi, psi^2) of column c into a window row pair: lane 0 of entry c and/or
  // lane 1 of entry c - h; columns nx-1 and 0 also fill the periodic
  // entries -1 and nx
  auto put1 = [&](float2 *ps, float2 *sq, int c, float p, float q) {
    if (c <= h) {
      ps[c + 1].x = p;
      sq[c + 1].x = q;
    }
    if (c >= h - 1) {
      ps[c - h + 1].y = p;
      sq[c - h + 1].y = q;
    }
  };
  auto put = [&](float2 *ps, float2 *sq, int c, float p, float q) {
    put1(ps, sq, c, p, q);
    if (c == nx - 1) put1(ps, sq, -1, p, q);
    if (c == 0) put1(ps, sq, nx, p, q);
  };
  auto putr = [&](int c, float r) {
    M.wrho[c + 1] = r;
    if (c == nx - 1) M.wrho[0] = r;
    if (c == 0) M.wrho[nx + 1] = r;
  };

  float2 rc = make_float2(0.0f, 0.0f), rp = rc, rp2 = rc;  // densities of rows v, v-1, v-2 (own columns)
  bool ok = true;
  int slot_prev = 0;  // stage of the row loaded in the previous iteration

  auto body = [&](int j) {
    const int v = it.y0 - 1 + j;
    const unsigned start = rg.consumed;
    int slot = slot_prev;
    float2 *pcur = M.wpsi + (size_t)(j & 3) * kWP, *qcur = M.wsq + (size_t)(j & 3) * kWP;
    const bool solid = v == 0 || v == ny - 1;
    if (!solid) {
      const int s = rg.cslot;
      if (++rg.cslot == K) rg.cslot = 0;
      slot = s;
      const unsigned ph = (rg.wph >> s) & 1u;
      if (!mbar_wait(smem_u32(&M.bars[s]), ph, wait_ns)) ok = false;
      rg.wph ^= 1u << s;
      ++rg.consumed;
      const float *st = M.stage + (size_t)s * 9 * nx;
      const bool brow = v == 1 || v == ny - 2;  // boundary row: the ghost rule reads its neighbours
      if (act0) {
        const float *q0 = st + c0, *q1 = st + c1;
        float2 fin[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) fin[a] = make_float2(q0[a * nx], q1[a * nx]);
        const float2 r = add2(add2(add2(add2(fin[0], fin[1]), add2(fin[2], fin[3])),
                                   add2(add2(fin[4], fin[5]), add2(fin[6], fin[7]))),
                              fin[8]);
        rc = r;
        float2 ps, ps2;
        eos_node2<KIND>(P, r, ps, ps2);
        // window entry c0 + 1 is the pair (c0, c1): one 64-bit store per
        // quantity; the pair reversed also fills entry 0 (columns nx-1 and
        // h-1, from the thread with c0 = h-1) and entry h+1 (columns h and 0,
        // from the thread with c0 = 0), as put() would
        pcur[c0 + 1] = ps;
        qcur[c0 + 1] = ps2;
        if (c0 == h - 1 || c0 == 0) {
          const int e = c0 == 0 ? h + 1 : 0;
          pcur[e] = make_float2(ps.y, ps.x);
          qcur[e] = make_float2(ps2.y, ps2.x);
        }
        if (brow) {
          putr(c0, r.x);
          putr(c1, r.y);
        }
        // unstable unless 0 < rho <= rho_max, tested on the bits (positive
        // floats order like their bit patterns; -0, negatives, +inf and NaN
        // land at or above rho_max's pattern after the decrement)
        const unsigned mx = __float_as_uint(P.rho_max);
        bad |= (__float_as_uint(r.x) - 1u >= mx) | (__float_as_uint(r.y) - 1u >= mx);
      }
      // bottom ghost row (Eqs. 19-21) once rows 1 and 2 are in: row 1's
      // densities in wrho (written last iteration), row 2's in registers
      if (geo && it.y0 == 1 && v == 2) {
        float2 *gp = M.wpsi + (size_t)((j - 2) & 3) * kWP, *gq = M.wsq + (size_t)((j - 2) & 3) * kWP;
        if (act0) {
          const float4 e = ghost_value<KIND>(P, M.wrho[c0], M.wrho[c0 + 1], M.wrho[c0 + 2], rc.x, c0, 0);
          put(gp, gq, c0, e.y, e.z);
        }
        if (act1) {
          const float4 e = ghost_value<KIND>(P, M.wrho[c1], M.wrho[c1 + 1], M.wrho[c1 + 2], rc.y, c1, 0);
          put(gp, gq, c1, e.y, e.z);
        }
      }
    } else if (!geo || v == ny - 1) {
      // Martys-Chen: solid rows carry psi = U = 0.  Geometric: the top ghost
      // row from rows ny-2 (wrho) and ny-3 (registers); the bottom one is filled at v == 2.
      if (act0) {
        float4 e = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (geo) e = ghost_value<KIND>(P, M.wrho[c0], M.wrho[c0 + 1], M.wrho[c0 + 2], rp2.x, c0, 1);
        put(pcur, qcur, c0, e.y, e.z);
      }
      if (act1) {
        float4 e = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (geo) e = ghost_value<KIND>(P, M.wrho[c1], M.wrho[c1 + 1], M.wrho[c1 + 2], rp2.y, c1, 1);
        put(pcur, qcur, c1, e.y, e.z);
      }
    }
    // window row j complete; row j's stage read (refillable); a row wait
    // that ran out in any thread ends the item in all of them
    ok = !__syncthreads_or(!ok);
    if (!ok) return;
    released = start_prev;  // every row before row j-1 is collided
    start_prev = start;
    if (tid == 0) issue();

    // ---- collide row v-1 (its populations are in the stage of the previous iteration) ----
    const int y = v - 1;
    if (act0 && j >= 1 && y >= it.y0 && y < it.y1) {
      const float2 *pm = M.wpsi + (size_t)((j - 2) & 3) * kWP, *qm = M.wsq + (size_t)((j - 2) & 3) * kWP;
      const float2 *p0 = M.wpsi + (size_t)((j - 1) & 3) * kWP, *q0 = M.wsq + (size_t)((j - 1) & 3) * kWP;
      const float2 *pp = pcur, *qp = qcur;
      const bool wall_dn = y == 1, wall_up = y == ny - 2;
      // warp-uniform plane pointers; each store adds one 32-bit element offset
      // (9 nx ny < 2^31 is checked at creation)
      const unsigned un = (unsigned)n;
      float *const o0 = dst, *const o1 = o0 + un, *const o2 = o1 + un, *const o3 = o2 + un, *const o4 = o3 + un;
      float *const o5 = o4 + un, *const o6 = o5 + un, *const o7 = o6 + un, *const o8 = o7 + un;
      const unsigned ry = (unsigned)y * nx, rym = ry - nx, ryp = ry + nx;
      auto push = [&](unsigned x, float f0, float f1, float f2, float f3, float f4, float f5, float f6, float f7,
                      float f8) {
        const unsigned xm = x == 0 ? nx - 1 : x - 1, xp = x == (unsigned)nx - 1 ? 0 : x + 1;
        o0[ry + x] = f0;
        o1[ry + xp] = f1;
        o3[ry + xm] = f3;
        if (wall_up) {
          o4[ry + x] = f2;
          o7[ry + x] = f5;
          o8[ry + x] = f6;
        } else {
          o2[ryp + x] = f2;
          o5[ryp + xp] = f5;
          o6[ryp + xm] = f6;
        }
        if (wall_dn) {
          o2[ry + x] = f4;
          o5[ry + x] = f7;
          o6[ry + x] = f8;
        } else {
          o4[rym + x] = f4;
          o7[rym + xm] = f7;
          o8[rym + xp] = f8;
        }
      };
      const int i = tid + 1;
      float2 pn[9], qn[9], fs[9];
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
      const float *sp = M.stage + (size_t)slot_prev * 9 * nx;
      const float *fa = sp + c0, *fb = sp + c1;
      float2 fcol[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) fcol[a] = make_float2(fa[a * nx], fb[a * nx]);
      collide_node2<UNIT, MCW>(P, fcol, pn, qn, rp, y, fs);
      push((unsigned)c0, fs[0].x, fs[1].x, fs[2].x, fs[3].x, fs[4].x, fs[5].x, fs[6].x, fs[7].x, fs[8].x);
      if (act1) push((unsigned)c1, fs[0].y, fs[1].y, fs[2].y, fs[3].y, fs[4].y, fs[5].y, fs[6].y, fs[7].y, fs[8].y);
    }
    rp2 = rp;
    rp = rc;
    slot_prev = slot;
  };
  for (int j = 0; j < R && ok; ++j) body(j);
  return ok;
}

// KIND, MCW: the EOS and wetting rule of every instance of the launch when
// they all share them (fixed at compile time: no branch in the per-node
// arithmetic), else -1 (read per instance)
template <int NT, int KIND, int MCW>
__global__ void __launch_bounds__(NT, 768 / NT) k_batch(BatchArgs A) {
  constexpr int kWP = NT + 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ BInst sP;
  __shared__ BItem s_it;
  __shared__ int s_go, s_skip, s_bad, s_step, s_idx, s_timeout;
  unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int S = A.stages, nxs = A.nxs;
  Smem M;
  M.stage = (float *)base;
  M.wpsi = (float2 *)(M.stage + (size_t)S * 9 * nxs);
  M.wsq = M.wpsi + kSlots * kWP;
  M.wrho = (float *)(M.wsq + kSlots * kWP);
  M.bars = (unsigned long long *)(M.wrho + ((nxs + 2 + 1) & ~1));
  const int tid = threadIdx.x;
  const unsigned total = (unsigned)A.steps * (unsigned)A.nitems;
  if (tid == 0) {
    s_timeout = 0;
    for (int s = 0; s < kMaxRing; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&M.bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  Ring rg{0u, 0u, 0u, 1, 0, 0};

  for (;;) {
    if (tid == 0) {
      int go = 0;
      const unsigned q = atomicAdd(A.next, 1u);
      if (q < total && !*(volatile int *)A.abort) {
        const int s = (int)(q / (unsigned)A.nitems), ii = (int)(q - (unsigned)s * (unsigned)A.nitems);
        const BItem it = A.items[ii];
        const BInst *gp = A.inst + it.inst;
        go = 1;
        // every item of the instance has finished step s-1 of this launch
        if (s > 0 && !wait_ge(A.bar + it.inst, (unsigned)(s * gp->items), A.abort, A.wait_ns)) {
          if (!*(volatile int *)A.abort) {
            atomicOr(A.iflag + it.inst, 2);
            atomicOr(gp->flag + 1, 1);
          }
          atomicExch(A.abort, 1);
          go = 0;
        }
        if (go) {
          // the rows about to be loaded by the bulk (asynchronous-proxy) copies
          // were written by generic stores of this and other CTAs before the
          // barrier just acquired
          asm volatile("fence.proxy.async.global;" ::: "memory");
          sP = *gp;
          s_it = it;
          s_step = s;
          s_idx = ii;
          // a blown-up instance is carried along (its barriers still count), not computed
          s_skip = *(volatile const int *)(A.iflag + it.inst) & 1;
          s_bad = 0;
        }
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const BItem it = s_it;
    const int par = A.cur[it.inst] ^ ((A.phase + s_step) & 1);
    bool bad = false;
    if (!s_skip) {
      bool ok;
      if (sP.unit)
        ok = sweep<true, NT, KIND, MCW>(sP, it, sP.f[par], sP.f[par ^ 1], M, nxs, S, rg, A.wait_ns, bad);
      else if (NT == 256 && KIND >= 0 && sP.nx == 2 * NT)
        // the widest instances, fixed at compile time in the specialised
        // kernels (every thread owns one lane pair)
        ok = sweep<false, NT, KIND, MCW, 2 * NT>(sP, it, sP.f[par], sP.f[par ^ 1], M, nxs, S, rg, A.wait_ns, bad);
      else
        ok = sweep<false, NT, KIND, MCW>(sP, it, sP.f[par], sP.f[par ^ 1], M, nxs, S, rg, A.wait_ns, bad);
      if (!ok) s_timeout = 1;
    }
    if (bad) s_bad = 1;
    if (tid == 0 && !s_skip)
      atomicAdd(A.work + it.inst, (unsigned long long)(it.y1 - it.y0) * (unsigned long long)sP.nx);
    __syncthreads();  // every store of the item issued; shared state free for the next entry
    if (s_timeout) {
      if (tid == 0) {
        atomicOr(A.iflag + it.inst, 2);
        atomicOr(sP.flag + 1, 1);
        atomicExch(A.abort, 1);
      }
      break;
    }
    if (tid == 0) {
      if (s_bad) {
        atomicOr(A.iflag + it.inst, 1);
        atomicOr(sP.flag, 1);
      }
      if (!(it.inst == A.hold && s_idx == sP.first)) {
        __threadfence();
        atomicAdd(A.bar + it.inst, 1u);
      }
    }
  }
  // no bulk copy may still be writing into this CTA's shared memory when it
  // exits (only possible after a timeout): wait for them, bounded
  if (tid == 0) {
    unsigned ph = rg.wph;
    for (unsigned k = rg.consumed; k < rg.issued; ++k) {
      const int s = (int)(k % (unsigned)rg.K);
      mbar_wait(smem_u32(&M.bars[s]), (ph >> s) & 1u, A.wait_ns);
      ph ^= 1u << s;
    }
  }
}

typedef void (*BatchKernel)(BatchArgs);
template <int NT>
BatchKernel pick_batch(int kind) {
  if (kind == LBM_EOS_CARNAHAN_STARLING) return k_batch<NT, LBM_EOS_CARNAHAN_STARLING, 0>;
  if (kind == LBM_EOS_PIECEWISE) return k_batch<NT, LBM_EOS_PIECEWISE, 0>;
  return k_batch<NT, -1, -1>;
}
// kind: the EOS every instance of the launch shares, all with geometric
// wetting; -1 otherwise (the generic kernel)
BatchKernel kernel_ptr(int nt, int kind) { return nt == 128 ? pick_batch<128>(kind) : pick_batch<256>(kind); }

size_t smem_bytes(int nxs, int stages, int nt) {
  return 128 + (size_t)stages * 9 * nxs * sizeof(float) + (size_t)2 * kSlots * (nt + 2) * sizeof(float2) +
         (size_t)((nxs + 2 + 1) & ~1) * sizeof(float) + (size_t)kMaxRing * 8;
}

int size_class(int nx) { return nx <= 128 ? 0 : nx <= 256 ? 1 : nx <= 384 ? 2 : 3; }

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct lbm_batch {
  int n;
  cudaStream_t stream;
  lbm_batch_config cfg;
  std::vector<lbm_ctx *> ctx;
  void *pool;                 // every instance's two distribution arrays
  size_t pool_bytes;
  std::vector<size_t> offset; // byte offset of each instance's state in the pool
  std::vector<BInst> hinst;
  // the launches of one chunk of steps: [0] 256-thread CTAs, [1] 128-thread
  // CTAs (split shape: the instances up to 256 wide); a part without items is
  // not launched
  struct Part {
    int nt;
    int kind;  // EOS kind shared by its instances, all geometric; -1: the generic kernel
    std::vector<BItem> items;
    BItem *d_items;
    size_t d_items_cap;
    int grid, nxs, smem, occ;
  } part[2];
  std::vector<int> hcur;      // array index of each instance's state at phase 0
  int phase;                  // steps since hcur was uploaded, mod 2
  BInst *d_inst;
  unsigned *d_bar;            // [n] arrival counters + [1] work counter
  int *d_abort;
  int *d_iflag;
  unsigned long long *d_work;  // [n] fluid-node updates computed per instance
  int *d_cur;
  int nsm;
  cudaGraphExec_t graph[2];   // per starting phase
  int graph_steps;
  unsigned long long graph_kernels;  // kernels one graph replay launches
  unsigned long long launches;
  long long steps;
  int status;
};

namespace {

#define BCK(x)                          \
  do {                                  \
    if ((x) != cudaSuccess) {           \
      cudaGetLastError();               \
      return LBM_ECUDA;                 \
    }                                   \
  } while (0)

void drop_graphs(lbm_batch *B) {
  for (int p = 0; p < 2; ++p)
    if (B->graph[p]) {
      cudaGraphExecDestroy(B->graph[p]);
      B->graph[p] = nullptr;
    }
  B->graph_steps = 0;
}

int resolve_config(const lbm_batch *B, const lbm_batch_config *in, lbm_batch_config *out) {
  lbm_batch_config c = *in;
  int nxmax = 0;
  for (int i = 0; i < B->n; ++i) nxmax = std::max(nxmax, B->ctx[i]->nx);
  if (c.threads == 0) c.threads = 256;
  if (c.threads != 256 && c.threads != 128) return LBM_EINVAL;
  if (nxmax > kMaxNx) return LBM_EUNSUPPORTED;
  if (c.stages == 0) c.stages = 4;
  if (c.stages < 3 || c.stages > 6) return LBM_EINVAL;
  for (int k = 0; k < 4; ++k) {
    if (c.band_rows[k] == 0) c.band_rows[k] = 32;
    if (c.band_rows[k] < 1) return LBM_EINVAL;
  }
  if (c.steps_per_launch == 0) c.steps_per_launch = 16;
  if (c.steps_per_launch < 1) return LBM_EINVAL;
  if (c.graph_launches < 0 || c.ctas_per_sm < 0) return LBM_EINVAL;
  if (c.wait_seconds == 0.0) c.wait_seconds = 2.0;
  if (!(c.wait_seconds > 0.0) || c.wait_seconds > 60.0) return LBM_EINVAL;
  if (c.hold_instance < -1 || c.hold_instance >= B->n) return LBM_EINVAL;
  *out = c;
  return LBM_OK;
}

// Items, CTA ranges, launch shape for B->cfg; uploads the tables.
int plan(lbm_batch *B) {
  const lbm_batch_config &c = B->cfg;
  int nxmax[2] = {0, 0};
  int kind[2] = {-2, -2};  // -2: no instance yet
  for (int s = 0; s < 2; ++s) {
    B->part[s].nt = s == 0 ? 256 : 128;
    B->part[s].items.clear();
    B->part[s].grid = B->part[s].nxs = B->part[s].smem = B->part[s].occ = 0;
  }
  for (int i = 0; i < B->n; ++i) {
    const lbm_ctx *C = B->ctx[i];
    const int s = c.threads == 128 && C->nx <= 256 ? 1 : 0;
    std::vector<BItem> &items = B->part[s].items;
    nxmax[s] = std::max(nxmax[s], C->nx);
    const int k = C->dp.wetting == LBM_WET_GEOMETRIC ? C->dp.eos_kind : -1;
    kind[s] = kind[s] == -2 || kind[s] == k ? k : -1;
    const int band = c.band_rows[size_class(C->nx)];
    B->hinst[i].first = (int)items.size();
    int cnt = 0;
    for (int y = 1; y < C->ny - 1; y += band) {
      items.push_back(BItem{i, y, std::min(y + band, C->ny - 1), 0});
      ++cnt;
    }
    B->hinst[i].items = cnt;
  }
  int dev = 0, optin = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  BCK(cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, dev));
  for (int s = 0; s < 2; ++s) {
    lbm_batch::Part &P = B->part[s];
    const int nitems = (int)P.items.size();
    if (nitems == 0) continue;
    if ((long long)nitems * c.steps_per_launch >= (1LL << 31)) return LBM_EUNSUPPORTED;
    P.nxs = (nxmax[s] + 3) & ~3;
    P.smem = (int)smem_bytes(P.nxs, c.stages, P.nt);
    P.kind = kind[s];
    const void *kern = (const void *)kernel_ptr(P.nt, P.kind);
    // the attribute is per kernel, not per batch: allow the device maximum so
    // that batches (and autotuner trials) with different rings coexist
    cudaFuncAttributes fa;
    BCK(cudaFuncGetAttributes(&fa, kern));
    const int dyn_max = optin - (int)fa.sharedSizeBytes;  // static + dynamic <= the opt-in limit
    if (P.smem > dyn_max) return LBM_EUNSUPPORTED;
    BCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
    int occ = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, P.nt, P.smem));
    if (occ < 1) return LBM_EUNSUPPORTED;
    // ctas_per_sm counts 256-thread CTAs; a 128-thread part may hold twice as many
    const int cap = c.ctas_per_sm * (256 / P.nt);
    if (c.ctas_per_sm > 0 && cap < occ) occ = cap;
    P.occ = occ;
    P.grid = std::min(B->nsm * occ, nitems);
    if ((size_t)nitems > P.d_items_cap) {
      cudaFree(P.d_items);
      P.d_items = nullptr;
      P.d_items_cap = 0;
      BCK(cudaMalloc(&P.d_items, (size_t)nitems * sizeof(BItem)));
      P.d_items_cap = nitems;
    }
    BCK(cudaMemcpyAsync(P.d_items, P.items.data(), (size_t)nitems * sizeof(BItem), cudaMemcpyHostToDevice,
                        B->stream));
  }
  BCK(cudaMemcpyAsync(B->d_inst, B->hinst.data(), (size_t)B->n * sizeof(BInst), cudaMemcpyHostToDevice, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  drop_graphs(B);
  return LBM_OK;
}

// The launches of `steps` steps starting at parity `phase`, one per part
// with items, in order on the stream (no synchronisation).  The parts hold
// different instances, so they need no ordering among themselves.
int launch(lbm_batch *B, int steps, int phase) {
  for (int s = 0; s < 2; ++s) {
    const lbm_batch::Part &P = B->part[s];
    if (P.items.empty()) continue;
    BatchArgs A;
    A.inst = B->d_inst;
    A.items = P.d_items;
    A.nitems = (int)P.items.size();
    A.bar = B->d_bar;
    A.next = B->d_bar + B->n;
    A.abort = B->d_abort;
    A.iflag = B->d_iflag;
    A.work = B->d_work;
    A.cur = B->d_cur;
    A.steps = steps;
    A.phase = phase;
    A.nxs = P.nxs;
    A.stages = B->cfg.stages;
    A.wait_ns = (unsigned long long)(B->cfg.wait_seconds * 1e9);
    A.hold = B->cfg.hold_instance;
    BCK(cudaMemsetAsync(B->d_bar, 0, (size_t)(B->n + 1) * sizeof(unsigned), B->stream));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(P.grid);
    lc.blockDim = dim3(P.nt);
    lc.dynamicSmemBytes = P.smem;
    lc.stream = B->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the barriers need it
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = steps > 1 ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&lc, kernel_ptr(P.nt, P.kind), A);
    BCK(e);
    ++B->launches;
  }
  return LBM_OK;
}

int sync_cur(lbm_batch *B) {
  bool same = true;
  for (int i = 0; i < B->n; ++i)
    if (B->ctx[i]->cur != (B->hcur[i] ^ B->phase)) same = false;
  if (same) return LBM_OK;
  for (int i = 0; i < B->n; ++i) B->hcur[i] = B->ctx[i]->cur;
  B->phase = 0;
  BCK(cudaMemcpyAsync(B->d_cur, B->hcur.data(), (size_t)B->n * sizeof(int), cudaMemcpyHostToDevice, B->stream));
  return LBM_OK;
}

int read_batch_flags(lbm_batch *B) {
  std::vector<int> fl(B->n);
  int ab = 0;
  BCK(cudaMemcpyAsync(fl.data(), B->d_iflag, (size_t)B->n * sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaMemcpyAsync(&ab, B->d_abort, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  for (int i = 0; i < B->n; ++i) {
    if (fl[i] & 2) B->ctx[i]->status = LBM_ETIMEOUT;
    else if (fl[i] & 1) B->ctx[i]->status = LBM_EUNSTABLE;
  }
  if (ab) B->status = LBM_ETIMEOUT;
  return B->status;
}

void fill_inst(BInst &I, const lbm_ctx *C, int *flag) {
  const lbm_dev_params &D = C->dp;
  memset(&I, 0, sizeof(I));
  I.kind = D.eos_kind;
  I.wetting = D.wetting;
  I.walls = 1;
  I.nx = C->nx;
  I.ny = C->ny;
  I.n_iter = D.n_iter;
  I.b4 = (float)(0.25 * D.b);
  I.RT2 = (float)(-2.0 * D.R * D.T);
  I.a2 = (float)(2.0 * D.a);
  I.r1 = (float)D.r1;
  I.r2 = (float)D.r2;
  I.pc0 = (float)(-2.0 * (D.thv - 1.0 / 3.0));
  I.pc1 = (float)(-2.0 * (D.thm - D.thv));
  I.pc2 = (float)(-2.0 * (D.thl - D.thm));
  I.A = (float)D.A;
  I.omA = (float)(1.0 - D.A);
  I.pre = (float)(-0.5 * D.kappa);
  I.halfA = (float)(0.5 * D.A);
  I.rho_max = (float)fmin(D.rho_max, 3.0e38);
  I.ghost_max = (float)fmin(D.ghost_max, 3.0e38);
  I.k = lbm_node::rate_consts(D.s);
  I.Gw = (float)D.Gw;
  I.coef = C->d_coef;
  I.unit = D.s[1] == 1.0 && D.s[2] == 1.0 && D.s[4] == 1.0 && D.s[7] == 1.0;
  I.f[0] = (float *)C->f[0];
  I.f[1] = (float *)C->f[1];
  I.flag = flag;
}

int run_steps(lbm_batch *B, int nsteps) {
  const int k = B->cfg.steps_per_launch;
  const int G = B->cfg.graph_launches;
  int done = 0;
  // whole graphs (an even number of steps each, so a replay ends on the phase it started from)
  if (G > 0 && B->stream && (long long)G * k % 2 == 0 && nsteps >= G * k) {
    const int p = B->phase;
    if (!B->graph[p]) {
      cudaGraph_t g = nullptr;
      BCK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
      int st = LBM_OK;
      const unsigned long long l0 = B->launches;
      for (int l = 0; l < G && st == LBM_OK; ++l) st = launch(B, k, p ^ (l * k & 1));
      cudaError_t e = cudaStreamEndCapture(B->stream, &g);
      B->graph_kernels = B->launches - l0;
      B->launches = l0;  // counted when replayed
      if (st != LBM_OK || e != cudaSuccess) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return LBM_ECUDA;
      }
      e = cudaGraphInstantiate(&B->graph[p], g, 0);
      cudaGraphDestroy(g);
      BCK(e);
      B->graph_steps = G * k;
    }
    while (nsteps - done >= B->graph_steps) {
      BCK(cudaGraphLaunch(B->graph[p], B->stream));
      B->launches += B->graph_kernels;
      done += B->graph_steps;
    }
  }
  while (done < nsteps) {
    const int m = std::min(k, nsteps - done);
    int st = launch(B, m, (B->phase + done) & 1);
    if (st) return st;
    done += m;
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_config_default(lbm_batch_config *c) {
  if (!c) return LBM_EINVAL;
  memset(c, 0, sizeof(*c));
  c->hold_instance = -1;
  return LBM_OK;
}

int lbm_batch_create(int n, const lbm_instance_desc *inst, const lbm_batch_config *cfg, void *stream,
                     lbm_batch **out) {
  if (!out || n < 1 || !inst) return LBM_EINVAL;
  *out = nullptr;
  lbm_batch *B = new (std::nothrow) lbm_batch();
  if (!B) return LBM_ENOMEM;
  B->n = n;
  B->stream = (cudaStream_t)stream;
  B->ctx.assign(n, nullptr);
  B->hinst.resize(n);
  B->hcur.assign(n, 0);
  // validate the geometry and size the pool
  size_t total = 0;
  B->offset.resize(n);
  for (int i = 0; i < n; ++i) {
    const lbm_instance_desc &d = inst[i];
    if (d.nx < 4 || d.ny < 5 || (d.nx % 4) != 0 || d.params.precision != 32) {
      delete B;
      return LBM_EINVAL;
    }
    B->offset[i] = total;
    total += (lbm_required_state_bytes(d.nx, d.ny, 32) + 255) & ~(size_t)255;
  }
  if (cudaMalloc(&B->pool, total) != cudaSuccess) {
    cudaGetLastError();
    delete B;
    return LBM_ENOMEM;
  }
  B->pool_bytes = total;
  std::vector<uint8_t> mask;
  int st = LBM_OK;
  for (int i = 0; i < n && st == LBM_OK; ++i) {
    const lbm_instance_desc &d = inst[i];
    mask.assign((size_t)d.nx * d.ny, 0);
    std::fill(mask.begin(), mask.begin() + d.nx, 1);
    std::fill(mask.end() - d.nx, mask.end(), 1);
    lbm_params p = d.params;
    p.kernel = LBM_KERNEL_REFERENCE;  // the instance's own step (if ever called alone) needs no fused plan
    st = lbm_create_with_buffer(d.nx, d.ny, &d.eos, d.T, d.tau, d.theta, mask.data(), &p, stream,
                                (char *)B->pool + B->offset[i], lbm_required_state_bytes(d.nx, d.ny, 32), &B->ctx[i]);
  }
  bool ok = st == LBM_OK && cudaMalloc(&B->d_inst, (size_t)n * sizeof(BInst)) == cudaSuccess &&
            cudaMalloc(&B->d_bar, (size_t)(n + 1) * sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&B->d_abort, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&B->d_iflag, (size_t)n * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&B->d_work, (size_t)n * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&B->d_cur, (size_t)n * sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_batch_destroy(B);
    return st != LBM_OK ? st : LBM_ENOMEM;
  }
  for (int i = 0; i < n; ++i) fill_inst(B->hinst[i], B->ctx[i], B->ctx[i]->d_flag);
  if (cudaMemsetAsync(B->d_abort, 0, sizeof(int), B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_iflag, 0, (size_t)n * sizeof(int), B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_work, 0, (size_t)n * sizeof(unsigned long long), B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_cur, 0, (size_t)n * sizeof(int), B->stream) != cudaSuccess) {
    cudaGetLastError();
    lbm_batch_destroy(B);
    return LBM_ECUDA;
  }
  lbm_batch_config c;
  lbm_batch_config_default(&c);
  if (cfg) c = *cfg;
  if ((st = resolve_config(B, &c, &B->cfg)) != LBM_OK || (st = plan(B)) != LBM_OK) {
    lbm_batch_destroy(B);
    return st;
  }
  *out = B;
  return LBM_OK;
}

int lbm_batch_size(const lbm_batch *B) { return B ? B->n : 0; }

lbm_ctx *lbm_batch_instance(lbm_batch *B, int i) {
  if (!B || i < 0 || i >= B->n) return nullptr;
  return B->ctx[i];
}

int lbm_batch_get_config(const lbm_batch *B, lbm_batch_config *cfg) {
  if (!B || !cfg) return LBM_EINVAL;
  *cfg = B->cfg;
  return LBM_OK;
}

int lbm_batch_set_config(lbm_batch *B, const lbm_batch_config *cfg) {
  if (!B || !cfg) return LBM_EINVAL;
  lbm_batch_config c;
  int st = resolve_config(B, cfg, &c);
  if (st) return st;
  const lbm_batch_config old = B->cfg;
  B->cfg = c;
  if ((st = plan(B)) != LBM_OK) {
    B->cfg = old;
    plan(B);
    return st;
  }
  return LBM_OK;
}

int lbm_batch_step(lbm_batch *B, int nsteps) {
  LbmRange nvtx_range("lbm_batch_step");
  if (!B || nsteps < 0) return LBM_EINVAL;
  if (B->status) return B->status;
  if (nsteps == 0) return LBM_OK;
  int st = sync_cur(B);
  if (st) return st;
  if ((st = run_steps(B, nsteps)) != LBM_OK) {
    B->status = st;
    return st;
  }
  B->phase = (B->phase + nsteps) & 1;
  B->steps += nsteps;
  for (int i = 0; i < B->n; ++i) {
    B->ctx[i]->cur ^= nsteps & 1;
    B->ctx[i]->steps += nsteps;
  }
  return read_batch_flags(B);
}

int lbm_batch_status(lbm_batch *B, int *inst_status) {
  if (!B) return LBM_EINVAL;
  int st = read_batch_flags(B);
  if (inst_status)
    for (int i = 0; i < B->n; ++i) inst_status[i] = B->ctx[i]->status;
  return st;
}

int lbm_batch_contact_angles(lbm_batch *B, int wall, double *theta, double *H, double *L, int *status) {
  if (!B || (wall != 0 && wall != 1) || !theta) return LBM_EINVAL;
  for (int i = 0; i < B->n; ++i) {
    double t = NAN, h = NAN, l = NAN;
    int st = lbm_contact_angle(B->ctx[i], wall, 0, B->ctx[i]->nx, &t, &h, &l);
    if (st == LBM_ECUDA) return st;
    theta[i] = t;
    if (H) H[i] = h;
    if (L) L[i] = l;
    if (status) status[i] = st;
  }
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch *B, int trial_steps, lbm_batch_config *best) {
  LbmRange nvtx_range("lbm_batch_autotune");
  if (!B || trial_steps < 2) return LBM_EINVAL;
  if (B->status) return B->status;
  trial_steps += trial_steps & 1;  // every trial ends on the parity it started from
  int st = sync_cur(B);
  if (st) return st;
  // the trials run on a copy of the state; the original is put back afterwards
  void *save = nullptr;
  if (cudaMalloc(&save, B->pool_bytes) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  std::vector<int> cur0(B->n);
  for (int i = 0; i < B->n; ++i) cur0[i] = B->ctx[i]->cur;
  const int phase0 = B->phase;
  std::vector<unsigned long long> work0(B->n);  // the trials' work is not the caller's
  cudaError_t e = cudaMemcpyAsync(work0.data(), B->d_work, (size_t)B->n * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(save, B->pool, B->pool_bytes, cudaMemcpyDeviceToDevice, B->stream);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  const lbm_batch_config start = B->cfg;
  lbm_batch_config cur = start;
  cur.graph_launches = 0;
  cur.hold_instance = -1;
  double best_ms = INFINITY;
  lbm_batch_config best_cfg = cur;
  auto trial = [&](const lbm_batch_config &c) -> int {
    lbm_batch_config r;
    if (resolve_config(B, &c, &r) != LBM_OK) return LBM_OK;  // not applicable to this batch
    B->cfg = r;
    int s = plan(B);
    if (s == LBM_EUNSUPPORTED) return LBM_OK;
    if (s) return s;
    s = run_steps(B, 2);  // warm-up
    if (s) return s;
    BCK(cudaEventRecord(t0, B->stream));
    s = run_steps(B, trial_steps);
    if (s) return s;
    BCK(cudaEventRecord(t1, B->stream));
    BCK(cudaEventSynchronize(t1));
    float ms = 0;
    BCK(cudaEventElapsedTime(&ms, t0, t1));
    int ab = 0;
    BCK(cudaMemcpy(&ab, B->d_abort, sizeof(int), cudaMemcpyDeviceToHost));
    if (ab) return LBM_ETIMEOUT;
    if (ms < best_ms) {
      best_ms = ms;
      best_cfg = r;
    }
    return LBM_OK;
  };
  if (e == cudaSuccess) {
    const int threads[2] = {128, 256};
    const int stages[3] = {3, 4, 5};
    const int bands[5] = {8, 16, 32, 64, 128};
    const int kk[3] = {1, 8, 32};
    // coordinate descent: threads x stages, then the band height per size class, then steps per launch
    for (int a = 0; a < 2 && st == LBM_OK; ++a)
      for (int b = 0; b < 3 && st == LBM_OK; ++b) {
        lbm_batch_config c = cur;
        c.threads = threads[a];
        c.stages = stages[b];
        st = trial(c);
      }
    cur = best_cfg;
    for (int cls = 0; cls < 4 && st == LBM_OK; ++cls) {
      bool present = false;
      for (int i = 0; i < B->n; ++i) present |= size_class(B->ctx[i]->nx) == cls;
      if (!present) continue;
      for (int b = 0; b < 5 && st == LBM_OK; ++b) {
        lbm_batch_config c = cur;
        c.band_rows[cls] = bands[b];
        st = trial(c);
      }
      cur = best_cfg;
    }
    for (int b = 0; b < 3 && st == LBM_OK; ++b) {
      lbm_batch_config c = cur;
      c.steps_per_launch = kk[b];
      st = trial(c);
    }
    cur = best_cfg;
  } else {
    cudaGetLastError();
    st = LBM_ECUDA;
  }
  // restore the state and install the winner (with the caller's graph and wait settings)
  if (st == LBM_OK) {
    cur.graph_launches = start.graph_launches;
    cur.wait_seconds = start.wait_seconds;
    cur.hold_instance = start.hold_instance;
    B->cfg = cur;
    st = plan(B);
  } else {
    B->cfg = start;
    plan(B);
  }
  if (cudaMemcpyAsync(B->pool, save, B->pool_bytes, cudaMemcpyDeviceToDevice, B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_iflag, 0, (size_t)B->n * sizeof(int), B->stream) != cudaSuccess ||
      cudaMemcpyAsync(B->d_work, work0.data(), (size_t)B->n * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                      B->stream) != cudaSuccess ||
      cudaStreamSynchronize(B->stream) != cudaSuccess) {
    cudaGetLastError();
    st = LBM_ECUDA;
  }
  for (int i = 0; i < B->n; ++i) {
    B->ctx[i]->cur = cur0[i];
    int z[2] = {0, 0};
    if (cudaMemcpy(B->ctx[i]->d_flag, z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) st = LBM_ECUDA;
    B->ctx[i]->status = 0;
  }
  B->phase = phase0 ^ 1;  // forces a re-upload of the per-instance array indices
  sync_cur(B);
  cudaFree(save);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (st == LBM_OK && best) *best = B->cfg;
  return st;
}

unsigned long long lbm_batch_launch_count(const lbm_batch *B) { return B ? B->launches : 0ULL; }

int lbm_batch_node_updates(lbm_batch *B, unsigned long long *updates) {
  if (!B || !updates) return LBM_EINVAL;
  BCK(cudaMemcpyAsync(updates, B->d_work, (size_t)B->n * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                      B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  return LBM_OK;
}

int lbm_batch_get_plan(const lbm_batch *B, int *grid, int *items, int *smem_bytes, int *ctas_per_sm) {
  if (!B) return LBM_EINVAL;
  const lbm_batch::Part &P0 = B->part[0], &P1 = B->part[1];
  if (grid) *grid = P0.grid + P1.grid;
  if (items) *items = (int)(P0.items.size() + P1.items.size());
  if (smem_bytes) *smem_bytes = std::max(P0.smem, P1.smem);
  if (ctas_per_sm) *ctas_per_sm = P0.items.empty() ? P1.occ : P0.occ;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  else cudaDeviceSynchronize();
  drop_graphs(B);
  for (lbm_ctx *C : B->ctx)
    if (C) lbm_destroy(C);
  cudaFree(B->pool);
  cudaFree(B->d_inst);
  for (int s = 0; s < 2; ++s) cudaFree(B->part[s].d_items);
  cudaFree(B->d_bar);
  cudaFree(B->d_abort);
  cudaFree(B->d_iflag);
  cudaFree(B->d_work);
  cudaFree(B->d_cur);
  cudaGetLastError();
  delete B;
}

}  // extern "C"
