// lbm_node.cuh -- per-node arithmetic of the FP32 step, shared by the
// single-domain fused kernel (lbm_fused.cu) and the batched kernel
// (lbm_batch.cu): EOS -> (rho, psi, psi^2) (Eqs. 10-11), ghost densities
// (Eqs. 19-21), and force + tensor + MRT collision (Eqs. 1-6, 9, 14-17).
//
// PT is the kernel's parameter block; it provides
//   kind, b4, RT2, a2, r1, r2, pc0, pc1, pc2   EOS constants (RT2 = -2RT, a2 = 2a)
//   omA, halfA, pre, Gw, wetting, walls, ny     force / Eq. 17 / Eq. 14
//   k (RateK)                                   relaxation constants, moments scaled by 1/N
//   n_iter, rho_max, ghost_max, nx, coef        ghost rule
#pragma once

#include "lbm_internal.h"

namespace lbm_node {

// Relaxation of Eq. 15 with the Eq. 6 forcing and the Eq. 16 source, folded
// into per-moment constants that already carry the 1/N_k of the inverse
// transform (N = 9, 36, 36, 6, 12, 6, 12, 4, 4):
//   r_k = m*_k / N_k = (1 - s_k)/N_k m_k + [s_k meq_k + (1 - s_k/2) S_k + C_k]/N_k
// with meq, S, C written out per moment (e, eps, q, nu); see collide_node2.
struct RateK {
  float e_m, e_v, e_0, e_F, e_Q;  // r_e   = e_m m_e + rho (e_v v^2 + e_0) + e_F vF + e_Q (Qxx + Qyy)
  float p_m, p_v, p_0, p_F;       // r_eps = p_m m_eps + rho (p_v v^2 + p_0) + p_F vF
  float q_m, q_j, q_F;            // r_qx  = q_m m_qx + q_j rho vx + q_F Fx (likewise y)
  float n_m, n_e, n_F2, n_F1, n_Q;  // r_pxx = n_m m_pxx + n_e (rho vx vx - rho vy vy) + n_F2 (vx Fx - vy Fy) + n_Q (Qxx - Qyy)
                                    // r_pxy = n_m m_pxy + n_e rho vx vy + n_F1 (vx Fy + vy Fx) + n_Q Qxy
};

// The constants from the rates s = (s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_nu, s_nu).
inline RateK rate_consts(const double *s) {
  const double se = s[1], sp = s[2], sq = s[4], sn = s[7];
  RateK k;
  // e: meq = rho (3 v^2 - 2), S = 6 vF, C = 1.5 s_e (Qxx + Qyy); N = 36
  k.e_m = (float)((1.0 - se) / 36.0);
  k.e_v = (float)(se / 12.0);
  k.e_0 = (float)(-se / 18.0);
  k.e_F = (float)((1.0 - 0.5 * se) / 6.0);
  k.e_Q = (float)(se / 24.0);
  // eps: meq = rho (1 - 3 v^2), S = -6 vF; N = 36
  k.p_m = (float)((1.0 - sp) / 36.0);
  k.p_v = (float)(-sp / 12.0);
  k.p_0 = (float)(sp / 36.0);
  k.p_F = (float)(-(1.0 - 0.5 * sp) / 6.0);
  // q: meq = -rho v, S = -F; N = 12
  k.q_m = (float)((1.0 - sq) / 12.0);
  k.q_j = (float)(-sq / 12.0);
  k.q_F = (float)(-(1.0 - 0.5 * sq) / 12.0);
  // nu: meq = rho (vx vx - vy vy), rho vx vy; S = 2 (vx Fx - vy Fy), vx Fy + vy Fx;
  // C = -s_nu (Qxx - Qyy), -s_nu Qxy; N = 4
  k.n_m = (float)((1.0 - sn) / 4.0);
  k.n_e = (float)(sn / 4.0);
  k.n_F2 = (float)((1.0 - 0.5 * sn) / 2.0);
  k.n_F1 = (float)((1.0 - 0.5 * sn) / 4.0);
  k.n_Q = (float)(-sn / 4.0);
  return k;
}

// sqrt for x >= 0 through the hardware reciprocal square root; exactly 0 at 0.
__device__ __forceinline__ float sqrt0(float x) { return x * rsqrtf(fmaxf(x, 1.17549435e-38f)); }

// -2U = 2 (rho/3 - p) of one node (Eq. 10 with G = -1, c = 1): Carnahan-Starling
//   p = rho R T (1 + e + e^2 - e^3)/(1 - e)^3 - a rho^2, e = b rho / 4,
//   -2U = rho (2/3 - 2 R T q + 2 a rho), q = (1 + e + e^2 - e^3)/(1 - e)^3,
// or Eq. 11 written branch-free:
//   p = rho th_v + (th_m - th_v)(rho - rho1)^+ + (th_l - th_m)(rho - rho2)^+.
// The same operations, lane by lane, as eos_node2 (identical bits).  KIND:
// the EOS when the caller fixes it at compile time (LBM_EOS_*), or -1 to
// read it from P.
template <int KIND = -1, class PT>
__device__ __forceinline__ float minus2u(const PT &P, float rho) {
  if (KIND < 0 ? P.kind == LBM_EOS_CARNAHAN_STARLING : KIND == LBM_EOS_CARNAHAN_STARLING) {
    const float e = P.b4 * rho;
    const float om = fmaf(e, -1.0f, 1.0f);
    const float num = fmaf(e, fmaf(e, om, 1.0f), 1.0f);
    const float q = __fdividef(num, (om * om) * om);
    return rho * fmaf(P.RT2, q, fmaf(P.a2, rho, 2.0f / 3.0f));
  }
  return fmaf(P.pc2, fmaxf(rho - P.r2, 0.0f), fmaf(P.pc1, fmaxf(rho - P.r1, 0.0f), P.pc0 * rho));
}

// Window entry of one node: rho, psi and psi^2 = -2U (psi = 0 where U >= 0).
// U itself is recovered as -psi^2/2 wherever the force needs it.
template <int KIND = -1, class PT>
__device__ __forceinline__ float4 eos_node(const PT &P, float rho) {
  const float psi2 = fmaxf(0.0f, minus2u<KIND>(P, rho));
  return make_float4(rho, sqrt0(psi2), psi2, 0.0f);
}

// Eqs. 19-21 ghost entry at column x from the boundary-row densities rl, ri1,
// rr (at x-1, x, x+1) and the second-row density ri2 (at x); gx indexes the
// wall coefficients; top: 0 or 1.
template <int KIND = -1, class PT>
__device__ __forceinline__ float4 ghost_value(const PT &P, float rl, float ri1, float rr, float ri2, int gx, int top) {
  float cc = (float)P.coef[top * P.nx + gx], cot = (float)P.coef[(2 + top) * P.nx + gx];
  float aa = rr - rl, g;
  if (P.n_iter <= 0) {
    g = fmaf(cot, fabsf(aa), ri2);
  } else {
    float d = 2.0f * (ri2 - ri1);
    g = ri2;
    for (int k = 0; k < P.n_iter; ++k) {
      g = fmaf(cc, sqrt0(fmaf(aa, aa, d * d)), ri2);
      d = ri2 - g;
    }
  }
  g = fminf(fmaxf(g, 0.0f), P.ghost_max);
  return g < P.rho_max ? eos_node<KIND>(P, g) : make_float4(g, 0.0f, 0.0f, 0.0f);  // psi = U = 0 at rho_max
}

// The same from window rows: r1 boundary row, r2 second row, column c stored
// at index c + 2.
template <int KIND = -1, class PT>
__device__ __forceinline__ float4 ghost_node(const PT &P, const float *r1, const float *r2, int c, int gx,
                                             int top) {
  return ghost_value<KIND>(P, r1[c + 1], r1[c + 2], r1[c + 3], r2[c + 2], gx, top);
}

// ---- two nodes at once ------------------------------------------------------
// The same node arithmetic on lane pairs (two nodes of one row that a thread
// owns) with the packed FP32 instructions of sm_100+: one instruction issues
// the operation for both nodes.  Each lane is an IEEE single-precision
// operation.

__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b lane by lane (packed subtraction, rounded like the scalar a - b)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
  return *reinterpret_cast<float2 *>(&r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// eos_node for two densities: the EOS arithmetic with packed instructions
// (the reciprocal, the maxima and the square roots lane by lane); each lane
// gets exactly eos_node's bits.  KIND as for minus2u.
template <int KIND = -1, class PT>
__device__ __forceinline__ void eos_node2(const PT &P, float2 rho, float2 &psi, float2 &psi2) {
  float2 m2u;
  if (KIND < 0 ? P.kind == LBM_EOS_CARNAHAN_STARLING : KIND == LBM_EOS_CARNAHAN_STARLING) {
    const float2 e = mul2(bc2(P.b4), rho);
    const float2 om = fma2(e, bc2(-1.0f), bc2(1.0f));
    const float2 num = fma2(e, fma2(e, om, bc2(1.0f)), bc2(1.0f));
    const float2 om3 = mul2(mul2(om, om), om);
    const float2 q = make_float2(__fdividef(num.x, om3.x), __fdividef(num.y, om3.y));
    m2u = mul2(rho, fma2(bc2(P.RT2), q, fma2(bc2(P.a2), rho, bc2(2.0f / 3.0f))));
  } else {
    const float2 d2 = sub2(rho, bc2(P.r2)), d1 = sub2(rho, bc2(P.r1));
    m2u = fma2(bc2(P.pc2), make_float2(fmaxf(d2.x, 0.0f), fmaxf(d2.y, 0.0f)),
               fma2(bc2(P.pc1), make_float2(fmaxf(d1.x, 0.0f), fmaxf(d1.y, 0.0f)), mul2(bc2(P.pc0), rho)));
  }
  psi2 = make_float2(fmaxf(0.0f, m2u.x), fmaxf(0.0f, m2u.y));
  psi = make_float2(sqrt0(psi2.x), sqrt0(psi2.y));
}

// Force (Eq. 9, + Eq. 14), Eq. 17 tensor, MRT collision with the Eq. 6
// forcing and the Eq. 16 source for two nodes.  f[9], psi[9], psi2[9]: lane
// pairs of the populations and of the neighbour values (psi, psi^2) at
// x+e_0..x+e_8; rho: the two densities; fs: f*.  UNIT: every non-conserved
// rate equals 1 (the relaxation matrix diag(0,1,...,1) of Sec. 3.1), so
// m* = m_eq + S/2 + C needs only rho and j from f.  MCW: the wetting rule
// when the caller fixes it at compile time (0 geometric, 1 Martys-Chen), or
// -1 to read it from P -- a fixed rule leaves no branch in the arithmetic.
template <bool UNIT, int MCW = -1, class PT>
__device__ __forceinline__ void collide_node2(const PT &P, const float2 *f, const float2 *psi, const float2 *psi2,
                                              float2 rho, int y, float2 *fs) {
  const float2 w1 = bc2(1.0f / 3.0f), w2 = bc2(1.0f / 12.0f);
  const float2 p0 = psi[0];
  // Eq. 9 (G = -1, U = -psi^2/2) and Eq. 17 (with its G/2 prefactor) weigh
  // the neighbours' psi and psi^2 with the same two coefficients, so both act
  // on one combined value per neighbour:
  //   g_a = (1 - A) psi_0 psi_a + (A/2) psi_a^2
  //   F   = sum_a w_a g_a e_a,    Q = (-kappa/2) sum_a w_a (g_a - g_0) e_a e_a
  const float2 c1 = mul2(bc2(P.omA), p0), hA = bc2(P.halfA);
  float2 g[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) g[k] = fma2(c1, psi[k], mul2(hA, psi2[k]));
  const float2 gd57 = sub2(g[5], g[7]), gd86 = sub2(g[8], g[6]);
  float2 Fx = fma2(w1, sub2(g[1], g[3]), mul2(w2, add2(gd57, gd86)));
  float2 Fy = fma2(w1, sub2(g[2], g[4]), mul2(w2, sub2(gd57, gd86)));
  const bool mc = MCW < 0 ? P.wetting == LBM_WET_MARTYS_CHEN : MCW == 1;
  if (mc && P.walls) {
    // Eq. 14 for flat solid rows: sum_a w_a S e_a = (0, -1/2) below, (0, 1/2) above
    const float ssy = (y == 1 ? -0.5f : 0.0f) + (y == P.ny - 2 ? 0.5f : 0.0f);
    Fy = fma2(mul2(bc2(-P.Gw), p0), bc2(ssy), Fy);
  }
  const float2 gs57 = add2(g[5], g[7]), gs68 = add2(g[6], g[8]);
  const float2 gq = mul2(w2, fma2(bc2(-4.0f), g[0], add2(gs57, gs68)));
  const float2 pre = bc2(P.pre), m2 = bc2(-2.0f);
  const float2 Qxx = mul2(pre, fma2(w1, fma2(m2, g[0], add2(g[1], g[3])), gq));
  const float2 Qyy = mul2(pre, fma2(w1, fma2(m2, g[0], add2(g[2], g[4])), gq));
  const float2 Qxy = mul2(pre, mul2(w2, sub2(gs57, gs68)));
  // moments (rho, e, eps, jx, qx, jy, qy, pxx, pxy); velocity with the
  // half-force shift
  const float2 s13 = sub2(f[1], f[3]), s24 = sub2(f[2], f[4]);
  const float2 d57 = sub2(f[5], f[7]), d86 = sub2(f[8], f[6]);
  const float2 jx = add2(s13, add2(d57, d86));
  const float2 jy = add2(s24, sub2(d57, d86));
  const float2 ir = make_float2(__fdividef(1.0f, rho.x), __fdividef(1.0f, rho.y));
  const float2 half = bc2(0.5f);
  const float2 vx = mul2(fma2(half, Fx, jx), ir), vy = mul2(fma2(half, Fy, jy), ir);
  const float2 rvx = mul2(rho, vx), rvy = mul2(rho, vy);
  const float2 v2 = fma2(vx, vx, mul2(vy, vy));
  const float2 vF = fma2(vx, Fx, mul2(vy, Fy));
  const float2 sQ = add2(Qxx, Qyy), dQ = sub2(Qxx, Qyy);
  // r_k = m*_k / N_k of the non-conserved moments (constants of RateK)
  float2 r1, r2, r4, r6, r7, r8;
  if (UNIT) {
    // every rate 1: m* = m_eq + S/2 + C
    r1 = fma2(rho, fma2(bc2(1.0f / 12.0f), v2, bc2(-1.0f / 18.0f)),
              fma2(bc2(1.0f / 12.0f), vF, mul2(bc2(1.0f / 24.0f), sQ)));
    r2 = fma2(rho, fma2(bc2(-1.0f / 12.0f), v2, bc2(1.0f / 36.0f)), mul2(bc2(-1.0f / 12.0f), vF));
    r4 = fma2(bc2(-1.0f / 12.0f), rvx, mul2(bc2(-1.0f / 24.0f), Fx));
    r6 = fma2(bc2(-1.0f / 12.0f), rvy, mul2(bc2(-1.0f / 24.0f), Fy));
    // (rvx vx - rvy vy + vx Fx - vy Fy - (Qxx - Qyy)) / 4
    r7 = mul2(bc2(0.25f), sub2(mul2(vx, add2(rvx, Fx)), fma2(vy, add2(rvy, Fy), dQ)));
    // (rvx vy + (vx Fy + vy Fx)/2 - Qxy) / 4
    r8 = fma2(bc2(0.25f), sub2(mul2(rvx, vy), Qxy), mul2(bc2(0.125f), fma2(vx, Fy, mul2(vy, Fx))));
  } else {
    const lbm_node::RateK &K = P.k;
    // non-conserved moments of f (rows e, eps, qx, qy, pxx, pxy of M)
    const float2 a13 = add2(f[1], f[3]), a24 = add2(f[2], f[4]);
    const float2 ax = add2(a13, a24), dg = add2(add2(f[5], f[6]), add2(f[7], f[8]));
    const float2 me = sub2(mul2(bc2(2.0f), dg), fma2(bc2(4.0f), f[0], ax));
    const float2 meps = fma2(bc2(4.0f), f[0], fma2(m2, ax, dg));
    const float2 mqx = fma2(m2, s13, add2(d57, d86));
    const float2 mqy = fma2(m2, s24, sub2(d57, d86));
    const float2 mpxx = sub2(a13, a24);
    const float2 mpxy = sub2(add2(f[5], f[7]), add2(f[6], f[8]));
    // relaxation (Eq. 15) with forcing S (Eq. 6) and source C (Eq. 16):
    // m* = m - s (m - m_eq) + (1 - s/2) S + C, divided by N
    r1 = fma2(bc2(K.e_m), me, fma2(rho, fma2(bc2(K.e_v), v2, bc2(K.e_0)),
                                   fma2(bc2(K.e_F), vF, mul2(bc2(K.e_Q), sQ))));
    r2 = fma2(bc2(K.p_m), meps, fma2(rho, fma2(bc2(K.p_v), v2, bc2(K.p_0)), mul2(bc2(K.p_F), vF)));
    r4 = fma2(bc2(K.q_m), mqx, fma2(bc2(K.q_j), rvx, mul2(bc2(K.q_F), Fx)));
    r6 = fma2(bc2(K.q_m), mqy, fma2(bc2(K.q_j), rvy, mul2(bc2(K.q_F), Fy)));
    // n_e (rvx vx - rvy vy) + n_F2 (vx Fx - vy Fy) = vx (n_e rvx + n_F2 Fx) - vy (n_e rvy + n_F2 Fy)
    const float2 ax7 = fma2(bc2(K.n_e), rvx, mul2(bc2(K.n_F2), Fx));
    const float2 ay7 = fma2(bc2(K.n_e), rvy, mul2(bc2(K.n_F2), Fy));
    r7 = fma2(bc2(K.n_m), mpxx, fma2(vx, ax7, sub2(mul2(bc2(K.n_Q), dQ), mul2(vy, ay7))));
    r8 = fma2(bc2(K.n_m), mpxy, fma2(mul2(bc2(K.n_e), rvx), vy,
                                     fma2(bc2(K.n_F1), fma2(vx, Fy, mul2(vy, Fx)), mul2(bc2(K.n_Q), Qxy))));
  }
  // back to populations: f* = M^T diag(1/N) m*.  rho/9 is rounded through one
  // correction step: a plain product with a rounded 1/9 biases the mass.
  const float2 c9 = bc2(1.0f / 9.0f);
  float2 r0 = mul2(rho, c9);
  r0 = fma2(fma2(bc2(-9.0f), r0, rho), c9, r0);
  const float2 i6 = bc2(1.0f / 6.0f);
  const float2 r3 = mul2(add2(jx, Fx), i6), r5 = mul2(add2(jy, Fy), i6);
  fs[0] = fma2(bc2(4.0f), sub2(r2, r1), r0);
  const float2 Aax = fma2(m2, r2, sub2(r0, r1));
  const float2 Bdg = fma2(bc2(2.0f), r1, add2(r0, r2));
  const float2 X1 = fma2(m2, r4, r3), Y1 = fma2(m2, r6, r5);
  fs[1] = add2(add2(Aax, X1), r7);
  fs[3] = add2(sub2(Aax, X1), r7);
  fs[2] = sub2(add2(Aax, Y1), r7);
  fs[4] = sub2(sub2(Aax, Y1), r7);
  const float2 X2 = add2(r3, r4), Y2 = add2(r5, r6);
  fs[5] = add2(add2(Bdg, X2), add2(Y2, r8));
  fs[6] = add2(sub2(Bdg, X2), sub2(Y2, r8));
  fs[7] = sub2(sub2(Bdg, X2), sub2(Y2, r8));
  fs[8] = sub2(add2(Bdg, X2), add2(Y2, r8));
}

}  // namespace lbm_node
