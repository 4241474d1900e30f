/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle for one timestep of the
 * single-component EOS-based pseudo-potential D2Q9 lattice Boltzmann method
 * with the geometric contact-angle wall rule of Hu, Li & Uddin,
 * "Contact Angle Adjustment in Equation of States Based Pseudo-Potential
 * Model" (arXiv:1501.05430), and with the Martys-Chen fluid-solid force
 * (Eq. 14) as the compared wetting variant.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference arm of bench.py may load it.  It shares no code, header, table or
 * constant with the CUDA path; the product never links it.
 *
 * Evaluation order.  Every floating-point expression below is written out in
 * one fixed ("canonical") order: sums run left to right in the listed index
 * order, integer matrix coefficients are applied as multiplications, and the
 * file must be compiled without FMA contraction (-ffp-contract=off) so that an
 * FP64 GPU build that follows the same order can be compared bit for bit.
 *
 * Pins.  Every function here is checked in tests/test_oracle_*.py against
 * something other than itself (printed Table 1 values, closed forms, textbook
 * special cases, invariants, brute force); see the header of each function.
 *
 * Layout: distribution functions are stored as f[a][y][x] (a = 0..8, row-major
 * nodes, x fastest).  Rows y = 0 and y = ny-1 are solid when the matching wall
 * flag is set; x is always periodic; y is periodic when there is no wall.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* D2Q9 lattice (Eq. 1): e_0 = (0,0), e_1..4 axis, e_5..8 diagonals.       */
/* ---------------------------------------------------------------------- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* Interaction weights w(|e|^2): w(1) = 1/3, w(2) = 1/12 (Sec. 2, after Eq. 7). */
static double orc_w(int a) { return a == 0 ? 0.0 : (a <= 4 ? 1.0 / 3.0 : 1.0 / 12.0); }

/* Orthogonal D2Q9 moment matrix M in the order (rho, e, eps, jx, qx, jy, qy,
 * pxx, pxy) that Eq. 4 lists its equilibria in.  Row norms N_k = sum_a M_ka^2
 * give M^-1 = M^T diag(1/N). */
static const double MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
static const double MNORM[9] = {9, 36, 36, 6, 12, 6, 12, 4, 4};

/* G: interaction strength of Eqs. 7-10.  Only G*psi^2 is physical; G = -1
 * makes psi^2 = 2(rho/3 - p) positive on the two-phase range. */
#define ORC_G (-1.0)

/* ---------------------------------------------------------------------- */
/* Equations of state                                                      */
/* ---------------------------------------------------------------------- */
enum { ORC_EOS_CS = 0, ORC_EOS_PIECEWISE = 1 };

/* eos[] = {a, b, R, theta_v, theta_m, theta_l, rho1, rho2} */

/* Carnahan-Starling: p = rho R T (1+eta+eta^2-eta^3)/(1-eta)^3 - a rho^2,
 * eta = b rho / 4.  Pinned by the literature critical point
 * (T_c = 0.3773 a/(bR), eta_c = 0.1304) and by a symbolic solve of
 * dp/drho = d2p/drho2 = 0 in tests/test_oracle_eos.py. */
static double orc_p_cs(const double *eos, double T, double rho) {
  double a = eos[0], b = eos[1], R = eos[2];
  double eta = (b * rho) * 0.25;
  double num = ((1.0 + eta) + eta * eta) - (eta * eta) * eta;
  double den = ((1.0 - eta) * (1.0 - eta)) * (1.0 - eta);
  return (((rho * R) * T) * num) / den - (a * rho) * rho;
}

/* Eq. 11: the three-branch self-tuning EOS.  At a breakpoint the lower branch
 * is taken; the branches agree there. */
static double orc_p_pw(const double *eos, double rho) {
  double thv = eos[3], thm = eos[4], thl = eos[5], r1 = eos[6], r2 = eos[7];
  if (rho <= r1) return rho * thv;
  if (rho <= r2) return r1 * thv + (rho - r1) * thm;
  return (r1 * thv + (r2 - r1) * thm) + (rho - r2) * thl;
}

double orc_pressure(int kind, const double *eos, double T, double rho) {
  return kind == ORC_EOS_CS ? orc_p_cs(eos, T, rho) : orc_p_pw(eos, rho);
}

/* Eq. 10 with c = 1 and G = -1: U = p - c_s^2 rho (c_s^2 = 1/3) and
 * psi = sqrt(2 U / G) = sqrt(max(0, -2U)). */
void orc_psi_U(int kind, const double *eos, double T, double rho, double *psi, double *U) {
  double p = orc_pressure(kind, eos, T, rho);
  double u = p - rho / 3.0;
  *U = u;
  *psi = sqrt(fmax(0.0, -2.0 * u));
}

/* CS critical point.  With K(eta) = eta (1+eta+eta^2-eta^3)/(1-eta)^3 the EOS
 * is p = (4RT/b) K(eta) - (16a/b^2) eta^2, so dp/drho = RT K'(eta) - (8a/b) eta
 * and d2p/drho2 = (b/4)(RT K''(eta) - 8a/b).  Both vanishing gives
 * eta K''(eta) = K'(eta), which with
 *   K'(eta)  = (1+4eta+4eta^2-4eta^3+eta^4)/(1-eta)^4,
 *   K''(eta) = (8+20eta-4eta^2)/(1-eta)^5
 * reduces to eta^5 - 5eta^4 + 4eta^3 + 20eta^2 + 5eta - 1 = 0 (a root near
 * 0.1304, independent of a, b, R); then T_c = 8a / (b R K''(eta_c)) and
 * rho_c = 4 eta_c / b.  Returns 0 on success. */
static double orc_cs_Kp(double eta) {
  double om = 1.0 - eta;
  return (1.0 + 4.0 * eta + 4.0 * eta * eta - 4.0 * eta * eta * eta + eta * eta * eta * eta) /
         (om * om * om * om);
}
static double orc_cs_Kpp(double eta) {
  double om = 1.0 - eta;
  return (8.0 + 20.0 * eta - 4.0 * eta * eta) / (om * om * om * om * om);
}
int orc_cs_critical(const double *eos, double *Tc, double *rhoc) {
  double lo = 0.05, hi = 0.3;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double g = ((((mid - 5.0) * mid + 4.0) * mid + 20.0) * mid + 5.0) * mid - 1.0;
    if (g > 0.0) hi = mid; else lo = mid;
  }
  double etac = 0.5 * (lo + hi);
  *Tc = 8.0 * eos[0] / (eos[1] * eos[2] * orc_cs_Kpp(etac));
  *rhoc = 4.0 * etac / eos[1];
  return 0;
}

/* dp/drho for CS (from K' above). */
static double orc_dp_cs(const double *eos, double T, double rho) {
  double eta = eos[1] * rho * 0.25;
  return eos[2] * T * orc_cs_Kp(eta) - 8.0 * eos[0] / eos[1] * eta;
}

/* CS chemical potential up to a constant:
 * mu = RT [ln eta + (8eta - 9eta^2 + 3eta^3)/(1-eta)^3] - 2 a rho,
 * i.e. the integral of (1/rho) dp/drho.  Differentiating the bracket gives
 * K'(eta)/eta, which is what makes this the Maxwell (equal-area) potential. */
static double orc_mu_cs(const double *eos, double T, double rho) {
  double eta = eos[1] * rho * 0.25, om = 1.0 - eta;
  return eos[2] * T * (log(eta) + (8.0 * eta - 9.0 * eta * eta + 3.0 * eta * eta * eta) / (om * om * om)) -
         2.0 * eos[0] * rho;
}

/* Root of p(rho) = ps on [lo, hi] where p is increasing; plain bisection. */
static double orc_bisect_p(const double *eos, double T, double ps, double lo, double hi) {
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_p_cs(eos, T, mid) > ps) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* Maxwell coexistence densities for CS at T < T_c: p(rho_v) = p(rho_l) and
 * mu(rho_v) = mu(rho_l).  Bisection on the saturation pressure between the
 * spinodal pressures.  Pinned against an independent scipy equal-area solve. */
int orc_cs_coexistence(const double *eos, double T, double *rho_v, double *rho_l) {
  double Tc, rc;
  orc_cs_critical(eos, &Tc, &rc);
  if (!(T > 0.0 && T < Tc)) return -1;
  double rmax = 4.0 / eos[1];
  /* spinodals: dp/drho = 0 on each side of rho_c */
  double lo = 1e-12 * rmax, hi = rc;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_dp_cs(eos, T, mid) > 0.0) lo = mid; else hi = mid;
  }
  double rsv = 0.5 * (lo + hi);
  lo = rc; hi = rmax * (1.0 - 1e-12);
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_dp_cs(eos, T, mid) < 0.0) lo = mid; else hi = mid;
  }
  double rsl = 0.5 * (lo + hi);
  double plo = orc_p_cs(eos, T, rsl), phi = orc_p_cs(eos, T, rsv);
  if (plo < 0.0) plo = 0.0;
  double rv = 0, rl = 0;
  for (int it = 0; it < 200; ++it) {
    double ps = 0.5 * (plo + phi);
    rv = orc_bisect_p(eos, T, ps, 1e-300, rsv);
    rl = orc_bisect_p(eos, T, ps, rsl, rmax * (1.0 - 1e-15));
    double dmu = orc_mu_cs(eos, T, rl) - orc_mu_cs(eos, T, rv);
    /* mu_l - mu_v = integral of dp/rho around the loop; it falls as p_s rises */
    if (dmu > 0.0) plo = ps; else phi = ps;
  }
  *rho_v = rv;
  *rho_l = rl;
  return 0;
}

/* Eqs. 12-13: breakpoints rho1, rho2 of Eq. 11 from (rho_v, rho_l) and the
 * three slopes.  Eq. 12 is linear and gives rho2 as a function of rho1; Eq. 13
 * is then solved for rho1 by bisection.  Pinned by Table 1. */
static double orc_pw_r2(double r1, double rv, double rl, double tv, double tm, double tl) {
  return (r1 * (tv - tm) - rv * tv + rl * tl) / (tl - tm);
}
static double orc_pw_chem(double r1, double r2, double rv, double rl, double tv, double tm, double tl) {
  return log(r1 / rv) * tv + log(r2 / r1) * tm + log(rl / r2) * tl;
}
int orc_piecewise_breakpoints(double rv, double rl, double tv, double tm, double tl, double *rho1,
                              double *rho2) {
  /* scan for a sign change of Eq. 13 along the feasible rho1 range */
  int N = 20000;
  double prev_r1 = 0, prev_g = 0;
  int found = 0;
  for (int i = 1; i < N; ++i) {
    double r1 = rv + (rl - rv) * (double)i / (double)N;
    double r2 = orc_pw_r2(r1, rv, rl, tv, tm, tl);
    if (!(r2 > r1 && r2 < rl)) { prev_g = 0; prev_r1 = 0; continue; }
    double g = orc_pw_chem(r1, r2, rv, rl, tv, tm, tl);
    if (prev_r1 > 0 && ((g > 0) != (prev_g > 0))) {
      double lo = prev_r1, hi = r1, glo = prev_g;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double gm = orc_pw_chem(mid, orc_pw_r2(mid, rv, rl, tv, tm, tl), rv, rl, tv, tm, tl);
        if ((gm > 0) == (glo > 0)) { lo = mid; glo = gm; } else hi = mid;
      }
      *rho1 = 0.5 * (lo + hi);
      *rho2 = orc_pw_r2(*rho1, rv, rl, tv, tm, tl);
      found = 1;
      break;
    }
    prev_r1 = r1;
    prev_g = g;
  }
  return found ? 0 : -1;
}

/* Inverse of the above: (rho_v, rho_l) from the breakpoints, i.e. the
 * coexistence densities that Eqs. 12-13 tie to a given Eq. 11 EOS.  Eq. 12
 * gives rho_l as a linear function of rho_v; Eq. 13 is bisected in rho_v. */
static double orc_pw_rl(double rv, double r1, double r2, double tv, double tm, double tl) {
  return r2 - ((r1 - rv) * tv + (r2 - r1) * tm) / tl;
}
int orc_piecewise_coexistence(const double *eos, double *rho_v, double *rho_l) {
  double tv = eos[3], tm = eos[4], tl = eos[5], r1 = eos[6], r2 = eos[7];
  double lo = r1 * 1e-9, hi = r1 * (1.0 - 1e-15);
  double glo = orc_pw_chem(r1, r2, lo, orc_pw_rl(lo, r1, r2, tv, tm, tl), tv, tm, tl);
  double ghi = orc_pw_chem(r1, r2, hi, orc_pw_rl(hi, r1, r2, tv, tm, tl), tv, tm, tl);
  if (!((glo > 0) != (ghi > 0))) return -1;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    double gm = orc_pw_chem(r1, r2, mid, orc_pw_rl(mid, r1, r2, tv, tm, tl), tv, tm, tl);
    if ((gm > 0) == (glo > 0)) { lo = mid; glo = gm; } else hi = mid;
  }
  *rho_v = 0.5 * (lo + hi);
  *rho_l = orc_pw_rl(*rho_v, r1, r2, tv, tm, tl);
  return 0;
}

int orc_coexistence(int kind, const double *eos, double T, double *rho_v, double *rho_l) {
  return kind == ORC_EOS_CS ? orc_cs_coexistence(eos, T, rho_v, rho_l)
                            : orc_piecewise_coexistence(eos, rho_v, rho_l);
}

/* Upper density bound of the EOS for the pseudo-potential: the smallest
 * rho > rho_l with U(rho) = 0 (psi^2 >= 0 below it), or DBL_MAX if U stays
 * negative.  Used to clamp ghost densities and to flag instability. */
double orc_rho_max(int kind, const double *eos, double T, double rho_l) {
  if (kind == ORC_EOS_CS) {
    double lo = rho_l, hi = 4.0 / eos[1] * (1.0 - 1e-12);
    double ulo = orc_p_cs(eos, T, lo) - lo / 3.0;
    if (ulo >= 0.0) return rho_l;
    for (int it = 0; it < 300; ++it) {
      double mid = 0.5 * (lo + hi);
      if (orc_p_cs(eos, T, mid) - mid / 3.0 < 0.0) lo = mid; else hi = mid;
    }
    return lo;
  }
  double tl = eos[5], r2 = eos[7];
  double U2 = orc_p_pw(eos, r2) - r2 / 3.0;
  double slope = tl - 1.0 / 3.0;
  if (slope <= 0.0) return DBL_MAX;
  double root = r2 - U2 / slope;
  return root > rho_l ? root : DBL_MAX;
}

/* ---------------------------------------------------------------------- */
/* Geometric ghost density (Eqs. 19-21)                                    */
/* ---------------------------------------------------------------------- */
/* rho_{i,0} from the boundary-row neighbours rho_{i-1,1}, rho_{i+1,1}, the
 * boundary node rho_{i,1} and the second row rho_{i,2}.
 *   n_iter == 0: Eq. 19, rho_{i,0} = rho_{i,2} + tan(pi/2-theta)|a|, with the
 *                coefficient cot = tan(pi/2-theta) passed in.
 *   n_iter >= 1: Eq. 21, n_iter evaluations of the right-hand side of Eq. 20,
 *                starting from (rho_{i,2}-rho_{i,0}) ~ 2(rho_{i,2}-rho_{i,1})
 *                and substituting each new rho_{i,0} back; c = sin(pi/2-theta).
 * Eq. 20 is read with a square root over the bracket (the extracted text lost
 * it): only then is the equation dimensionally consistent, and only then is
 * its fixed point exactly Eq. 19 (d^2 sin^2 = cos^2 a^2).
 * The result is clamped to [0, rho_max].
 * Pins: theta = 90 deg gives rho_{i,2}; c -> -c mirrors the correction; many
 * iterations converge to Eq. 19; uniform rows give rho_{i,2}. */
double orc_ghost(double r_im1_1, double r_ip1_1, double r_i1, double r_i2, double c, double cot,
                 int n_iter, double rho_max) {
  double a = r_ip1_1 - r_im1_1;
  double g;
  if (n_iter <= 0) {
    g = r_i2 + cot * fabs(a);
  } else {
    double d = 2.0 * (r_i2 - r_i1);
    g = r_i2;
    for (int k = 0; k < n_iter; ++k) {
      double s = a * a + d * d;
      g = r_i2 + c * sqrt(s);
      d = r_i2 - g;
    }
  }
  return fmin(fmax(g, 0.0), rho_max);
}

/* ---------------------------------------------------------------------- */
/* Node collision: Eqs. 4, 6, 15 (with the Eq. 16 source)                 */
/* ---------------------------------------------------------------------- */
/* f[9] in, fs[9] out.  rho is the node density (already summed), F the total
 * force, Qxx/Qyy/Qxy the Eq. 17 tensor, s[9] the relaxation rates
 * (s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_nu, s_nu) of Eq. 2.
 * The velocity in Eqs. 4 and 6 is v = (j + F/2)/rho.
 * Eq. 6's last entry is read as v_x F_y + v_y F_x (the pxy moment of the Guo
 * forcing term); the printed v_x F_x + v_y F_y is not symmetric in x<->y.
 * Eq. 16's entry for pxx is read as -s_nu (Qxx - Qyy), the same coefficient as
 * the pxy entry (both are components of one traceless tensor).
 * Pins: with all rates equal this must equal the textbook BGK collision with
 * Guo forcing; the rest state is a fixed point; mass is conserved and the
 * momentum change equals F. */
void orc_collide(const double *f, double rho, double Fx, double Fy, double Qxx, double Qyy, double Qxy,
                 const double *s, double *fs) {
  double m[9];
  for (int k = 0; k < 9; ++k) {
    double acc = 0.0;
    for (int a = 0; a < 9; ++a)
      if (MM[k][a] != 0.0) acc = acc + MM[k][a] * f[a];
    m[k] = acc;
  }
  double vx = (m[3] + 0.5 * Fx) / rho;
  double vy = (m[5] + 0.5 * Fy) / rho;
  double v2 = vx * vx + vy * vy;
  double meq[9];
  meq[0] = rho;
  meq[1] = rho * (-2.0 + 3.0 * v2);
  meq[2] = rho * (1.0 - 3.0 * v2);
  meq[3] = rho * vx;
  meq[4] = -(rho * vx);
  meq[5] = rho * vy;
  meq[6] = -(rho * vy);
  meq[7] = rho * (vx * vx - vy * vy);
  meq[8] = rho * (vx * vy);
  double vF = vx * Fx + vy * Fy;
  double S[9];
  S[0] = 0.0;
  S[1] = 6.0 * vF;
  S[2] = -(6.0 * vF);
  S[3] = Fx;
  S[4] = -Fx;
  S[5] = Fy;
  S[6] = -Fy;
  S[7] = 2.0 * (vx * Fx - vy * Fy);
  S[8] = vx * Fy + vy * Fx;
  double C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  C[1] = (1.5 * s[1]) * (Qxx + Qyy);
  C[7] = -(s[7] * (Qxx - Qyy));
  C[8] = -(s[8] * Qxy);
  double r[9];
  for (int k = 0; k < 9; ++k) {
    double ms = ((m[k] - s[k] * (m[k] - meq[k])) + (1.0 - 0.5 * s[k]) * S[k]) + C[k];
    r[k] = ms / MNORM[k];
  }
  for (int a = 0; a < 9; ++a) {
    double acc = 0.0;
    for (int k = 0; k < 9; ++k)
      if (MM[k][a] != 0.0) acc = acc + MM[k][a] * r[k];
    fs[a] = acc;
  }
}

/* Equilibrium distribution f_eq = M^-1 m_eq(rho, v) (Eq. 4).  Pinned against
 * the textbook second-order D2Q9 equilibrium. */
void orc_feq(double rho, double vx, double vy, double *feq) {
  double v2 = vx * vx + vy * vy;
  double meq[9];
  meq[0] = rho;
  meq[1] = rho * (-2.0 + 3.0 * v2);
  meq[2] = rho * (1.0 - 3.0 * v2);
  meq[3] = rho * vx;
  meq[4] = -(rho * vx);
  meq[5] = rho * vy;
  meq[6] = -(rho * vy);
  meq[7] = rho * (vx * vx - vy * vy);
  meq[8] = rho * (vx * vy);
  double r[9];
  for (int k = 0; k < 9; ++k) r[k] = meq[k] / MNORM[k];
  for (int a = 0; a < 9; ++a) {
    double acc = 0.0;
    for (int k = 0; k < 9; ++k)
      if (MM[k][a] != 0.0) acc = acc + MM[k][a] * r[k];
    feq[a] = acc;
  }
}

/* ---------------------------------------------------------------------- */
/* Simulation state                                                        */
/* ---------------------------------------------------------------------- */
typedef struct {
  int nx, ny, wall_bot, wall_top;
  int kind;
  double eos[8];
  double T;
  double A, kappa, Gw;
  int n_iter, wetting; /* wetting 0 = geometric (Eqs. 19-21), 1 = Martys-Chen (Eq. 14) */
  double s[9];
  double rho_max;            /* instability bound; psi = U = 0 at and above it */
  double ghost_max;          /* upper clamp of the ghost densities */
  double *c_bot, *c_top;     /* sin(pi/2 - theta) per wall node */
  double *cot_bot, *cot_top; /* tan(pi/2 - theta) per wall node (Eq. 19 only) */
  double *f, *fn;            /* [9][ny][nx] */
  double *rho, *psi, *U;     /* [ny][nx]; wall rows hold the ghost values */
  double *Fx, *Fy, *Qxx, *Qyy, *Qxy; /* [ny][nx], last computed step */
  long long steps;
  int unstable;
} orc_sim;

static int is_solid_row(const orc_sim *S, int y) {
  return (S->wall_bot && y == 0) || (S->wall_top && y == S->ny - 1);
}
static int is_fluid(const orc_sim *S, int y) { return !is_solid_row(S, y); }
static int wrapx(const orc_sim *S, int x) { return (x % S->nx + S->nx) % S->nx; }
static int wrapy(const orc_sim *S, int y) { return (y % S->ny + S->ny) % S->ny; }
#define IDX(S, y, x) ((size_t)(y) * (size_t)(S)->nx + (size_t)(x))
#define FIDX(S, a, y, x) (((size_t)(a) * (size_t)(S)->ny + (size_t)(y)) * (size_t)(S)->nx + (size_t)(x))

/* params[] = {A, kappa, G_w, s_rho, s_e, s_eps, s_j, s_q, s_nu}
 * theta[ny*nx] in radians, read at the wall rows only.  Ghost densities are
 * clamped to [0, ghost_max] (ghost_max <= 0 means rho_max). */
void *orc_create(int nx, int ny, int wall_bot, int wall_top, int kind, const double *eos, double T,
                 const double *params, int n_iter, int wetting, const double *theta, double rho_max,
                 double ghost_max) {
  orc_sim *S = (orc_sim *)calloc(1, sizeof(orc_sim));
  S->nx = nx; S->ny = ny; S->wall_bot = wall_bot; S->wall_top = wall_top;
  S->kind = kind;
  memcpy(S->eos, eos, sizeof(S->eos));
  S->T = T;
  S->A = params[0]; S->kappa = params[1]; S->Gw = params[2];
  double s_rho = params[3], s_e = params[4], s_eps = params[5], s_j = params[6], s_q = params[7],
         s_nu = params[8];
  double s[9] = {s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_nu, s_nu};
  memcpy(S->s, s, sizeof(s));
  S->n_iter = n_iter; S->wetting = wetting;
  S->rho_max = rho_max;
  S->ghost_max = (ghost_max > 0.0 && ghost_max < rho_max) ? ghost_max : rho_max;
  size_t n = (size_t)nx * (size_t)ny;
  S->c_bot = calloc(nx, sizeof(double)); S->c_top = calloc(nx, sizeof(double));
  S->cot_bot = calloc(nx, sizeof(double)); S->cot_top = calloc(nx, sizeof(double));
  for (int x = 0; x < nx; ++x) {
    double tb = theta ? theta[IDX(S, 0, x)] : M_PI / 2;
    double tt = theta ? theta[IDX(S, ny - 1, x)] : M_PI / 2;
    S->c_bot[x] = sin(M_PI / 2 - tb); S->cot_bot[x] = tan(M_PI / 2 - tb);
    S->c_top[x] = sin(M_PI / 2 - tt); S->cot_top[x] = tan(M_PI / 2 - tt);
  }
  S->f = calloc(9 * n, sizeof(double)); S->fn = calloc(9 * n, sizeof(double));
  S->rho = calloc(n, sizeof(double)); S->psi = calloc(n, sizeof(double)); S->U = calloc(n, sizeof(double));
  S->Fx = calloc(n, sizeof(double)); S->Fy = calloc(n, sizeof(double));
  S->Qxx = calloc(n, sizeof(double)); S->Qyy = calloc(n, sizeof(double)); S->Qxy = calloc(n, sizeof(double));
  return S;
}

void orc_destroy(void *h) {
  orc_sim *S = (orc_sim *)h;
  if (!S) return;
  free(S->c_bot); free(S->c_top); free(S->cot_bot); free(S->cot_top);
  free(S->f); free(S->fn); free(S->rho); free(S->psi); free(S->U);
  free(S->Fx); free(S->Fy); free(S->Qxx); free(S->Qyy); free(S->Qxy);
  free(S);
}

/* f := f_eq(rho, v = 0) at every fluid node; wall rows are left at zero. */
void orc_set_rho(void *h, const double *rho) {
  orc_sim *S = (orc_sim *)h;
  double feq[9];
  for (int y = 0; y < S->ny; ++y)
    for (int x = 0; x < S->nx; ++x) {
      for (int a = 0; a < 9; ++a) S->f[FIDX(S, a, y, x)] = 0.0;
      if (!is_fluid(S, y)) continue;
      orc_feq(rho[IDX(S, y, x)], 0.0, 0.0, feq);
      for (int a = 0; a < 9; ++a) S->f[FIDX(S, a, y, x)] = feq[a];
    }
}

void orc_set_f(void *h, const double *f) {
  orc_sim *S = (orc_sim *)h;
  memcpy(S->f, f, 9 * (size_t)S->nx * S->ny * sizeof(double));
}
void orc_get_f(void *h, double *f) {
  orc_sim *S = (orc_sim *)h;
  memcpy(f, S->f, 9 * (size_t)S->nx * S->ny * sizeof(double));
}

/* rho = f0 + f1 + ... + f8, left to right (Eq. 1's zeroth moment). */
static double node_rho(const orc_sim *S, const double *f, int y, int x) {
  double r = 0.0;
  for (int a = 0; a < 9; ++a) r = r + f[FIDX(S, a, y, x)];
  return r;
}

/* Fill rho, psi, U at fluid nodes and the ghost values on the wall rows. */
static void orc_fields(orc_sim *S) {
  int nx = S->nx, ny = S->ny;
  for (int y = 0; y < ny; ++y) {
    if (!is_fluid(S, y)) continue;
    for (int x = 0; x < nx; ++x) {
      double r = node_rho(S, S->f, y, x), p, u;
      S->rho[IDX(S, y, x)] = r;
      orc_psi_U(S->kind, S->eos, S->T, r, &p, &u);
      S->psi[IDX(S, y, x)] = p;
      S->U[IDX(S, y, x)] = u;
    }
  }
  for (int w = 0; w < 2; ++w) {
    int on = w == 0 ? S->wall_bot : S->wall_top;
    if (!on) continue;
    int yg = w == 0 ? 0 : ny - 1;      /* ghost row */
    int y1 = w == 0 ? 1 : ny - 2;      /* boundary row */
    int y2 = w == 0 ? 2 : ny - 3;      /* second row */
    for (int x = 0; x < nx; ++x) {
      if (S->wetting == 1) {
        /* Martys-Chen: solid neighbours carry no pseudo-potential; the wall
         * acts only through the Eq. 14 force. */
        S->rho[IDX(S, yg, x)] = 0.0;
        S->psi[IDX(S, yg, x)] = 0.0;
        S->U[IDX(S, yg, x)] = 0.0;
        continue;
      }
      const double *c = w == 0 ? S->c_bot : S->c_top;
      const double *cot = w == 0 ? S->cot_bot : S->cot_top;
      double g = orc_ghost(S->rho[IDX(S, y1, wrapx(S, x - 1))], S->rho[IDX(S, y1, wrapx(S, x + 1))],
                           S->rho[IDX(S, y1, x)], S->rho[IDX(S, y2, x)], c[x], cot[x], S->n_iter,
                           S->ghost_max);
      double p, u;
      /* rho_max is the root of U = p - rho/3 (Eq. 10), so psi = U = 0 there
       * by definition; evaluating the EOS at the root would only return the
       * square root of a rounding residue. */
      if (g >= S->rho_max) { p = 0.0; u = 0.0; }
      else orc_psi_U(S->kind, S->eos, S->T, g, &p, &u);
      S->rho[IDX(S, yg, x)] = g;
      S->psi[IDX(S, yg, x)] = p;
      S->U[IDX(S, yg, x)] = u;
    }
  }
}

/* Force (Eq. 9 plus Eq. 14 for Martys-Chen) and Eq. 17 tensor at fluid node
 * (x, y).  Neighbours on a wall row take the ghost values (geometric) or zero
 * (Martys-Chen).  Eqs. 7-8 as printed drop e_alpha; Eq. 9 carries it.  Eq. 17
 * is read with the prefactor G/2 of the G-scaled form it is quoted from.
 * Pins: uniform psi gives F = 0; smooth fields give F -> -grad U with second
 * order; a periodic box conserves momentum; sigma scales as 1 - kappa. */
static void orc_force_Q(const orc_sim *S, int y, int x, double *Fx, double *Fy, double *Qxx, double *Qyy,
                        double *Qxy) {
  double psi0 = S->psi[IDX(S, y, x)];
  double spx = 0, spy = 0, sUx = 0, sUy = 0, ssx = 0, ssy = 0;
  double qxx1 = 0, qyy1 = 0, qxy1 = 0, qxx2 = 0, qyy2 = 0, qxy2 = 0;
  for (int a = 1; a < 9; ++a) {
    int yn = wrapy(S, y + EY[a]), xn = wrapx(S, x + EX[a]);
    double pn = S->psi[IDX(S, yn, xn)], un = S->U[IDX(S, yn, xn)];
    double w = orc_w(a);
    double solid = is_solid_row(S, yn) ? 1.0 : 0.0;
    if (EX[a] != 0) {
      double tp = w * pn, tu = w * un, ts = w * solid;
      if (EX[a] > 0) { spx = spx + tp; sUx = sUx + tu; ssx = ssx + ts; }
      else { spx = spx - tp; sUx = sUx - tu; ssx = ssx - ts; }
    }
    if (EY[a] != 0) {
      double tp = w * pn, tu = w * un, ts = w * solid;
      if (EY[a] > 0) { spy = spy + tp; sUy = sUy + tu; ssy = ssy + ts; }
      else { spy = spy - tp; sUy = sUy - tu; ssy = ssy - ts; }
    }
    double t1 = w * (pn - psi0);
    double t2 = w * (pn * pn - psi0 * psi0);
    int exx = EX[a] * EX[a], eyy = EY[a] * EY[a], exy = EX[a] * EY[a];
    if (exx) { qxx1 = qxx1 + t1; qxx2 = qxx2 + t2; }
    if (eyy) { qyy1 = qyy1 + t1; qyy2 = qyy2 + t2; }
    if (exy > 0) { qxy1 = qxy1 + t1; qxy2 = qxy2 + t2; }
    if (exy < 0) { qxy1 = qxy1 - t1; qxy2 = qxy2 - t2; }
  }
  double cpsi = ((1.0 - S->A) * ORC_G) * psi0;
  double fx = -(S->A * sUx) - cpsi * spx;
  double fy = -(S->A * sUy) - cpsi * spy;
  if (S->wetting == 1) {
    double gp = S->Gw * psi0;
    fx = fx + (-(gp * ssx));
    fy = fy + (-(gp * ssy));
  }
  double pre = S->kappa * (ORC_G * 0.5);
  double c1 = (1.0 - S->A) * psi0, c2 = S->A * 0.5;
  *Fx = fx;
  *Fy = fy;
  *Qxx = pre * ((c1 * qxx1) + (c2 * qxx2));
  *Qyy = pre * ((c1 * qyy1) + (c2 * qyy2));
  *Qxy = pre * ((c1 * qxy1) + (c2 * qxy2));
}

/* One full timestep in the paper's order: rho -> psi, U (Eqs. 10-11) -> ghost
 * rows (Eqs. 19-21) -> F (Eq. 9, Eq. 14) -> Q, C (Eqs. 16-17) -> collision
 * (Eqs. 4, 6, 15) -> streaming (left side of Eq. 1) with half-way bounce-back
 * at the solid rows.  Returns 0, or -4 when a fluid density is NaN, <= 0 or
 * above rho_max after the step. */
int orc_step(void *h, int nsteps) {
  orc_sim *S = (orc_sim *)h;
  int nx = S->nx, ny = S->ny;
  double fl[9], fs[9];
  for (int it = 0; it < nsteps; ++it) {
    orc_fields(S);
    memset(S->fn, 0, 9 * (size_t)nx * ny * sizeof(double));
    for (int y = 0; y < ny; ++y) {
      if (!is_fluid(S, y)) continue;
      for (int x = 0; x < nx; ++x) {
        double Fx, Fy, Qxx, Qyy, Qxy;
        orc_force_Q(S, y, x, &Fx, &Fy, &Qxx, &Qyy, &Qxy);
        S->Fx[IDX(S, y, x)] = Fx; S->Fy[IDX(S, y, x)] = Fy;
        S->Qxx[IDX(S, y, x)] = Qxx; S->Qyy[IDX(S, y, x)] = Qyy; S->Qxy[IDX(S, y, x)] = Qxy;
        for (int a = 0; a < 9; ++a) fl[a] = S->f[FIDX(S, a, y, x)];
        orc_collide(fl, S->rho[IDX(S, y, x)], Fx, Fy, Qxx, Qyy, Qxy, S->s, fs);
        for (int a = 0; a < 9; ++a) {
          int yt = wrapy(S, y + EY[a]);
          if (is_solid_row(S, yt)) {
            S->fn[FIDX(S, OPP[a], y, x)] = fs[a];  /* half-way bounce-back */
          } else {
            S->fn[FIDX(S, a, yt, wrapx(S, x + EX[a]))] = fs[a];
          }
        }
      }
    }
    double *t = S->f; S->f = S->fn; S->fn = t;
    S->steps++;
    for (int y = 0; y < ny; ++y) {
      if (!is_fluid(S, y)) continue;
      for (int x = 0; x < nx; ++x) {
        double r = node_rho(S, S->f, y, x);
        if (!(r > 0.0) || r > S->rho_max) S->unstable = 1;
      }
    }
    if (S->unstable) return -4;
  }
  return 0;
}

/* Fields of the current state: rho at fluid nodes (ghost rows included after
 * orc_fields), psi, U and the force and Eq. 17 tensor of the NEXT step. */
void orc_get_fields(void *h, double *rho, double *psi, double *U, double *Fx, double *Fy, double *Qxx,
                    double *Qyy, double *Qxy) {
  orc_sim *S = (orc_sim *)h;
  size_t n = (size_t)S->nx * S->ny;
  orc_fields(S);
  for (int y = 0; y < S->ny; ++y) {
    for (int x = 0; x < S->nx; ++x) {
      size_t i = IDX(S, y, x);
      double fx = 0, fy = 0, qxx = 0, qyy = 0, qxy = 0;
      if (is_fluid(S, y)) orc_force_Q(S, y, x, &fx, &fy, &qxx, &qyy, &qxy);
      if (Fx) Fx[i] = fx;
      if (Fy) Fy[i] = fy;
      if (Qxx) Qxx[i] = qxx;
      if (Qyy) Qyy[i] = qyy;
      if (Qxy) Qxy[i] = qxy;
    }
  }
  if (rho) memcpy(rho, S->rho, n * sizeof(double));
  if (psi) memcpy(psi, S->psi, n * sizeof(double));
  if (U) memcpy(U, S->U, n * sizeof(double));
}

/* Macroscopic density and (half-force shifted) velocity u = (j + F/2)/rho at
 * fluid nodes; zero on the wall rows. */
void orc_get_macro(void *h, double *rho, double *ux, double *uy) {
  orc_sim *S = (orc_sim *)h;
  orc_fields(S);
  for (int y = 0; y < S->ny; ++y)
    for (int x = 0; x < S->nx; ++x) {
      size_t i = IDX(S, y, x);
      if (!is_fluid(S, y)) {
        if (rho) rho[i] = 0.0;
        if (ux) ux[i] = 0.0;
        if (uy) uy[i] = 0.0;
        continue;
      }
      double fx, fy, qxx, qyy, qxy;
      orc_force_Q(S, y, x, &fx, &fy, &qxx, &qyy, &qxy);
      double jx = 0.0, jy = 0.0;
      for (int a = 0; a < 9; ++a) {
        if (MM[3][a] != 0.0) jx = jx + MM[3][a] * S->f[FIDX(S, a, y, x)];
        if (MM[5][a] != 0.0) jy = jy + MM[5][a] * S->f[FIDX(S, a, y, x)];
      }
      double r = S->rho[i];
      if (rho) rho[i] = r;
      if (ux) ux[i] = (jx + 0.5 * fx) / r;
      if (uy) uy[i] = (jy + 0.5 * fy) / r;
    }
}

/* Total mass: sum of rho over fluid nodes, row-major order. */
double orc_mass(void *h) {
  orc_sim *S = (orc_sim *)h;
  double m = 0.0;
  for (int y = 0; y < S->ny; ++y) {
    if (!is_fluid(S, y)) continue;
    for (int x = 0; x < S->nx; ++x) m = m + node_rho(S, S->f, y, x);
  }
  return m;
}

/* ---------------------------------------------------------------------- */
/* Apparent contact angle (the paper only says angles were "measured")     */
/* ---------------------------------------------------------------------- */
/* On a density field rho[ny][nx] and a droplet sitting on `wall` (0 bottom,
 * 1 top) inside columns [x0, x1):
 *   - the centre column xc is the column with the largest sum of rho over
 *     the wall's half of the domain (bottom: rows 1 .. ny/2-1, top: rows
 *     ny/2 .. ny-2); ties go to the lowest x;
 *   - the base row is the boundary row (1 or ny-2); L is the distance
 *     between the linearly interpolated rho_mid crossings that bound the
 *     liquid run of the base row containing xc;
 *   - H is the distance from the base row to the linearly interpolated
 *     rho_mid crossing found walking away from the wall along xc;
 *   - theta = 2 atan2(2H, L), exact for a circular cap cut by the base row.
 * Returns 0, or -1 if the base row at xc is not liquid or a liquid run
 * reaches the region edge or the domain middle. */
int orc_contact_angle_field(const double *rho, int nx, int ny, int wall, int x0, int x1, double rho_mid,
                            double *theta, double *H, double *L, int *xc_out) {
  int ylo = wall == 0 ? 1 : ny / 2, yhi = wall == 0 ? ny / 2 : ny - 1; /* [ylo, yhi) */
  int base = wall == 0 ? 1 : ny - 2, dir = wall == 0 ? 1 : -1;
  double best = -DBL_MAX;
  int xc = -1;
  for (int x = x0; x < x1; ++x) {
    double cs = 0.0;
    for (int y = ylo; y < yhi; ++y) cs = cs + rho[(size_t)y * nx + x];
    if (cs > best) { best = cs; xc = x; }
  }
  if (xc_out) *xc_out = xc;
  const double *row = rho + (size_t)base * nx;
  if (!(row[xc] >= rho_mid)) return -1;
  int xl = xc, xr = xc;
  while (xl - 1 >= x0 && row[xl - 1] >= rho_mid) xl--;
  while (xr + 1 < x1 && row[xr + 1] >= rho_mid) xr++;
  if (xl - 1 < x0 || xr + 1 >= x1) return -1;
  double xleft = (double)(xl - 1) + (rho_mid - row[xl - 1]) / (row[xl] - row[xl - 1]);
  double xright = (double)xr + (row[xr] - rho_mid) / (row[xr] - row[xr + 1]);
  int y = base, steps = 0;
  int ymax = wall == 0 ? yhi : ylo - 1; /* exclusive end of the walk */
  while (y + dir != ymax && rho[(size_t)(y + dir) * nx + xc] >= rho_mid) { y += dir; steps++; }
  if (y + dir == ymax) return -1;
  double ra = rho[(size_t)y * nx + xc], rb = rho[(size_t)(y + dir) * nx + xc];
  double h = (double)steps + (ra - rho_mid) / (ra - rb);
  *H = h;
  *L = xright - xleft;
  *theta = 2.0 * atan2(2.0 * h, *L);
  return 0;
}
