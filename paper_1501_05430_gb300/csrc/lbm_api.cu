// lbm_api.cu -- the C ABI of liblbm (include/lbm.h): context management,
// host-side thermodynamic set-up (critical point, coexistence, EOS bounds)
// and the orchestration of the device kernels for one timestep.
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <new>

#include "lbm_internal.h"

namespace {

// ---------------------------------------------------------------------------
// Host thermodynamics
// ---------------------------------------------------------------------------

// Brent's method (inverse quadratic interpolation with bisection fallback) for
// a root of g on [a, b] with g(a), g(b) of opposite signs.
double brent(const std::function<double(double)> &g, double a, double b, double tol = 0.0, int maxit = 400) {
  double fa = g(a), fb = g(b);
  if (fa == 0.0) return a;
  if (fb == 0.0) return b;
  double c = a, fc = fa, d = b - a, e = d;
  for (int it = 0; it < maxit; ++it) {
    if ((fb > 0) == (fc > 0)) { c = a; fc = fa; d = b - a; e = d; }
    if (fabs(fc) < fabs(fb)) { a = b; b = c; c = a; fa = fb; fb = fc; fc = fa; }
    double t = 2.0 * DBL_EPSILON * fabs(b) + 0.5 * tol;
    double m = 0.5 * (c - b);
    if (fabs(m) <= t || fb == 0.0) return b;
    if (fabs(e) >= t && fabs(fa) > fabs(fb)) {
      double s = fb / fa, p, q;
      if (a == c) {
        p = 2.0 * m * s;
        q = 1.0 - s;
      } else {
        double qq = fa / fc, r = fb / fc;
        p = s * (2.0 * m * qq * (qq - r) - (b - a) * (r - 1.0));
        q = (qq - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (p > 0) q = -q; else p = -p;
      if (2.0 * p < 3.0 * m * q - fabs(t * q) && p < fabs(0.5 * e * q)) { e = d; d = p / q; }
      else { d = m; e = m; }
    } else {
      d = m;
      e = m;
    }
    a = b;
    fa = fb;
    b += fabs(d) > t ? d : (m > 0 ? t : -t);
    fb = g(b);
  }
  return b;
}

struct CS {
  double a, b, R;
  double eta(double r) const { return b * r * 0.25; }
  double p(double T, double r) const {
    double e = eta(r), om = 1.0 - e;
    return r * R * T * (1.0 + e + e * e - e * e * e) / (om * om * om) - a * r * r;
  }
  // dp/drho = R T (1 + 4e + 4e^2 - 4e^3 + e^4)/(1-e)^4 - 2 a rho
  double dp(double T, double r) const {
    double e = eta(r), om = 1.0 - e;
    return R * T * (1.0 + 4.0 * e + 4.0 * e * e - 4.0 * e * e * e + e * e * e * e) / (om * om * om * om) - 2.0 * a * r;
  }
  // chemical potential (integral of dp/rho) up to a constant
  double mu(double T, double r) const {
    double e = eta(r), om = 1.0 - e;
    return R * T * (log(e) + e * (8.0 - 9.0 * e + 3.0 * e * e) / (om * om * om)) - 2.0 * a * r;
  }
  double rmax() const { return 4.0 / b; }
};

// Critical point: the packing fraction solves e^5 - 5e^4 + 4e^3 + 20e^2 + 5e - 1 = 0
// (dp/drho = d2p/drho2 = 0 with T eliminated); Newton from e = 0.13.
void cs_critical(const CS &cs, double *Tc, double *rc) {
  double e = 0.13;
  for (int it = 0; it < 60; ++it) {
    double g = ((((e - 5.0) * e + 4.0) * e + 20.0) * e + 5.0) * e - 1.0;
    double dg = (((5.0 * e - 20.0) * e + 12.0) * e + 40.0) * e + 5.0;
    double step = g / dg;
    e -= step;
    if (fabs(step) < 1e-17) break;
  }
  double om = 1.0 - e;
  double kpp = (8.0 + 20.0 * e - 4.0 * e * e) / (om * om * om * om * om);
  *Tc = 8.0 * cs.a / (cs.b * cs.R * kpp);
  *rc = 4.0 * e / cs.b;
}

// Maxwell construction: the saturation pressure p_s at which the vapour and
// liquid branch densities have equal chemical potential (Brent on p_s, Brent
// for the branch densities at each p_s).
int cs_coexistence(const CS &cs, double T, double *rv, double *rl) {
  double Tc, rc;
  cs_critical(cs, &Tc, &rc);
  if (!(T > 0.0 && T < Tc)) return LBM_EINVAL;
  double top = cs.rmax() * (1.0 - 1e-13);
  auto dp = [&](double r) { return cs.dp(T, r); };
  double sv = brent(dp, 1e-14 * rc, rc);  // vapour spinodal
  double sl = brent(dp, rc, top);          // liquid spinodal
  double plo = fmax(cs.p(T, sl), 0.0), phi = cs.p(T, sv);
  double vap = 0, liq = 0;
  auto branches = [&](double ps) {
    vap = brent([&](double r) { return cs.p(T, r) - ps; }, 1e-300, sv);
    liq = brent([&](double r) { return cs.p(T, r) - ps; }, sl, top);
    return cs.mu(T, liq) - cs.mu(T, vap);
  };
  double ps = brent(branches, plo * (1.0 + 1e-15) + 1e-300, phi * (1.0 - 1e-15));
  branches(ps);
  *rv = vap;
  *rl = liq;
  return LBM_OK;
}

// Eq. 11 pressure and the Eqs. 12-13 relations between (rho_v, rho_l) and the
// breakpoints (rho1, rho2).
double pw_p(const lbm_eos &e, double r) {
  if (r <= e.rho1) return r * e.theta_v;
  if (r <= e.rho2) return e.rho1 * e.theta_v + (r - e.rho1) * e.theta_m;
  return e.rho1 * e.theta_v + (e.rho2 - e.rho1) * e.theta_m + (r - e.rho2) * e.theta_l;
}

int pw_coexistence(const lbm_eos &e, double *rv, double *rl) {
  // Eq. 12 gives rho_l(rho_v); Eq. 13 is then a scalar equation in rho_v.
  auto liq = [&](double v) { return e.rho2 - ((e.rho1 - v) * e.theta_v + (e.rho2 - e.rho1) * e.theta_m) / e.theta_l; };
  auto chem = [&](double v) {
    double l = liq(v);
    return e.theta_v * log(e.rho1 / v) + e.theta_m * log(e.rho2 / e.rho1) + e.theta_l * log(l / e.rho2);
  };
  double lo = e.rho1 * 1e-12, hi = e.rho1 * (1.0 - 1e-14);
  if (!(liq(hi) > e.rho2)) return LBM_EINVAL;
  double glo = chem(lo), ghi = chem(hi);
  if (!isfinite(glo) || !isfinite(ghi) || (glo > 0) == (ghi > 0)) return LBM_EINVAL;
  double v = brent(chem, lo, hi);
  *rv = v;
  *rl = liq(v);
  return (*rl > e.rho2) ? LBM_OK : LBM_EINVAL;
}

double eos_p(const lbm_eos &e, double T, double r) {
  if (e.kind == LBM_EOS_CARNAHAN_STARLING) return CS{e.a, e.b, e.R}.p(T, r);
  return pw_p(e, r);
}

// Smallest rho > rho_l with p(rho) = rho/3 (psi^2 = 2(rho/3 - p) >= 0 below it).
double eos_rho_max(const lbm_eos &e, double T, double rl) {
  auto U = [&](double r) { return eos_p(e, T, r) - r / 3.0; };
  if (e.kind == LBM_EOS_CARNAHAN_STARLING) {
    CS cs{e.a, e.b, e.R};
    double top = cs.rmax() * (1.0 - 1e-13);
    if (U(rl) >= 0.0) return rl;
    return brent(U, rl, top);
  }
  double slope = e.theta_l - 1.0 / 3.0;
  if (slope <= 0.0) return DBL_MAX;
  double root = e.rho2 - U(e.rho2) / slope;
  return root > rl ? root : DBL_MAX;
}

// Coexistence densities and the derived bounds of a context (lbm_eos_bounds).
int eos_bounds(const lbm_eos &e, double T, double *rv, double *rl, double *rmax, double *rmid) {
  int st = e.kind == LBM_EOS_CARNAHAN_STARLING ? cs_coexistence(CS{e.a, e.b, e.R}, T, rv, rl)
                                               : pw_coexistence(e, rv, rl);
  if (st != LBM_OK) return LBM_EINVAL;
  *rmax = eos_rho_max(e, T, *rl);
  *rmid = 0.5 * (*rv + *rl);
  return LBM_OK;
}

int validate_eos(const lbm_eos *e) {
  if (!e) return LBM_EINVAL;
  if (e->kind == LBM_EOS_CARNAHAN_STARLING) {
    if (!(e->a > 0 && e->b > 0 && e->R > 0)) return LBM_EINVAL;
    return LBM_OK;
  }
  if (e->kind == LBM_EOS_PIECEWISE) {
    if (!(e->rho1 > 0 && e->rho2 > e->rho1 && e->theta_v > 0 && e->theta_v < 1.0 / 3.0 && e->theta_m < 0 &&
          e->theta_l > 0))
      return LBM_EINVAL;
    return LBM_OK;
  }
  return LBM_EINVAL;
}

// ---------------------------------------------------------------------------
// Context helpers
// ---------------------------------------------------------------------------

#define CK(call)                                   \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) {                       \
      C->status = LBM_ECUDA;                       \
      return LBM_ECUDA;                            \
    }                                              \
  } while (0)

size_t real_size(int precision) { return precision == 64 ? sizeof(double) : sizeof(float); }
size_t n_nodes(const lbm_ctx *C) { return (size_t)C->nx * C->ny; }

// The device address of pinned (page-locked) host memory that the current
// device maps, or NULL for any other pointer (pageable host memory, device
// memory, pinned memory of another device): kernels read such host memory
// directly.
void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  int dev = -1;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || a.device != dev) return nullptr;
  return a.devicePointer;
}

int ensure_fields(lbm_ctx *C) {
  if (C->d_fields) return LBM_OK;
  if (cudaMalloc(&C->d_fields, 3 * n_nodes(C) * real_size(C->precision)) != cudaSuccess) {
    C->d_fields = nullptr;
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  return LBM_OK;
}

int ensure_aux(lbm_ctx *C) {
  if (C->d_aux) return LBM_OK;
  if (cudaMalloc(&C->d_aux, 7 * n_nodes(C) * sizeof(double)) != cudaSuccess) {
    C->d_aux = nullptr;
    cudaGetLastError();
    return LBM_ENOMEM;
  }
  return LBM_OK;
}

// Reference-path fields (rho, psi, U incl. ghost rows) of the current state.
int compute_fields(lbm_ctx *C) {
  int st = ensure_fields(C);
  if (st) return st;
  CK(lbm_ref_fields(C, C->f[C->cur], C->d_fields, &C->launches));
  return LBM_OK;
}

int read_flags(lbm_ctx *C) {
  int h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, C->d_flag, sizeof(h), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  if (h[1]) C->status = LBM_ETIMEOUT;
  else if (h[0]) C->status = LBM_EUNSTABLE;
  return C->status;
}

// One step from array src to src ^ 1, with the kernel chosen at creation.
cudaError_t launch_step(lbm_ctx *C, int src, unsigned long long *launches) {
  const int dst = src ^ 1;
  if (C->kernel_in_use == LBM_KERNEL_FUSED) return lbm_fused_step(C, src, launches);
  cudaError_t e = lbm_ref_fields(C, C->f[src], C->d_fields, launches);
  if (e == cudaSuccess) e = lbm_ref_collide(C, C->f[src], C->f[dst], C->d_fields, launches);
  return e;
}

int launches_per_step(const lbm_ctx *C) { return C->kernel_in_use == LBM_KERNEL_FUSED ? 1 : 2; }

// Steps per captured graph (even), or 0 when graphs are off or impossible
// (the legacy default stream cannot be captured).
int graph_steps(const lbm_ctx *C) {
  int g = C->params.graph_steps;
  if (g <= 0 || !C->stream) return 0;
  return g + (g & 1);
}

// Capture G steps starting from array `start` into an executable graph.
int capture_steps(lbm_ctx *C, int start, int G, cudaGraphExec_t *out) {
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(C->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  unsigned long long dummy = 0;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < G && e == cudaSuccess; ++k) e = launch_step(C, start ^ (k & 1), &dummy);
  cudaError_t e2 = cudaStreamEndCapture(C->stream, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return LBM_ECUDA;
  }
  return LBM_OK;
}

// The graph lengths of a context and their executable graphs for both
// starting arrays (captured once; capture only records launches).
int ensure_graphs(lbm_ctx *C, int G) {
  if (C->graphs_ready) return LBM_OK;
  int n = 0;
  C->graph_len[n++] = G;
  int p2 = 1;
  while (p2 * 2 < G && p2 < (1 << 30)) p2 *= 2;
  for (; p2 >= 2 && n < lbm_ctx::kMaxGraphs; p2 /= 2)
    if (p2 < G) C->graph_len[n++] = p2;
  C->ngraph = n;
  for (int start = 0; start < 2; ++start)
    for (int k = 0; k < n; ++k) {
      if (C->step_graph[start][k]) continue;  // kept from an interrupted earlier attempt
      int st = capture_steps(C, start, C->graph_len[k], &C->step_graph[start][k]);
      if (st) return st;
    }
  C->graphs_ready = 1;
  return LBM_OK;
}

int create_impl(int nx, int ny, const lbm_eos *eos, double T, double tau, const double *theta,
                const uint8_t *wall_mask, const lbm_params *params, void *stream, void *state, size_t state_bytes,
                lbm_ctx **out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  lbm_params P;
  if (params) P = *params; else lbm_params_default(&P);
  if (nx < 4 || ny < 5 || !(tau > 0.5) || validate_eos(eos)) return LBM_EINVAL;
  if (P.precision != 32 && P.precision != 64) return LBM_EINVAL;
  if (P.n_iter < 0 || P.n_iter > 64) return LBM_EINVAL;
  if (P.wetting != LBM_WET_GEOMETRIC && P.wetting != LBM_WET_MARTYS_CHEN) return LBM_EINVAL;
  if (P.kernel < LBM_KERNEL_AUTO || P.kernel > LBM_KERNEL_FUSED) return LBM_EINVAL;
  if (P.check_every < 0 || P.graph_steps < 0) return LBM_EINVAL;
  if ((size_t)nx * (size_t)ny > ((size_t)1 << 31) / 9) return LBM_EUNSUPPORTED;
  // walls: none, or exactly the two full rows y = 0 and y = ny - 1
  int walls = 0;
  if (wall_mask) {
    size_t nsolid = 0;
    for (size_t i = 0; i < (size_t)nx * ny; ++i) nsolid += wall_mask[i] ? 1 : 0;
    if (nsolid) {
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          int want = (y == 0 || y == ny - 1);
          if ((wall_mask[(size_t)y * nx + x] != 0) != (want != 0)) return LBM_EUNSUPPORTED;
        }
      walls = 1;
    }
  }
  double rv = 0, rl = 0, rmax = 0, rmid = 0;
  if (eos_bounds(*eos, T, &rv, &rl, &rmax, &rmid) != LBM_OK) return LBM_EINVAL;
  if (theta && walls) {
    for (int x = 0; x < nx; ++x) {
      double tb = theta[x], tt = theta[(size_t)(ny - 1) * nx + x];
      if (!(tb > 0.0 && tb < M_PI) || !(tt > 0.0 && tt < M_PI)) return LBM_EINVAL;
    }
  }
  lbm_ctx *C = new (std::nothrow) lbm_ctx();
  if (!C) return LBM_ENOMEM;
  memset(C, 0, sizeof(*C));
  C->nx = nx;
  C->ny = ny;
  C->walls = walls;
  C->precision = P.precision;
  C->kernel_req = P.kernel;
  C->eos = *eos;
  C->T = T;
  C->tau = tau;
  C->params = P;
  C->rho_v = rv;
  C->rho_l = rl;
  C->rho_max = P.rho_max > 0 ? P.rho_max : rmax;
  C->rho_mid = P.rho_mid > 0 ? P.rho_mid : rmid;
  C->ghost_max = P.rho_ghost_max > 0 ? fmin(P.rho_ghost_max, C->rho_max) : C->rho_max;
  C->stream = (cudaStream_t)stream;
  lbm_dev_params &D = C->dp;
  D.nx = nx;
  D.ny = ny;
  D.walls = walls;
  D.eos_kind = eos->kind;
  D.a = eos->a;
  D.b = eos->b;
  D.R = eos->R;
  D.T = T;
  D.thv = eos->theta_v;
  D.thm = eos->theta_m;
  D.thl = eos->theta_l;
  D.r1 = eos->rho1;
  D.r2 = eos->rho2;
  D.A = P.A;
  D.kappa = P.kappa;
  D.Gw = P.G_w;
  double inv = 1.0 / tau;
  double se = P.s_e > 0 ? P.s_e : inv, seps = P.s_eps > 0 ? P.s_eps : inv, sj = P.s_j > 0 ? P.s_j : inv,
         sq = P.s_q > 0 ? P.s_q : inv, snu = P.s_nu > 0 ? P.s_nu : inv;
  double s[9] = {0.0, se, seps, sj, sq, sj, sq, snu, snu};
  memcpy(D.s, s, sizeof(s));
  D.n_iter = P.n_iter;
  D.wetting = P.wetting;
  D.rho_max = C->rho_max;
  D.ghost_max = C->ghost_max;

  size_t n = (size_t)nx * ny, rs = real_size(P.precision);
  size_t need = 2 * 9 * n * rs;
  int st = LBM_OK;
  if (state) {
    if (state_bytes < need || ((uintptr_t)state & 255)) { delete C; return LBM_EINVAL; }
    C->state = state;
    C->owns_state = 0;
  } else {
    if (cudaMalloc(&C->state, need) != cudaSuccess) { cudaGetLastError(); delete C; return LBM_ENOMEM; }
    C->owns_state = 1;
  }
  C->f[0] = C->state;
  C->f[1] = (char *)C->state + 9 * n * rs;
  C->red_len = 1024;
  bool ok = cudaMalloc(&C->d_coef, 4 * (size_t)nx * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&C->d_dcoef, 4 * (size_t)nx * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&C->d_flag, 4 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&C->d_rho64, n * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&C->d_red, C->red_len * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&C->d_res, 16 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_destroy(C);
    return LBM_ENOMEM;
  }
  // Eqs. 19-21 coefficients per wall node: c = sin(pi/2 - theta) (Eqs. 20-21),
  // cot = tan(pi/2 - theta) (Eq. 19)
  // and their theta derivatives for the adjoint: -cos(pi/2 - theta), -1/cos^2(pi/2 - theta)
  double *coef = (double *)malloc(8 * (size_t)nx * sizeof(double));
  if (!coef) { lbm_destroy(C); return LBM_ENOMEM; }
  double *dcoef = coef + 4 * (size_t)nx;
  for (int x = 0; x < nx; ++x) {
    double tb = theta ? theta[x] : M_PI / 2;
    double tt = theta ? theta[(size_t)(ny - 1) * nx + x] : M_PI / 2;
    coef[x] = sin(M_PI / 2 - tb);
    coef[nx + x] = sin(M_PI / 2 - tt);
    coef[2 * nx + x] = tan(M_PI / 2 - tb);
    coef[3 * nx + x] = tan(M_PI / 2 - tt);
    double cb = cos(M_PI / 2 - tb), ct = cos(M_PI / 2 - tt);
    dcoef[x] = -cb;
    dcoef[nx + x] = -ct;
    dcoef[2 * nx + x] = -1.0 / (cb * cb);
    dcoef[3 * nx + x] = -1.0 / (ct * ct);
  }
  cudaError_t e1 = cudaMemcpy(C->d_coef, coef, 4 * (size_t)nx * sizeof(double), cudaMemcpyHostToDevice);
  if (e1 == cudaSuccess)
    e1 = cudaMemcpy(C->d_dcoef, dcoef, 4 * (size_t)nx * sizeof(double), cudaMemcpyHostToDevice);
  free(coef);
  if (e1 != cudaSuccess || cudaMemsetAsync(C->state, 0, need, C->stream) != cudaSuccess ||
      cudaMemsetAsync(C->d_flag, 0, 4 * sizeof(int), C->stream) != cudaSuccess) {
    cudaGetLastError();
    lbm_destroy(C);
    return LBM_ECUDA;
  }
  // kernel selection
  C->fused_ok = 0;
  if (P.precision == 32 && P.kernel != LBM_KERNEL_REFERENCE) lbm_fused_plan(C);
  if (P.kernel == LBM_KERNEL_FUSED && !C->fused_ok) { lbm_destroy(C); return LBM_EUNSUPPORTED; }
  C->kernel_in_use = C->fused_ok ? LBM_KERNEL_FUSED : LBM_KERNEL_REFERENCE;
  if (C->kernel_in_use == LBM_KERNEL_REFERENCE && (st = ensure_fields(C)) != LBM_OK) {
    lbm_destroy(C);
    return st;
  }
  if (cudaStreamSynchronize(C->stream) != cudaSuccess) { cudaGetLastError(); lbm_destroy(C); return LBM_ECUDA; }
  *out = C;
  return LBM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Public API
// ---------------------------------------------------------------------------
extern "C" {

const char *lbm_strerror(int status) {
  switch (status) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "simulation unstable (density NaN, <= 0 or above rho_max)";
    case LBM_EUNSUPPORTED: return "unsupported configuration";
    case LBM_ETIMEOUT: return "device-side wait timed out";
    case LBM_ENOCONTACT: return "no contact line found in the region";
    default: return "unknown status";
  }
}

int lbm_params_default(lbm_params *p) {
  if (!p) return LBM_EINVAL;
  memset(p, 0, sizeof(*p));
  p->A = -0.6;
  p->kappa = 0.5;
  p->G_w = 0.0;
  p->n_iter = 4;
  p->wetting = LBM_WET_GEOMETRIC;
  p->precision = 32;
  p->kernel = LBM_KERNEL_AUTO;
  p->check_every = 100;
  p->graph_steps = 64;
  return LBM_OK;
}

int lbm_eos_critical(const lbm_eos *eos, double *Tc, double *rho_c) {
  if (!eos || !Tc || !rho_c || validate_eos(eos)) return LBM_EINVAL;
  if (eos->kind != LBM_EOS_CARNAHAN_STARLING) return LBM_EUNSUPPORTED;
  cs_critical(CS{eos->a, eos->b, eos->R}, Tc, rho_c);
  return LBM_OK;
}

int lbm_coexistence(const lbm_eos *eos, double T, double *rho_v, double *rho_l) {
  if (!eos || !rho_v || !rho_l || validate_eos(eos)) return LBM_EINVAL;
  if (eos->kind == LBM_EOS_CARNAHAN_STARLING) return cs_coexistence(CS{eos->a, eos->b, eos->R}, T, rho_v, rho_l);
  return pw_coexistence(*eos, rho_v, rho_l);
}

int lbm_eos_bounds(const lbm_eos *eos, double T, double *rho_v, double *rho_l, double *rho_max, double *rho_mid) {
  if (!eos || validate_eos(eos)) return LBM_EINVAL;
  double v[4];
  int st = eos_bounds(*eos, T, &v[0], &v[1], &v[2], &v[3]);
  if (st) return st;
  double *out[4] = {rho_v, rho_l, rho_max, rho_mid};
  for (int k = 0; k < 4; ++k)
    if (out[k]) *out[k] = v[k];
  return LBM_OK;
}

size_t lbm_required_state_bytes(int nx, int ny, int precision) {
  if (nx <= 0 || ny <= 0 || (precision != 32 && precision != 64)) return 0;
  return 2 * 9 * (size_t)nx * (size_t)ny * real_size(precision);
}

int lbm_create(int nx, int ny, const lbm_eos *eos, double T, double tau, const double *theta,
               const uint8_t *wall_mask, const lbm_params *params, void *stream, lbm_ctx **out) {
  return create_impl(nx, ny, eos, T, tau, theta, wall_mask, params, stream, nullptr, 0, out);
}

int lbm_create_with_buffer(int nx, int ny, const lbm_eos *eos, double T, double tau, const double *theta,
                           const uint8_t *wall_mask, const lbm_params *params, void *stream, void *state,
                           size_t state_bytes, lbm_ctx **out) {
  if (!state) return LBM_EINVAL;
  return create_impl(nx, ny, eos, T, tau, theta, wall_mask, params, stream, state, state_bytes, out);
}

int lbm_set_rho(lbm_ctx *C, const double *rho) {
  if (!C || !rho) return LBM_EINVAL;
  if (C->status) return C->status;
  // Pinned host memory is read by the kernel in place (the GPU maps it; on
  // GB300 over the NVLink-C2C host link, at about the copy engine's rate, and
  // the check and the equilibria overlap the transfer); other host memory is
  // staged through a device copy.  The new state goes to the second
  // distribution array, which becomes the current one only once every fluid
  // density has passed the check: a rejected input leaves the state untouched.
  const double *src = (const double *)mapped_host(rho);
  if (!src) {
    CK(cudaMemcpyAsync(C->d_rho64, rho, n_nodes(C) * sizeof(double), cudaMemcpyHostToDevice, C->stream));
    src = C->d_rho64;
  }
  CK(cudaMemsetAsync(C->d_flag + 2, 0, sizeof(int), C->stream));
  CK(lbm_ref_set_rho(C, src, C->f[C->cur ^ 1], C->d_flag + 2, &C->launches));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, C->d_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  if (bad) return LBM_EINVAL;
  C->cur ^= 1;
  return LBM_OK;
}

int lbm_init_droplets(lbm_ctx *C, int n, const double *xc, const double *radius, const int *wall, double width) {
  if (!C || n < 0 || (n > 0 && (!xc || !radius || !wall)) || !(width > 0)) return LBM_EINVAL;
  if (C->status) return C->status;
  if (n > C->red_len / 3) return LBM_EINVAL;
  double *h = (double *)malloc((size_t)(3 * n + 1) * sizeof(double));
  if (!h) return LBM_ENOMEM;
  for (int k = 0; k < n; ++k) {
    if (!(radius[k] > 0) || (wall[k] != 0 && wall[k] != 1)) { free(h); return LBM_EINVAL; }
    h[3 * k] = xc[k];
    h[3 * k + 1] = radius[k];
    h[3 * k + 2] = (double)wall[k];
  }
  cudaError_t e = n ? cudaMemcpyAsync(C->d_red, h, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, C->stream)
                    : cudaSuccess;
  if (e == cudaSuccess) e = cudaStreamSynchronize(C->stream);
  free(h);
  CK(e);
  CK(lbm_ref_droplets(C, n, C->d_red, width, C->d_rho64, &C->launches));
  CK(lbm_ref_set_rho(C, C->d_rho64, C->f[C->cur], nullptr, &C->launches));
  CK(cudaStreamSynchronize(C->stream));
  return LBM_OK;
}

int lbm_step(lbm_ctx *C, int nsteps) {
  LbmRange nvtx_range("lbm_step");
  if (!C || nsteps < 0) return LBM_EINVAL;
  if (C->status) return C->status;
  const int G = graph_steps(C);
  int it = 0;
  if (G > 0 && nsteps >= 2) {
    int st = ensure_graphs(C, G);
    if (st) return st;
    // whole graphs, longest first (even lengths: each replay starts and ends
    // on the same array); at most one step is left for a direct launch
    for (int k = 0; k < C->ngraph; ++k) {
      const int len = C->graph_len[k];
      while (nsteps - it >= len) {
        CK(cudaGraphLaunch(C->step_graph[C->cur][k], C->stream));
        C->launches += (unsigned long long)len * launches_per_step(C);
        const long long before = C->steps;
        C->steps += len;
        it += len;
        const int ce = C->params.check_every;
        if (ce > 0 && C->steps / ce != before / ce) {
          st = read_flags(C);
          if (st) return st;
        }
      }
    }
  }
  for (; it < nsteps; ++it) {
    CK(launch_step(C, C->cur, &C->launches));
    C->cur ^= 1;
    C->steps++;
    if (C->params.check_every > 0 && C->steps % C->params.check_every == 0) {
      int st = read_flags(C);
      if (st) return st;
    }
  }
  return LBM_OK;
}

int lbm_status(lbm_ctx *C) {
  if (!C) return LBM_EINVAL;
  if (C->status) return C->status;
  return read_flags(C);
}

// The copy stream and chunk events of lbm_get_rho, made at its first use.
bool ensure_xfer(lbm_ctx *C) {
  if (C->xfer) return true;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (int c = 0; c < 8; ++c) {
    if (cudaEventCreateWithFlags(&C->xfer_ev[c], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (int k = 0; k < c; ++k) cudaEventDestroy(C->xfer_ev[k]);
      cudaStreamDestroy(s);
      return false;
    }
  }
  C->xfer = s;
  return true;
}

int lbm_get_rho(lbm_ctx *C, double *rho) {
  if (!C || !rho) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  // Through a device buffer and the copy engine, whatever the destination:
  // kernel stores into pinned host memory crossed the GB300 host link at
  // ~124 GB/s, the copy engine at ~177 GB/s (both measured on 67 MB).  Large
  // fields go in 8 row chunks: the copy of each chunk (on a second stream)
  // overlaps the density kernel of the next.
  const size_t n = n_nodes(C);
  if (n >= ((size_t)1 << 20) && C->ny >= 8 && ensure_xfer(C)) {
    const int K = 8, rows = (C->ny + K - 1) / K;
    for (int c = 0; c < K; ++c) {
      const int r0 = c * rows, r1 = std::min(C->ny, r0 + rows);
      if (r1 <= r0) break;
      const size_t off = (size_t)r0 * C->nx, cnt = (size_t)(r1 - r0) * C->nx;
      CK(lbm_rho64_rows(C, C->f[C->cur], C->d_rho64, r0, r1, &C->launches));
      CK(cudaEventRecord(C->xfer_ev[c], C->stream));
      CK(cudaStreamWaitEvent(C->xfer, C->xfer_ev[c], 0));
      CK(cudaMemcpyAsync(rho + off, C->d_rho64 + off, cnt * sizeof(double), cudaMemcpyDeviceToHost, C->xfer));
    }
    CK(cudaStreamSynchronize(C->xfer));
    return LBM_OK;
  }
  CK(lbm_rho64(C, C->f[C->cur], C->d_rho64, &C->launches));
  CK(cudaMemcpyAsync(rho, C->d_rho64, n * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return LBM_OK;
}

int lbm_get_fields(lbm_ctx *C, double *rho, double *psi, double *U, double *Fx, double *Fy, double *Qxx,
                   double *Qyy, double *Qxy) {
  if (!C) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  int st = compute_fields(C);
  if (st) return st;
  if ((st = ensure_aux(C)) != LBM_OK) return st;
  CK(lbm_ref_macro(C, C->f[C->cur], C->d_fields, C->d_aux, &C->launches));
  size_t n = n_nodes(C), rs = real_size(C->precision);
  double *outs[3] = {rho, psi, U};
  void *host = nullptr;
  if (rho || psi || U) {
    host = malloc(3 * n * rs);
    if (!host) return LBM_ENOMEM;
    cudaError_t e = cudaMemcpyAsync(host, C->d_fields, 3 * n * rs, cudaMemcpyDeviceToHost, C->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(C->stream);
    if (e != cudaSuccess) { free(host); C->status = LBM_ECUDA; return LBM_ECUDA; }
    for (int k = 0; k < 3; ++k) {
      if (!outs[k]) continue;
      for (size_t i = 0; i < n; ++i)
        outs[k][i] = rs == 8 ? ((double *)host)[k * n + i] : (double)((float *)host)[k * n + i];
    }
    free(host);
  }
  double *o7[5] = {Fx, Fy, Qxx, Qyy, Qxy};
  for (int k = 0; k < 5; ++k)
    if (o7[k]) CK(cudaMemcpyAsync(o7[k], C->d_aux + (2 + k) * n, n * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return LBM_OK;
}

int lbm_get_u(lbm_ctx *C, double *ux, double *uy) {
  if (!C) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  int st = compute_fields(C);
  if (st) return st;
  if ((st = ensure_aux(C)) != LBM_OK) return st;
  CK(lbm_ref_macro(C, C->f[C->cur], C->d_fields, C->d_aux, &C->launches));
  size_t n = n_nodes(C);
  if (ux) CK(cudaMemcpyAsync(ux, C->d_aux, n * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  if (uy) CK(cudaMemcpyAsync(uy, C->d_aux + n, n * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return LBM_OK;
}

int lbm_get_f(lbm_ctx *C, double *f) {
  if (!C || !f) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  size_t cnt = 9 * n_nodes(C);
  if (C->precision == 64) {
    CK(cudaMemcpyAsync(f, C->f[C->cur], cnt * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    return LBM_OK;
  }
  float *tmp = (float *)malloc(cnt * sizeof(float));
  if (!tmp) return LBM_ENOMEM;
  cudaError_t e = cudaMemcpyAsync(tmp, C->f[C->cur], cnt * sizeof(float), cudaMemcpyDeviceToHost, C->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(C->stream);
  if (e == cudaSuccess)
    for (size_t i = 0; i < cnt; ++i) f[i] = (double)tmp[i];
  free(tmp);
  CK(e);
  return LBM_OK;
}

int lbm_set_f(lbm_ctx *C, const double *f) {
  if (!C || !f) return LBM_EINVAL;
  if (C->status) return C->status;
  size_t cnt = 9 * n_nodes(C);
  if (C->precision == 64) {
    CK(cudaMemcpyAsync(C->f[C->cur], f, cnt * sizeof(double), cudaMemcpyHostToDevice, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    return LBM_OK;
  }
  float *tmp = (float *)malloc(cnt * sizeof(float));
  if (!tmp) return LBM_ENOMEM;
  for (size_t i = 0; i < cnt; ++i) tmp[i] = (float)f[i];
  cudaError_t e = cudaMemcpyAsync(C->f[C->cur], tmp, cnt * sizeof(float), cudaMemcpyHostToDevice, C->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(C->stream);
  free(tmp);
  CK(e);
  return LBM_OK;
}

int lbm_contact_angle(lbm_ctx *C, int wall, int x0, int x1, double *theta, double *H, double *L) {
  if (!C || (wall != 0 && wall != 1) || x0 < 0 || x1 > C->nx || x0 >= x1) return LBM_EINVAL;
  if (!C->walls) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  CK(lbm_rho64(C, C->f[C->cur], C->d_rho64, &C->launches));
  CK(lbm_angle(C, C->d_rho64, wall, x0, x1, C->rho_mid, C->d_res, &C->launches));
  double r[5];
  CK(cudaMemcpyAsync(r, C->d_res, sizeof(r), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  if (r[4] != 0.0) return LBM_ENOCONTACT;
  if (theta) *theta = r[0];
  if (H) *H = r[1];
  if (L) *L = r[2];
  return LBM_OK;
}

int lbm_mass(lbm_ctx *C, double *mass) {
  if (!C || !mass) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  CK(lbm_rho64(C, C->f[C->cur], C->d_rho64, &C->launches));
  CK(lbm_reduce_mass(C, C->d_rho64, C->d_red, C->red_len, C->d_res, &C->launches));
  CK(cudaMemcpyAsync(mass, C->d_res, sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return LBM_OK;
}

int lbm_max_speed(lbm_ctx *C, double *umax) {
  if (!C || !umax) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  int st = compute_fields(C);
  if (st) return st;
  if ((st = ensure_aux(C)) != LBM_OK) return st;
  CK(lbm_ref_macro(C, C->f[C->cur], C->d_fields, C->d_aux, &C->launches));
  size_t n = n_nodes(C);
  CK(lbm_reduce_max_speed(C, C->d_aux, C->d_aux + n, C->d_red, C->red_len, C->d_res, &C->launches));
  CK(cudaMemcpyAsync(umax, C->d_res, sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return LBM_OK;
}

// Checkpoint image: 4 x int64 header {magic, precision, nx*ny, steps} + state.
static const int64_t kMagic = 0x4c424d3253544154LL;

size_t lbm_state_bytes(lbm_ctx *C) {
  if (!C) return 0;
  return 4 * sizeof(int64_t) + 9 * n_nodes(C) * real_size(C->precision);
}

int lbm_save(lbm_ctx *C, void *host, size_t bytes) {
  if (!C || !host || bytes != lbm_state_bytes(C)) return LBM_EINVAL;
  if (C->status == LBM_ECUDA) return C->status;
  int64_t hdr[4] = {kMagic, C->precision, (int64_t)n_nodes(C), C->steps};
  memcpy(host, hdr, sizeof(hdr));
  CK(cudaMemcpyAsync((char *)host + sizeof(hdr), C->f[C->cur], bytes - sizeof(hdr), cudaMemcpyDeviceToHost,
                     C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return LBM_OK;
}

int lbm_load(lbm_ctx *C, const void *host, size_t bytes) {
  if (!C || !host || bytes != lbm_state_bytes(C)) return LBM_EINVAL;
  if (C->status) return C->status;
  int64_t hdr[4];
  memcpy(hdr, host, sizeof(hdr));
  if (hdr[0] != kMagic || hdr[1] != C->precision || hdr[2] != (int64_t)n_nodes(C)) return LBM_EINVAL;
  CK(cudaMemcpyAsync(C->f[C->cur], (const char *)host + sizeof(hdr), bytes - sizeof(hdr), cudaMemcpyHostToDevice,
                     C->stream));
  CK(cudaStreamSynchronize(C->stream));
  C->steps = hdr[3];
  return LBM_OK;
}

int lbm_get_info(lbm_ctx *C, lbm_info *info) {
  if (!C || !info) return LBM_EINVAL;
  memset(info, 0, sizeof(*info));
  info->nx = C->nx;
  info->ny = C->ny;
  info->walls = C->walls;
  info->precision = C->precision;
  info->kernel_in_use = C->kernel_in_use;
  info->wetting = C->params.wetting;
  info->T = C->T;
  info->tau = C->tau;
  info->rho_v = C->rho_v;
  info->rho_l = C->rho_l;
  info->rho_max = C->rho_max;
  info->rho_mid = C->rho_mid;
  info->tile_w = C->fused_ok ? C->tile_w : 0;
  info->tile_blocks = C->fused_ok ? C->tile_blocks : 0;
  info->tile_stages = C->fused_ok ? C->tile_stages : 0;
  info->steps_done = C->steps;
  return LBM_OK;
}

unsigned long long lbm_launch_count(lbm_ctx *C) { return C ? C->launches : 0ULL; }

int lbm_sync(lbm_ctx *C) {
  if (!C) return LBM_EINVAL;
  CK(cudaStreamSynchronize(C->stream));
  return LBM_OK;
}

void lbm_destroy(lbm_ctx *C) {
  if (!C) return;
  cudaStreamSynchronize(C->stream);
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < lbm_ctx::kMaxGraphs; ++k)
      if (C->step_graph[p][k]) cudaGraphExecDestroy(C->step_graph[p][k]);
  lbm_adjoint_free_tape(C);
  if (C->owns_state && C->state) cudaFree(C->state);
  if (C->d_coef) cudaFree(C->d_coef);
  if (C->d_dcoef) cudaFree(C->d_dcoef);
  if (C->d_flag) cudaFree(C->d_flag);
  if (C->d_rho64) cudaFree(C->d_rho64);
  if (C->xfer) {
    for (int c = 0; c < 8; ++c) cudaEventDestroy(C->xfer_ev[c]);
    cudaStreamDestroy(C->xfer);
  }
  if (C->d_fields) cudaFree(C->d_fields);
  if (C->d_aux) cudaFree(C->d_aux);
  if (C->d_red) cudaFree(C->d_red);
  if (C->d_res) cudaFree(C->d_res);
  cudaGetLastError();
  delete C;
}

}  // extern "C"
