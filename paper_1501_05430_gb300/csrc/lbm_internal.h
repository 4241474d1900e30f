// lbm_internal.h -- private declarations shared by the liblbm translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/lbm.h"

// NVTX range over a scope (the library's entry points), so that a profiler
// timeline shows which call launched which kernels; free without a tool.
struct LbmRange {
  explicit LbmRange(const char *name) { nvtxRangePushA(name); }
  ~LbmRange() { nvtxRangePop(); }
  LbmRange(const LbmRange &) = delete;
  LbmRange &operator=(const LbmRange &) = delete;
};

// Device-side model constants, passed by value to every kernel.
// The EOS and model parameters are kept in double; kernels of the float
// instantiation convert them once per thread.
struct lbm_dev_params {
  int nx, ny;
  int walls;      // 1: rows 0 and ny-1 solid; 0: periodic in y as well
  int eos_kind;
  double a, b, R, T;
  double thv, thm, thl, r1, r2;
  double A, kappa, Gw;
  double s[9];    // rates in moment order (rho, e, eps, jx, qx, jy, qy, pxx, pxy)
  int n_iter, wetting;
  double rho_max;     // instability bound; psi = U = 0 at and above it
  double ghost_max;   // upper clamp of the ghost densities (<= rho_max)
};

// Per-wall-node coefficients of Eqs. 19-21, computed on the host:
// c = sin(pi/2 - theta), cot = tan(pi/2 - theta); [0..nx) bottom, [nx..2nx) top.
struct lbm_wall_coeffs {
  const double *c;
  const double *cot;
};

struct lbm_ctx {
  int nx, ny, walls, precision;
  int kernel_req, kernel_in_use;
  lbm_eos eos;
  double T, tau;
  lbm_params params;
  lbm_dev_params dp;
  double rho_v, rho_l, rho_max, rho_mid, ghost_max;
  cudaStream_t stream;
  int owns_state;
  void *state;           // two [9][ny][nx] arrays, contiguous
  void *f[2];
  int cur;               // index of the array holding the current state
  long long steps;
  unsigned long long launches;
  int status;            // sticky failure
  // device scratch
  double *d_coef;        // 4*nx: c_bot, c_top, cot_bot, cot_top
  double *d_dcoef;       // 4*nx: their derivatives in theta (adjoint)
  struct lbm_tape *tape; // adjoint record (lbm_adjoint.cu); NULL when none
  int *d_flag;           // [0]: instability, [1]: timeout, [2]: lbm_set_rho input check
  double *d_rho64;       // nx*ny, measurement density
  cudaStream_t xfer;     // lbm_get_rho: copy stream and its chunk events (lazy; NULL until first needed)
  cudaEvent_t xfer_ev[8];
  void *d_fields;        // 3*nx*ny reals: rho, psi, U (reference kernels)
  double *d_aux;         // 7*nx*ny doubles for lbm_get_u / lbm_get_fields (lazy)
  double *d_red;         // reduction partials
  double *d_res;         // small results
  int red_len;
  // fused kernel plan
  int fused_ok, fused_unit;  // fused kernel usable; unit-rate specialisation
  int fused_cols;            // columns per thread of the fused kernel
  int tile_w, tile_blocks, tile_stages, fused_smem;
  unsigned char tmaps[4][128];   // CUtensorMap for f[0], f[1]: main box, halo box
  // lbm_step graphs, captured at the first lbm_step for both starting arrays:
  // graph_len[0] = graph_steps (even), then every power of two 2 <= 2^k below
  // it, largest first, so that any step count replays as whole graphs plus at
  // most one direct launch
  static constexpr int kMaxGraphs = 17;
  int ngraph, graphs_ready;
  int graph_len[kMaxGraphs];
  cudaGraphExec_t step_graph[2][kMaxGraphs];
};

// ---- lbm_ref.cu: unfused kernels in the canonical evaluation order --------
// All launchers return the cudaError_t of the launch and add the number of
// kernels launched to *launches.
cudaError_t lbm_ref_fields(const lbm_ctx *C, const void *f, void *fields, unsigned long long *launches);
cudaError_t lbm_ref_collide(const lbm_ctx *C, const void *fin, void *fout, const void *fields,
                            unsigned long long *launches);
cudaError_t lbm_ref_macro(const lbm_ctx *C, const void *f, const void *fields, double *out7,
                          unsigned long long *launches);
// f := f_eq(rho, 0) from device or mapped host densities; with bad != NULL,
// *bad |= 1 if a fluid-node density is not finite or not > 0 (bad zeroed by
// the caller; f is written all the same)
cudaError_t lbm_ref_set_rho(const lbm_ctx *C, const double *rho, void *f, int *bad, unsigned long long *launches);
cudaError_t lbm_ref_droplets(const lbm_ctx *C, int n, const double *drop, double width, double *rho,
                             unsigned long long *launches);

// ---- lbm_fused.cu: single-pass FP32 step ------------------------------------
int lbm_fused_plan(lbm_ctx *C);  // sets fused_ok, tile_*, tensor maps
cudaError_t lbm_fused_step(lbm_ctx *C, int src, unsigned long long *launches);
// The same step between any two state arrays of the context's shape (16-byte
// aligned): the adjoint's recorded forward and its segment replays.
cudaError_t lbm_fused_step_between(lbm_ctx *C, const void *src, void *dst, unsigned long long *launches);

// ---- lbm_adjoint.cu: discrete adjoint ---------------------------------------
void lbm_adjoint_free_tape(lbm_ctx *C);

// ---- lbm_measure.cu: reductions -------------------------------------------
cudaError_t lbm_rho64(const lbm_ctx *C, const void *f, double *rho, unsigned long long *launches);
// the same for rows [row0, row1) only (rho indexed like the whole field)
cudaError_t lbm_rho64_rows(const lbm_ctx *C, const void *f, double *rho, int row0, int row1,
                           unsigned long long *launches);
cudaError_t lbm_reduce_mass(const lbm_ctx *C, const double *rho, double *partial, int npart, double *res,
                            unsigned long long *launches);
cudaError_t lbm_reduce_max_speed(const lbm_ctx *C, const double *ux, const double *uy, double *partial,
                                 int npart, double *res, unsigned long long *launches);
cudaError_t lbm_angle(const lbm_ctx *C, const double *rho, int wall, int x0, int x1, double rho_mid, double *res,
                      unsigned long long *launches);
