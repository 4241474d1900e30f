/*
 * lbm.h -- C ABI of liblbm, a GB300 (sm_103a) implementation of the
 * single-component EOS-based pseudo-potential D2Q9 lattice Boltzmann method
 * with the geometric contact-angle wall rule of
 *   A. Hu, L. Li, R. Uddin, "Contact Angle Adjustment in Equation of States
 *   Based Pseudo-Potential Model", arXiv:1501.05430,
 * and the Martys-Chen fluid-solid force (Eq. 14) as the compared variant.
 *
 * One timestep (lbm_step) is, per fluid node and in this order:
 *   rho = sum_a f_a                          (Eq. 1, zeroth moment)
 *   U = p(rho) - rho/3, psi = sqrt(-2U)      (Eq. 10 with c = 1, G = -1;
 *                                             p from Eq. 11 or Carnahan-Starling)
 *   ghost-row densities on the solid rows    (Eqs. 19-21, geometric wetting)
 *   F = hybrid interaction force             (Eq. 9; + Eq. 14 for Martys-Chen)
 *   Q tensor and source C                    (Eqs. 16-17)
 *   MRT collision with forcing               (Eqs. 2, 4-6, 15)
 *   streaming with half-way bounce-back      (left side of Eq. 1)
 *
 * Conventions shared by every entry point:
 *  - Status: every int-returning call returns LBM_OK (0) or a negative LBM_E*
 *    code; lbm_strerror() names it.  After LBM_EUNSTABLE, LBM_ECUDA or
 *    LBM_ETIMEOUT a context is failed for good: later calls on it return the
 *    same code.
 *  - Grid: nx columns (x, periodic) by ny rows (y).  Host arrays of node
 *    values are row-major [ny][nx] (index y*nx + x) and are double.  The
 *    distribution functions are [9][ny][nx] with the D2Q9 order
 *    e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1)
 *    e7=(-1,-1) e8=(1,-1).
 *  - Walls: either no solid node at all (fully periodic box) or exactly the
 *    two full rows y = 0 and y = ny-1 (flat walls, the only geometry for which
 *    Eqs. 19-21 are defined).  Those rows hold no fluid; on them the library
 *    keeps the ghost densities of Eqs. 19-21.
 *  - Ownership: inputs are copied during the call; the caller keeps them.
 *    Outputs go to caller-allocated buffers.  A context owns the device
 *    memory it allocates; lbm_create_with_buffer lets the caller own the
 *    distribution-function storage instead (e.g. a PyTorch tensor).
 *  - Streams: all device work of a context is ordered on the stream given to
 *    lbm_create (NULL = the legacy default stream).  Getters synchronise that
 *    stream before they return.  A context is not thread-safe.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define LBM_OK 0
#define LBM_EINVAL (-1)       /* invalid argument (sizes, tau <= 1/2, T >= T_c, ...) */
#define LBM_ENOMEM (-2)       /* device or host allocation failed */
#define LBM_ECUDA (-3)        /* a CUDA call failed (no device, launch error, ...) */
#define LBM_EUNSTABLE (-4)    /* a fluid density became NaN, <= 0 or > rho_max */
#define LBM_EUNSUPPORTED (-5) /* valid request this build does not support (wall shape, ...) */
#define LBM_ETIMEOUT (-6)     /* a bounded device-side wait gave up */
#define LBM_ENOCONTACT (-7)   /* angle measurement found no contact line in the region */

/* ---- enumerations ----------------------------------------------------- */
enum { LBM_EOS_CARNAHAN_STARLING = 0, LBM_EOS_PIECEWISE = 1 };
enum { LBM_WET_GEOMETRIC = 0, LBM_WET_MARTYS_CHEN = 1 };
/* Kernel choice for lbm_step: AUTO takes the fused single-pass kernel when the
 * context qualifies (FP32, nx % 4 == 0) and the unfused reference kernels
 * otherwise; REFERENCE forces the unfused kernels (the path that follows the
 * canonical evaluation order, bit-identical to an FP64 CPU evaluation in the
 * same order); FUSED demands the fused kernel (LBM_EUNSUPPORTED if the
 * context does not qualify). */
enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_REFERENCE = 1, LBM_KERNEL_FUSED = 2 };

/* Equation of state.
 *  kind = LBM_EOS_CARNAHAN_STARLING: p = rho R T (1+e+e^2-e^3)/(1-e)^3 - a rho^2,
 *         e = b rho / 4 (uses a, b, R).
 *  kind = LBM_EOS_PIECEWISE: Eq. 11, the three linear branches with slopes
 *         theta_v, theta_m (< 0), theta_l and breakpoints rho1 < rho2 (Table 1
 *         gives the paper's values; T is ignored). */
typedef struct lbm_eos {
  int kind;
  double a, b, R;
  double theta_v, theta_m, theta_l, rho1, rho2;
} lbm_eos;

/* Model and run parameters.  Fill with lbm_params_default() first. */
typedef struct lbm_params {
  double A;          /* Eq. 9 mixing parameter (Sec. 3.1: -0.6) */
  double kappa;      /* Eq. 17 surface-tension parameter (Sec. 3.1: 0.5) */
  double G_w;        /* Eq. 14 fluid-solid strength (Martys-Chen only) */
  int n_iter;        /* right-hand-side evaluations of Eq. 21 (Sec. 4.2.1: 4);
                        0 = Eq. 19 alone */
  int wetting;       /* LBM_WET_GEOMETRIC or LBM_WET_MARTYS_CHEN */
  int precision;     /* 32 (float state) or 64 (double state) */
  int kernel;        /* LBM_KERNEL_* */
  double s_e, s_eps, s_j, s_q, s_nu; /* Eq. 2 rates for e, eps, j, q, nu;
                        0 means 1/tau.  s_rho is irrelevant (rho is conserved). */
  int check_every;   /* read the device stability flag every this many steps
                        inside lbm_step (0 = only when lbm_status is called) */
  double rho_mid;    /* density of the contour used by lbm_contact_angle;
                        0 means (rho_v + rho_l)/2 of the context */
  double rho_max;    /* instability bound; 0 means the smallest rho > rho_l
                        with p(rho) = rho/3 (psi^2 >= 0 below it) */
  double rho_ghost_max; /* upper clamp of the Eqs. 19-21 ghost densities
                        (lower clamp 0); 0 means rho_max */
  int graph_steps;   /* when the context has a non-NULL stream, lbm_step
                        replays captured CUDA graphs: of this many steps
                        (rounded up to even) while at least that many remain,
                        then of the powers of two below it, largest first, so
                        that at most one step of a call runs as a direct launch.
                        All of them are captured by the first lbm_step of two or
                        more steps, for both state arrays (call it before any
                        capture of the context's stream).  0 = one launch
                        sequence per step.  Results are the same either way. */
} lbm_params;

/* Values of a created context (for bookkeeping and tests). */
typedef struct lbm_info {
  int nx, ny, walls, precision, kernel_in_use, wetting;
  double T, tau, rho_v, rho_l, rho_max, rho_mid;
  int tile_w, tile_blocks, tile_stages;  /* fused-kernel launch shape (0 if unused) */
  long long steps_done;
} lbm_info;

typedef struct lbm_ctx lbm_ctx;

/* Human-readable name of a status code (static string, never NULL). */
const char *lbm_strerror(int status);

/* Defaults of Sec. 3.1: A = -0.6, kappa = 0.5, G_w = 0, n_iter = 4, geometric
 * wetting, FP32, AUTO kernel, all rates 1/tau, check_every = 100, graph_steps = 64,
 * rho_mid = rho_max = 0 (derived).  LBM_EINVAL if p is NULL. */
int lbm_params_default(lbm_params *p);

/* Carnahan-Starling critical point: T_c and rho_c where dp/drho and
 * d2p/drho2 both vanish.  LBM_EUNSUPPORTED for the piecewise EOS (Eq. 11 has
 * no critical point), LBM_EINVAL for NULL pointers or a, b, R <= 0. */
int lbm_eos_critical(const lbm_eos *eos, double *Tc, double *rho_c);

/* Coexistence densities rho_v < rho_l.  Carnahan-Starling: the Maxwell
 * (equal-area) construction at temperature T (0 < T < T_c, else LBM_EINVAL).
 * Piecewise: the densities that Eqs. 12-13 tie to the given breakpoints (T
 * ignored).  LBM_EINVAL when no solution exists. */
int lbm_coexistence(const lbm_eos *eos, double T, double *rho_v, double *rho_l);

/* The density bounds lbm_create derives for a context whose params.rho_max
 * and params.rho_mid are 0, computed on the host (no device call):
 *  rho_v, rho_l: the coexistence densities of lbm_coexistence;
 *  rho_max:      the smallest rho > rho_l with p(rho) = rho/3, i.e. where
 *                psi^2 = 2 (rho/3 - p) of Eq. 10 (c = 1, G = -1) returns to 0
 *                (Brent's method on the Carnahan-Starling branch; the linear
 *                liquid branch of Eq. 11 in closed form, DBL_MAX when its slope
 *                theta_l is <= 1/3 and psi^2 stays positive).  It is the upper
 *                clamp of the Eqs. 19-21 ghost densities and the instability
 *                bound of lbm_step;
 *  rho_mid:      (rho_v + rho_l)/2, the contour of lbm_contact_angle.
 * Any output pointer may be NULL.  LBM_EINVAL as for lbm_coexistence. */
int lbm_eos_bounds(const lbm_eos *eos, double T, double *rho_v, double *rho_l, double *rho_max,
                   double *rho_mid);

/* Create a context on the current CUDA device.
 *  nx >= 4, ny >= 5; tau > 1/2 (viscous rate s_nu = 1/tau unless set).
 *  eos, T: equation of state and absolute temperature (for Carnahan-Starling
 *          0 < T < T_c; multiply T/T_c by lbm_eos_critical()).
 *  theta:  NULL (90 degrees everywhere) or nx*ny contact angles in radians,
 *          read only on the two solid rows, each in (0, pi).  The geometric
 *          rule uses sin(pi/2 - theta) (Eqs. 20-21) or tan(pi/2 - theta)
 *          (Eq. 19, n_iter = 0), evaluated on the host.
 *  wall_mask: NULL (no walls) or nx*ny bytes, 1 = solid; must be empty or
 *          exactly the rows y = 0 and y = ny-1 (else LBM_EUNSUPPORTED).
 *  params: NULL for the defaults.
 *  stream: a cudaStream_t (NULL = legacy default stream).
 * The distribution functions start at zero; set them with lbm_set_rho,
 * lbm_init_droplets, lbm_set_f or lbm_load.  Returns LBM_ENOMEM when the
 * device memory (2 * 9 * nx * ny reals plus O(nx*ny) scratch) is not
 * available. */
int lbm_create(int nx, int ny, const lbm_eos *eos, double T, double tau, const double *theta,
               const uint8_t *wall_mask, const lbm_params *params, void *stream, lbm_ctx **out);

/* Bytes of caller-owned device storage that lbm_create_with_buffer needs:
 * two copies of the 9*nx*ny distribution functions in the given precision. */
size_t lbm_required_state_bytes(int nx, int ny, int precision);

/* As lbm_create, but the two distribution-function arrays live in device
 * memory the caller owns (at least lbm_required_state_bytes bytes, 256-byte
 * aligned, valid until lbm_destroy).  LBM_EINVAL if state is NULL, too small or
 * misaligned. */
int lbm_create_with_buffer(int nx, int ny, const lbm_eos *eos, double T, double tau,
                           const double *theta, const uint8_t *wall_mask,
                           const lbm_params *params, void *stream, void *state,
                           size_t state_bytes, lbm_ctx **out);

/* f := f_eq(rho, u = 0) (Eq. 4 equilibria mapped back by M^-1) at every fluid
 * node, from nx*ny host densities (wall-row entries ignored).  Densities must
 * be finite and > 0 at fluid nodes (else LBM_EINVAL, and the state is left as
 * it was).  Pinned (page-locked) host memory is read by the device in place;
 * other host memory is first copied to the device.  Synchronises. */
int lbm_set_rho(lbm_ctx *ctx, const double *rho);

/* Initial droplets built on the device: rho = max over droplets k of
 * (rho_l + rho_v)/2 - (rho_l - rho_v)/2 tanh(2 (r_k - R_k)/width), r_k the
 * distance (periodic in x) to (xc[k], 1) for wall[k] = 0 (bottom) or
 * (xc[k], ny-2) for wall[k] = 1 (top); then f := f_eq(rho, 0).  With n = 0 the
 * domain is filled with vapour.  rho_v, rho_l are the context's coexistence
 * densities. */
int lbm_init_droplets(lbm_ctx *ctx, int n, const double *xc, const double *radius, const int *wall,
                      double width);

/* Advance nsteps timesteps (nsteps >= 0).  Work is queued on the context's
 * stream; the call returns once it is queued, except when a stability check
 * falls due (params.check_every), which synchronises.  LBM_EUNSTABLE when the
 * check finds a fluid density NaN, <= 0 or > rho_max. */
int lbm_step(lbm_ctx *ctx, int nsteps);

/* Synchronise and read the device stability flag: LBM_OK or LBM_EUNSTABLE. */
int lbm_status(lbm_ctx *ctx);

/* Density at every node (nx*ny doubles): sum_a f_a (summed in double, left
 * to right) at fluid nodes, 0 on the solid rows.  The ghost densities that the
 * wall rule gives the solid rows for the current state come from
 * lbm_get_fields.  Synchronises. */
int lbm_get_rho(lbm_ctx *ctx, double *rho);

/* Velocity u = (sum_a f_a e_a + F/2)/rho (the half-force shifted velocity of
 * Eqs. 4 and 6) at fluid nodes, 0 on solid rows; nx*ny doubles each; either
 * pointer may be NULL. */
int lbm_get_u(lbm_ctx *ctx, double *ux, double *uy);

/* Copy of the distribution functions, 9*nx*ny doubles in [9][ny][nx] order
 * (solid rows read as 0).  lbm_set_f writes them (rounded to the context's
 * precision). */
int lbm_get_f(lbm_ctx *ctx, double *f);
int lbm_set_f(lbm_ctx *ctx, const double *f);

/* Fields of the current state as the next step will use them, each nx*ny
 * doubles or NULL: rho, psi, U (with the ghost values on the solid rows), the
 * interaction force (Eq. 9 [+ Eq. 14]) and the Eq. 17 tensor at fluid nodes. */
int lbm_get_fields(lbm_ctx *ctx, double *rho, double *psi, double *U, double *Fx, double *Fy,
                   double *Qxx, double *Qyy, double *Qxy);

/* Apparent contact angle of the droplet sitting on `wall` (0 = bottom,
 * 1 = top) within columns [x0, x1) (0 <= x0 < x1 <= nx).  The paper reports
 * measured angles without a procedure; this one is:
 *  - the centre column xc maximises sum_y rho over the wall's half of the
 *    domain (bottom: rows 1 .. ny/2-1, top: ny/2 .. ny-2; ties: lowest x);
 *  - L: distance between the linearly interpolated rho_mid crossings that
 *    bound the liquid run of the boundary row (1 or ny-2) containing xc;
 *  - H: distance from the boundary row to the interpolated rho_mid crossing
 *    found walking away from the wall along xc;
 *  - theta = 2 atan2(2H, L), exact for a circular cap cut by the boundary row.
 * Outputs may be NULL.  LBM_ENOCONTACT if the boundary row is not liquid at xc
 * or a liquid run reaches the region edge / the domain middle. */
int lbm_contact_angle(lbm_ctx *ctx, int wall, int x0, int x1, double *theta, double *H, double *L);

/* Total mass sum rho over fluid nodes (FP64 accumulation, fixed order). */
int lbm_mass(lbm_ctx *ctx, double *mass);

/* Largest |u| over fluid nodes (the spurious-velocity measure). */
int lbm_max_speed(lbm_ctx *ctx, double *umax);

/* Checkpoint: the raw state (distribution functions in the context's
 * precision plus the step counter) as an opaque byte image of
 * lbm_state_bytes() bytes; lbm_load restores it bit for bit.  LBM_EINVAL on a
 * size mismatch. */
size_t lbm_state_bytes(lbm_ctx *ctx);
int lbm_save(lbm_ctx *ctx, void *host, size_t bytes);
int lbm_load(lbm_ctx *ctx, const void *host, size_t bytes);

/* Context facts; number of kernels this context has launched so far. */
int lbm_get_info(lbm_ctx *ctx, lbm_info *info);
unsigned long long lbm_launch_count(lbm_ctx *ctx);

/* Block until all queued work of the context is done (LBM_ECUDA on error). */
int lbm_sync(lbm_ctx *ctx);

/* Free everything the context owns (not a caller-owned state buffer). */
void lbm_destroy(lbm_ctx *ctx);

/* ---- allocation-free entry point ------------------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory: code that runs under another framework's allocator
 * (which must own every device byte), embedders whose device allocation is
 * disabled or budgeted to zero, and real-time loops where cudaMalloc's implicit
 * synchronisation is not allowed.  It computes what lbm_mass computes -- the
 * sum of rho = sum_a f_a over the fluid nodes -- directly from a
 * distribution-function array the caller owns.
 *
 *  f:         device pointer, [9][ny][nx] floats (precision 32) or doubles (64);
 *             rows 0 and ny-1 are skipped when walls = 1.
 *  mass:      device pointer to one double that receives the result.
 *  stream:    cudaStream_t the two kernels are queued on (NULL = legacy default);
 *             the call returns once they are queued.
 * Scratch: the block partial sums live in a fixed device array of
 * LBM_NOALLOC_MAX_PARTIALS doubles (8 KiB), compiled into the library and held
 * by every GPU that loads it until the process exits.  Every call on a device
 * shares that array; it is fully rewritten by each call, so nothing carries
 * over, but calls that overlap on the GPU (different streams) race on it.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  No device memory is allocated or freed.
 * Errors: LBM_EINVAL for NULL pointers, precision not 32/64, walls not 0/1,
 * too few rows, or nx * ny > LBM_NOALLOC_MAX_NODES; LBM_ECUDA if the lookup or
 * a launch fails. */
#define LBM_NOALLOC_MAX_PARTIALS 1024
#define LBM_NOALLOC_MAX_NODES (1 << 28)
int lbm_mass_noalloc(const void *f, int nx, int ny, int precision, int walls, double *mass, void *stream);

/* ---- discrete adjoint ---------------------------------------------------- *
 * Gradients of a function of the final density with respect to the wall
 * angles (theta per wall node, through sin(pi/2 - theta) of Eqs. 20-21 or
 * tan(pi/2 - theta) of Eq. 19) and the EOS temperature T, by the reverse-time
 * (adjoint) of the step, with the initial state held fixed.  The recorded
 * forward and the segment replays of the backward sweep run the context's own
 * step kernel, so the recorded trajectory is the one lbm_step produces: at
 * precision 64 the canonical reference kernels (bit-identical to an FP64
 * evaluation of the step in that order), at precision 32 the fused kernel when
 * the context uses it.  The reverse sweep transposes the canonical step at each
 * recorded state, so in FP32 the gradient is the canonical step's transpose
 * evaluated along the fused kernel's trajectory (the two steps differ by
 * rounding only).  Kinks: d sqrt(s)/ds = 0 at s = 0, d|a|/da = 0 at a = 0, a
 * clamped ghost density passes no gradient.
 *
 * lbm_adjoint_record: advance the context by nsteps from its current state,
 * keeping the state every checkpoint_every steps on the device (the tape:
 * ceil(nsteps / checkpoint_every) + checkpoint_every states plus O(nx ny)
 * scratch).  Replaces an earlier tape.  Returns LBM_OK, LBM_EUNSTABLE,
 * LBM_EINVAL (nsteps or checkpoint_every < 1), LBM_EUNSUPPORTED
 * (n_iter > 64), LBM_ENOMEM, LBM_ECUDA.
 *
 * lbm_adjoint_backward: given dL/drho at the final (recorded) time,
 * dl_drho[ny][nx] (host, values on the solid rows ignored), walk the tape back
 * and write dL/dtheta to dl_dtheta[2][nx] (row 0: bottom wall, row 1: top
 * wall; zero for Martys-Chen and periodic boxes), dL/dT to *dl_dT, and
 * dL/df at the recorded start to dl_df0[9][ny][nx]; each output may be NULL.
 * The tape is kept, so backward may run again with another dl_drho.  The
 * context's state is not changed.  LBM_EINVAL without a tape. */
int lbm_adjoint_record(lbm_ctx *ctx, int nsteps, int checkpoint_every);
int lbm_adjoint_backward(lbm_ctx *ctx, const double *dl_drho, double *dl_dtheta, double *dl_dT, double *dl_df0);
/* Free the tape (lbm_destroy does it too). */
int lbm_adjoint_release(lbm_ctx *ctx);

/* ---- batched sweep ----------------------------------------------------- *
 * Many independent droplet instances -- each with its own grid size, EOS
 * temperature, relaxation rates and wall-angle field -- advanced together by
 * one persistent kernel per launch (the contact-angle x density-ratio sweeps
 * of Secs. 3.1 and 4.2 run as one job instead of one solver per case).
 *
 * Every instance has solid rows at y = 0 and y = ny-1, precision 32, and
 * nx a multiple of 4 and at most 512.  Its state lives in one device pool
 * owned by the batch.
 * Each instance is cut into work items (bands of whole fluid rows); one launch
 * advances every instance by steps_per_launch steps, and the CTAs that share
 * an instance meet at a per-instance barrier between its steps (no barrier
 * across instances).  Per node the arithmetic is that of lbm_step's FP32
 * fused kernel, so an instance gives the same bits as a lone context that
 * runs the fused kernel. */
typedef struct lbm_batch lbm_batch;

typedef struct {
  int nx, ny;            /* grid; rows 0 and ny-1 solid; nx % 4 == 0 */
  lbm_eos eos;
  double T, tau;         /* as for lbm_create */
  const double *theta;   /* [ny][nx] radians (rows 0 and ny-1 read) or NULL = pi/2 */
  lbm_params params;     /* precision must be 32; kernel is ignored */
} lbm_instance_desc;

/* Launch shape.  Zero fields take the defaults in brackets. */
typedef struct {
  int threads;           /* 256 [default]: every instance in one launch of 256-thread
                            CTAs; 128: the instances up to 256 wide in a launch of their
                            own with 128-thread CTAs (a 256-wide row then keeps every
                            thread busy), the wider ones in 256-thread CTAs.  Thread
                            t < nx/2 owns columns t and t + nx/2 of a row */
  int ctas_per_sm;       /* cap on resident CTAs per SM, in 256-thread CTAs (twice as
                            many 128-thread ones) [occupancy maximum] */
  int stages;            /* shared memory of the copy ring, in rows of the widest
                            instance, 3..6 [4]; each work item repacks it into
                            min(16, stages x widest / nx) rows of its own width */
  int band_rows[4];      /* fluid rows per work item for nx in (0,128], (128,256],
                            (256,384], (384, ...) [32 each] */
  int steps_per_launch;  /* steps advanced by one launch [16] */
  int graph_launches;    /* launches captured per CUDA graph and replayed [0 = no graph];
                            used when graph_launches * steps_per_launch is even and the
                            batch has a non-NULL stream */
  double wait_seconds;   /* bound on every barrier wait [2 s], at most 60 */
  int hold_instance;     /* testing aid, -1 normally: the given instance's first work
                            item never arrives at its barrier, so the other items of
                            that instance wait until wait_seconds runs out */
} lbm_batch_config;

int lbm_batch_config_default(lbm_batch_config *cfg);

/* Create n instances.  inst[i].theta is copied.  cfg may be NULL (defaults).
 * stream: cudaStream_t for all the batch's work (NULL = legacy default; CUDA
 * graphs need a non-NULL stream).  Each instance starts with f = 0; set it
 * with lbm_set_rho / lbm_init_droplets / lbm_set_f on lbm_batch_instance().
 * Errors: LBM_EINVAL (n < 1, an instance's sizes, precision or parameters),
 * LBM_EUNSUPPORTED (an instance wider than 512), LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_create(int n, const lbm_instance_desc *inst, const lbm_batch_config *cfg, void *stream,
                     lbm_batch **out);
int lbm_batch_size(const lbm_batch *b);

/* The context of instance i, owned by the batch (never lbm_destroy it).  Every
 * lbm_* call works on it (setters, getters, measurements, checkpoints, even
 * lbm_step for that instance alone); it shares the batch's stream.  NULL if i
 * is out of range. */
lbm_ctx *lbm_batch_instance(lbm_batch *b, int i);

/* Advance every instance by nsteps.  Returns LBM_OK, LBM_ETIMEOUT if a
 * barrier wait ran out (the batch is then failed for good; the instances
 * concerned report LBM_ETIMEOUT), or LBM_ECUDA.  An instance that becomes
 * unstable is flagged (its lbm_status() returns LBM_EUNSTABLE) and left
 * frozen while the others go on; the call still returns LBM_OK.
 * Synchronises the stream before it returns. */
int lbm_batch_step(lbm_batch *b, int nsteps);

/* Batch status (LBM_OK or LBM_ETIMEOUT); inst_status[n] (may be NULL)
 * receives each instance's status. */
int lbm_batch_status(lbm_batch *b, int *inst_status);

/* Apparent contact angle of every instance on one wall over its full width
 * (as lbm_contact_angle).  theta[n] required; H, L, status may be NULL.
 * status[i] = LBM_OK or LBM_ENOCONTACT (theta[i] = NaN then). */
int lbm_batch_contact_angles(lbm_batch *b, int wall, double *theta, double *H, double *L, int *status);

/* Pick the launch shape by timing trial_steps steps of candidate
 * configurations on a copy of the current state (threads x stages, then the
 * band height of each size class present, then steps_per_launch), install the
 * fastest and put the state back.  best (may be NULL) receives it.
 * Needs one extra state-sized device allocation while it runs. */
int lbm_batch_autotune(lbm_batch *b, int trial_steps, lbm_batch_config *best);

int lbm_batch_get_config(const lbm_batch *b, lbm_batch_config *cfg);
/* Install a launch shape (validated as in lbm_batch_create). */
int lbm_batch_set_config(lbm_batch *b, const lbm_batch_config *cfg);
/* Plan of the current shape: CTAs per launch, work items, dynamic shared
 * memory per CTA, resident CTAs per SM.  With threads = 128 and instances on
 * both sides of 256 columns, CTAs and items are summed over the two launches,
 * the shared memory is the larger one and the CTAs per SM are the 256-thread
 * launch's.  Any pointer may be NULL. */
int lbm_batch_get_plan(const lbm_batch *b, int *grid, int *items, int *smem_bytes, int *ctas_per_sm);
/* Kernel launches issued by lbm_batch_step so far (graph replays included). */
unsigned long long lbm_batch_launch_count(const lbm_batch *b);
/* Fluid-node updates the batched kernel has computed for each instance since
 * lbm_batch_create, into updates[lbm_batch_size(b)] (host): one per fluid node
 * and step while the instance is stable.  An instance flagged unstable is
 * frozen -- its remaining steps are skipped, not computed -- so its count
 * stops at (about) the step where the flag was raised; lbm_batch_autotune's
 * trials are not counted.  Throughput = the change of the sum over a timed
 * interval / its duration.  Synchronises the batch's stream. */
int lbm_batch_node_updates(lbm_batch *b, unsigned long long *updates);
void lbm_batch_destroy(lbm_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
