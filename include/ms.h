/*
 * ms.h -- C ABI of the GB300 (sm_103a) Ti-6Al-4V microstructure point solver.
 *
 * The library advances the phenomenological phase model of Proell et al.,
 * arXiv 2402.17580 (beta, stable alpha_s, martensitic alpha_m) at every point
 * of a part, one explicit time step at a time:
 *
 *   m = (X_as, X_am)                                  Sec. 3.1 (state vector)
 *   m~ = m^n + dt * m_diff(T^n, m^n)                  Sec. 3.1, eq:explicit_integration
 *   m^{n+1} = g(T^{n+1}, m~)                          Sec. 3.1, eq:explicit_correction
 *   X_beta = X_sol(T) - X_as - X_am, X_sol = 1 - g(T) Sec. 3.1, eq:time_integration_beta_postprocess
 *
 * with the rates of Sec. 2.2 (eq:beta_to_alpha_s, eq:alpha_m_to_alpha_s,
 * eq:alpha_s_to_beta), the instantaneous martensite terms
 * (eq:inst_martensite_formation, eq:inst_martensite_dissolution), the alpha_s
 * regularisation and the analytical initiation of Appendix A
 * (eq:analytical_solution_beta).  Points are independent (Sec. 3: no
 * communication), so the library is a data-parallel point solver.
 *
 * Conventions for every entry point:
 *  - return value: MS_OK (0) or a negative MS_ERR_* code; no exceptions cross
 *    the ABI; ms_strerror() gives a message, ms_last_error() the detail of the
 *    last failure on the calling thread.
 *  - host arrays are owned by the caller and are only read / written during
 *    the call (the library copies).  Device pointers (flag MS_PTR_DEVICE) are
 *    borrowed for the call only and never freed by the library.
 *  - a context owns all device memory it allocates and its CUDA stream (or
 *    uses the stream given to ms_set_stream, which it never destroys).
 *  - calls on one context must not overlap (one host thread at a time);
 *    different contexts are independent.
 *  - points are in natural order: specimen by specimen, and inside a
 *    specimen's grid i (x) fastest, then j (y), then k (z).
 */
#ifndef MS_H
#define MS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define MS_OK                   0
#define MS_ERR_INVALID_ARG     -1  /* bad pointer, size, dt, fraction or parameter      */
#define MS_ERR_OOM             -2  /* device or host allocation failed                   */
#define MS_ERR_CUDA            -3  /* a CUDA runtime call failed (see ms_last_error)     */
#define MS_ERR_DEVICE_TIMEOUT  -4  /* a bounded device wait gave up                      */
#define MS_ERR_NONFINITE       -5  /* a fraction became NaN or infinite on the device    */
#define MS_ERR_STATE           -6  /* call out of order (e.g. run_track without points)  */
#define MS_ERR_UNSUPPORTED     -7  /* option not available in this build or context     */

/* precision of the stored fractions (the arithmetic of the rates is FP32) */
#define MS_F32      0  /* fractions stored and accumulated in FP32                       */
#define MS_F64ACC   1  /* fractions stored and accumulated in FP64                       */
#define MS_KAHAN    2  /* FP32 fractions with a compensation term (two floats each)      */
#define MS_F64      3  /* everything in FP64: temperatures, rates, fractions (the GPU
                          spot-check path; FP64 exp2 / log2 instead of the SFU)        */

/* flags for ms_step */
#define MS_PTR_DEVICE  1  /* T_prev / T_new are device pointers (else host pointers)    */

/* bits of ms_params.flags */
#define MS_FLAG_TIME_KERNELS 1  /* time every hot-kernel launch with CUDA events on the
                                   context stream (read back by ms_stats)            */
#define MS_FLAG_GRAPH        2  /* ms_run_track captures its launch sequence (source
                                   table, active set, persistent hot kernel per chunk
                                   of S steps) into a CUDA graph on first use and
                                   replays it when called again with the same start
                                   step, step count and dt (e.g. after ms_fill_state) */
#define MS_FLAG_FMA_TRANSCENDENTALS 8  /* MS_F32: the hot kernels (ms_run_track,
                                   ms_step) evaluate exp2 and log2 as polynomials on
                                   the FMA pipe (IEEE-754 range reduction, a fitted
                                   polynomial by Estrin's scheme: the paper's fast
                                   transcendentals, Sec. 3.3) instead of the SFU;
                                   relative error about 1e-7, like the SFU's.  Off
                                   by default: on GB300 the SFU path measured
                                   faster (the kernels are bound by instruction
                                   issue, which the polynomials add to) */
#define MS_FLAG_COUNT_OPS    4  /* the explicit hot kernel counts the phase model's
                                   transcendentals on the branch each point takes
                                   (ms_stats model_sfu_ex2 / model_sfu_slow); off by
                                   default: the counting costs instructions in the
                                   kernel, so timed runs leave it off and the counts
                                   come from a separate run of the same work       */

/* time integration of the diffusive rates (ms_params.integrator), Sec. 3 */
#define MS_EXPLICIT 0  /* forward Euler + correction g (eq:explicit_integration) */
#define MS_IMPLICIT 1  /* Crank-Nicolson + g, fixed-point iteration with a WRMS
                          stop, substeps of at most dt_sub with the temperature
                          linear in time (eq:implicit_integration and
                          eq:implicit_fp_iteration).  The iteration starts from
                          g(T^{n+1}, m^n) as the paper's implicit algorithm
                          does; w_j = 1 / (eps_abs + |m_{i+1,j}| eps_rel); App. A
                          initiation steps take the closed form as in the
                          explicit scheme.  MS_F32 and MS_F64 only; not with
                          an attached surrogate or ms_run_track_noalloc.    */

/* ---------------------------------------------------------------- params */
/* Model constants and options.  ms_params_default() fills the paper's values:
 * Table 1/2 (T_s, T_l, T_as_start, T_as_end, T_am_start, T_inf, k_alpha_eq,
 * k_am_eq), Table 3 (c_as, c_b, k1, k2, k3, f), T_reg = 100 K (Sec. 2.2) and
 * the App. A exit threshold 1e-15.  Readings where the paper is ambiguous:
 *   martensite_literal  0: X_am <- max(X_am, X_am^eq) below T_am,start (default),
 *                       1: X_am <- X_am^eq (eq:inst_martensite_formation literally)
 *   init_ba_steps       0: one analytical beta -> alpha_s step when X_as == 0,
 *                       1: keep the analytical step until the App. A exit rule
 *   init_exit_floor     App. A initiation of alpha_s -> beta ends when
 *                       X~_beta * dt > init_exit AND X~_beta >= init_exit_floor
 *                       (default 1e-3: FP32 cannot resolve smaller X~_beta
 *                       against 0.9; 0 restores the literal rule)
 *   T_thr               active-set threshold [K]: a 128-point tile may skip a
 *                       step only if it stays below T_thr and its martensite
 *                       is saturated, or if all its points sit on the
 *                       untouched state X_as = 0.9, X_am = 0 and it stays
 *                       below T_as_end, where the step is the identity
 *                       (<= 0 disables all skipping)                        */
typedef struct ms_params {
  double T_s, T_l;                /* solidus, liquidus [K]                       */
  double T_as_start, T_as_end;    /* beta -> alpha_s range [K]                   */
  double T_am_start, T_inf;       /* martensite start, ambient [K]               */
  double k_alpha_eq, k_am_eq;     /* equilibrium constants [1/K]                 */
  double c_as, c_b;               /* logistic exponents                          */
  double k1, k2, k3, f;           /* rate constant k_as(T) = k1/(1+exp(-k3(T-k2))), k_b = f k_as */
  double T_reg;                   /* regularisation width [K]                    */
  double init_exit;               /* App. A exit threshold on X~ * dt            */
  double init_exit_floor;         /* reading A5 floor on X~                       */
  double T_thr;                   /* active-set threshold [K]                    */
  int32_t martensite_literal;     /* reading A3                                  */
  int32_t init_ba_steps;          /* reading A6                                  */
  int32_t precision;              /* MS_F32 | MS_F64ACC | MS_KAHAN               */
  int32_t steps_per_launch;       /* S: steps per state load in ms_run_track (1..512) */
  int32_t rebuild_steps;          /* active-set rebuild period (multiple of S; 0 = S) */
  int32_t block_threads;          /* CTA size, multiple of 32 (0 = library choice) */
  int32_t flags;                  /* MS_FLAG_* bits                               */
  int32_t integrator;             /* MS_EXPLICIT or MS_IMPLICIT (Sec. 3)          */
  double  dt_sub;                 /* implicit: largest substep [s] (Sec. 3: 0.01;
                                     <= 0: no subcycling)                        */
  double  fp_eps_abs, fp_eps_rel; /* implicit: WRMS tolerances (Sec. 3: 1e-10, 1e-3) */
  int32_t fp_max_iter;            /* implicit: fixed-point iteration cap (100)    */
  int32_t tile_order;             /* ms_run_track with the active set: the order in
                                     which the persistent warps take the active
                                     tiles.  0 (default): heaviest first, by the
                                     cycles per step the hot kernel last spent on
                                     each tile (four classes against the previous
                                     launch's mean), so the launch's tail is made of
                                     cheap tiles; 1: tile index order.  Results do
                                     not depend on it.                            */
  /* Far field of the moving sources in ms_run_track (default 5e-3 m; 0 =
   * off: every source summed point by point).  In a tile of 128 points
   * inside one grid row, at a level whose sources all move along +-x, a
   * source that lies behind every point of the tile's x-range by at least
   * max(farfield_dist, 4 x the range) is evaluated at the 8 Chebyshev nodes
   * of that range, the sum over such sources is interpolated to the 128
   * points (Lagrange weights), and the other sources are summed point by
   * point.  Behind a source its term (ms_heat_source) is analytic in x
   * within a distance of the order of |xi| of the tile (the exponent
   * v p^2 / (2 alpha (R - xi)) has a positive real part there), so the
   * interpolation error per source is at most 4 M rho^-7 / (rho - 1) for any
   * Bernstein ellipse rho around the range that avoids the source, M the
   * term's bound on it; the 4-range guard keeps rho of about 17 or more on
   * any grid spacing, and for 128 points at 10 um and 5 mm, rho = 10 already
   * gives M <= A P / (2 pi k 2.1 mm) and <= 4.2e-5 K per source at P = 250 W
   * (the FP32 rounding of the direct sum is of the same order).  An
   * approximation of the direct sum, in every path whose arithmetic is FP32
   * (MS_F32, MS_F64ACC, MS_KAHAN, explicit or MS_IMPLICIT, and the hybrid
   * kernel); the full-FP64 path (MS_F64) always sums point by point.  The
   * library keeps 4 KB of interpolation weights on the device.             */
  double  farfield_dist;
} ms_params;

/* ------------------------------------------------------------ geometry */
/* A regular grid of points: x = origin[0] + i*spacing[0], y likewise with j,
 * z = origin[2] + (k + k_offset)*spacing[2] (spacing may be negative, e.g. z
 * going down).  k_offset (>= 0) makes the grid the z-planes k_offset ..
 * k_offset + nz - 1 of a larger grid with the same origin and spacing, with
 * the same coordinates to the bit: a z-slab shard of a block advances exactly
 * as those planes do in the block (ms_run_track, when nx * ny * k_offset is a
 * multiple of 128 so that the tiles coincide).  The thermal solver takes
 * k_offset = 0 only. */
typedef struct ms_grid {
  double origin[3];
  double spacing[3];
  int32_t dims[3];                /* nx, ny, nz (each >= 1)                     */
  int32_t k_offset;               /* first z-plane in the parent grid (>= 0)    */
} ms_grid;

/* ----------------------------------------------------- moving heat source */
/* The synthetic temperature driver evaluated on the device: every track of the
 * current layer that has started contributes a moving point source on a
 * half-space (thick-plate Rosenthal solution)
 *     dT = A P / (2 pi k R) * exp(-v (R + xi) / (2 alpha)),
 * R = |x - x_s|, xi = (x - x_s) . u (positive ahead of the source), with the
 * source at x_s = (x0, y0) + u v (t - t_start) on the layer surface and still
 * moving after its track ends.  T = min(T0 + s(t) * sum dT, T_max), where
 * s(t) = 1 during the layer's scan and falls linearly to 0 at the layer's
 * t_end (interlayer cool-down).  T_max = T_v + 1000 K (Sec. 2.1).  R = 0 gives
 * T_max.  Points above the current layer surface (z > z_surface + z_tol) are
 * not advanced.  Specimen-local time is t - t_offset. */
typedef struct ms_track {
  double x0, y0;                  /* start point on the layer surface [m]        */
  double ux, uy;                  /* unit direction                              */
  double v;                       /* speed [m/s]                                 */
  double P;                       /* power [W]                                   */
  double t_start;                 /* specimen-local start time [s]               */
  int32_t layer;                  /* index into the layer table                  */
  int32_t reserved;
} ms_track;

typedef struct ms_layer {
  double z_surface;               /* surface height during this layer [m]        */
  double t_begin;                 /* layer becomes current at this local time [s]*/
  double t_scan_end;              /* scan ends, cool-down scaling starts [s]      */
  double t_end;                   /* scaling reaches 0 [s]                        */
} ms_layer;

typedef struct ms_heat_source {
  double A;                       /* absorptivity                                */
  double k;                       /* conductivity [W/(m K)]                      */
  double alpha;                   /* diffusivity [m^2/s]                         */
  double T0;                      /* preheat / ambient [K]                       */
  double T_max;                   /* temperature cap [K]                         */
  double t_offset;                /* specimen start offset [s]                   */
  double z_tol;                   /* activity tolerance above the surface [m]    */
  int32_t n_tracks, n_layers;
  const ms_track* tracks;         /* tracks of one layer sorted by t_start       */
  const ms_layer* layers;
} ms_heat_source;

/* ------------------------------------------------------------- counters */
typedef struct ms_stats_t {
  int64_t steps;                  /* time levels advanced so far                 */
  int64_t point_updates;          /* points x steps advanced (dense count)       */
  int64_t tile_steps_total;       /* 128-point tiles x steps offered             */
  int64_t tile_steps_active;      /* ... of which were not skipped by the active set */
  int64_t launches;               /* kernel launches issued by the library       */
  double  last_run_ms;            /* device time of the last ms_run_track / ms_step */
  double  hot_kernel_ms;          /* summed device time of timed hot-kernel launches
                                     (MS_FLAG_TIME_KERNELS), since the last reset   */
  int64_t hot_kernel_launches;    /* number of launches in hot_kernel_ms          */
  int32_t device_error;           /* sticky device error word (0 = none)         */
  int32_t reserved;
  /* hybrid mode (ms_set_surrogate), since the last reset: point-windows of
   * MS_MLP_WINDOW x stride steps advanced by the MLP, point-windows advanced by the
   * explicit steps (band, initiation, layer change or a short tail), windows
   * re-run by the judge, and the largest |dX_as| or |dX_am| the judge saw
   * between the MLP and the explicit result of one window.                */
  int64_t surrogate_windows;
  int64_t ode_windows;
  int64_t judge_samples;
  double  judge_max_err;
  /* work of the plain hot kernel since the last reset: temperature
   * evaluations counted per point and started source, and point-steps on
   * which the phase model ran (the rest were skipped by the active set or the
   * warp vote of reading A9) */
  int64_t source_evaluations;
  int64_t model_point_steps;
  /* MS_IMPLICIT: fixed-point iterations done, and substeps that reached
   * fp_max_iter without meeting the WRMS stop (their last iterate is kept) */
  int64_t fp_iterations;
  int64_t fp_unconverged;
  /* explicit scheme, plain hot kernel: transcendental operations of the
   * phase model on the point-steps where it ran, counted on the branch each
   * point took (Sec. 2.2: exponentials of the equilibria and of k_as, the
   * powers x^p = 2^(p log2 x) of the rates, the reciprocal of k_as, and the
   * App. A closed form): ex2 class, and the log2 / reciprocal class; only
   * with MS_FLAG_COUNT_OPS (0 otherwise)                                     */
  int64_t model_sfu_ex2;
  int64_t model_sfu_slow;
  /* far field (farfield_dist > 0): source evaluations at the interpolation
   * nodes (8 per far source, tile and level), and point-source pairs whose
   * term came from the interpolation instead; source_evaluations then
   * counts the point-source pairs evaluated directly                       */
  int64_t farfield_node_evaluations;
  int64_t farfield_point_sources;
  int64_t judge_rejected;         /* judged tile-windows the judge sent back to
                                     the explicit steps (ms_set_judge_tol)       */
} ms_stats_t;

typedef struct ms_ctx ms_ctx;

/* ---------------------------------------------------------------- calls */

/* Library version string (static storage). */
const char* ms_version(void);

/* Message for a status code (static storage). */
const char* ms_strerror(int code);

/* Detail of the last failing call on this thread (thread-local storage). */
const char* ms_last_error(void);

/* sizeof of the public structs, for bindings to check their layouts:
 * which = 0 ms_params, 1 ms_grid, 2 ms_track, 3 ms_layer, 4 ms_heat_source,
 * 5 ms_stats_t.  Returns 0 for an unknown index. */
size_t ms_struct_size(int which);

#define MS_FF_TABLE_FLOATS 1032
/* The far field's interpolation table (ms_params.farfield_dist; not in the
 * paper): the Lagrange weights of the 8 Chebyshev points of the first kind
 * on a row tile's x-range [0, 1] at the tile's 128 points t_i = i / 127,
 * node-major (out[k * 128 + i]), then the 8 node positions (out[1024 + k]),
 * as the kernels use them.  Host only, no device work.  n_out is the
 * capacity of out in floats (at least MS_FF_TABLE_FLOATS).
 * Errors: INVALID_ARG (out NULL or too small). */
int ms_farfield_table(float* out, int32_t n_out);

/* Fill *p with the paper's constants and the default readings / options.
 * Errors: MS_ERR_INVALID_ARG if p is NULL. */
int ms_params_default(ms_params* p);

/* Check a parameter set as ms_create does, without creating anything (host
 * only, no CUDA call): the melt range 0 < T_s < T_l, T_as,end < T_as,start
 * and positive transformation temperatures (Table 2), positive rate and
 * equilibrium constants and c_as, c_b > 1 (Table 3), T_reg > 0, the App. A
 * exit thresholds >= 0, a finite T_thr, a known precision and integrator,
 * steps_per_launch and block_threads in range, a finite farfield_dist >= 0,
 * and for MS_IMPLICIT a finite dt_sub, eps_abs >= 0,
 * eps_rel > 0, fp_max_iter >= 1 with MS_F32 or MS_F64.
 * Returns MS_OK, MS_ERR_INVALID_ARG or MS_ERR_UNSUPPORTED, with the reason in
 * ms_last_error. */
int ms_params_check(const ms_params* p);

/* Create a context for n_points points on the current CUDA device and
 * allocate their state (all points start at the room-temperature
 * equilibrium X_as = 0.9, X_am = 0, App. A).  The parameters are copied.
 * Errors: INVALID_ARG (NULL, n_points <= 0, bad parameter), OOM, CUDA. */
int ms_create(const ms_params* p, int64_t n_points, ms_ctx** out);

/* Release all device memory and the owned stream.  NULL is ignored. */
void ms_destroy(ms_ctx* ctx);

/* Make the context launch on an existing CUDA stream (cudaStream_t passed as
 * void*; NULL = the context's own stream).  The stream is borrowed.  A
 * caller whose work runs on the legacy default stream (whose handle is NULL,
 * e.g. PyTorch's default stream) passes cudaStreamLegacy instead.  Waits
 * for the context's work on its old stream first.  Errors: INVALID_ARG (NULL
 * context), CUDA. */
int ms_set_stream(ms_ctx* ctx, void* cuda_stream);

/* Geometry for ms_run_track: n_specimens regular grids whose point counts add
 * up to the context's n_points (natural order, specimen after specimen).
 * Copied.  Errors: INVALID_ARG (count mismatch, bad dims), OOM, CUDA. */
int ms_set_points(ms_ctx* ctx, const ms_grid* grids, int32_t n_specimens);

/* Geometry for ms_run_track where the context's points are a subset of one
 * grid: point i of the context is grid point idx[i] (natural index of the
 * grid, i fastest), n == n_points.  Used to spot-check a large part on a
 * sample of its points (the FP64 path on 1e5 points of a 67M-point block).
 * Copied.  Errors: INVALID_ARG (n mismatch, index outside the grid), OOM, CUDA. */
int ms_set_points_subset(ms_ctx* ctx, const ms_grid* grid, const int64_t* idx, int64_t n);

/* Set the state of every point from host arrays of n_points doubles.
 * aux may be NULL (no initiation in progress) or give per point the App. A
 * variable: X~_beta > 0 of an active alpha_s -> beta initiation, -1 for an
 * active (init_ba_steps) beta -> alpha_s initiation, 0 for none.
 * Validates 0 <= X_as, 0 <= X_am, X_as + X_am <= 0.9 (+1e-6).
 * Resets the step counter to 0.  Errors: INVALID_ARG, NONFINITE, CUDA. */
int ms_set_state(ms_ctx* ctx, const double* x_as, const double* x_am, const double* aux);

/* Set every point to the same state (X_as = x_as, X_am = x_am, no initiation
 * in progress) with a device fill, no host copy, and reset the step counter.
 * Asynchronous.  Errors: INVALID_ARG (fractions outside [0, 0.9]), CUDA. */
int ms_fill_state(ms_ctx* ctx, double x_as, double x_am);

/* Reset the counters of ms_stats (not the state).  Synchronises the stream.
 * Errors: INVALID_ARG (NULL), CUDA. */
int ms_reset_stats(ms_ctx* ctx);

/* One explicit step of every point with given temperatures T_prev = T^n and
 * T_new = T^{n+1} (n_points floats each, Algorithm 1 / Algorithm 2; rates at
 * T^n, correction at T^{n+1}).  flags & MS_PTR_DEVICE: device pointers,
 * borrowed for the call (and T_new until the next ms_step or
 * ms_get_fractions, which reads it for X_beta and X_liq); else host pointers
 * (copied).  dt > 0 [s].  Asynchronous on the context stream for device
 * pointers.  Errors: INVALID_ARG, STATE (context has several specimens),
 * CUDA. */
int ms_step(ms_ctx* ctx, const float* T_prev, const float* T_new, double dt, int32_t flags);

/* Advance every point n_steps explicit steps of size dt under the moving
 * sources, src[s] being the heat source of specimen s (as many as given to
 * ms_set_points).  Temperatures are evaluated on the device at every time
 * level t_n = n * dt (n counts the steps since ms_set_state), so only the
 * phase state touches memory.  Asynchronous on the context stream.
 * Errors: INVALID_ARG (dt <= 0, n_steps < 0, bad source), STATE (no points),
 * OOM, CUDA. */
int ms_run_track(ms_ctx* ctx, const ms_heat_source* src, int64_t n_steps, double dt);

/* Copy the four fractions of every point to host arrays of n_points doubles:
 * X_as, X_am, X_beta = 1 - g(T) - X_as - X_am, X_liq = g(T) with T the
 * temperature of the last level (x_beta and x_liq may be NULL).  Synchronises
 * the stream and reports a sticky device error.  Errors: INVALID_ARG, STATE
 * (no temperature known yet for X_beta / X_liq), NONFINITE, CUDA. */
int ms_get_fractions(ms_ctx* ctx, double* x_as, double* x_am, double* x_beta, double* x_liq);

/* App. A variable of every point in the encoding of ms_set_state (n_points
 * doubles).  Errors: INVALID_ARG, CUDA. */
int ms_get_aux(ms_ctx* ctx, double* aux);

/* Temperature of every point at the current time level (the moving source of
 * the last ms_run_track, or T_new of the last ms_step), n_points doubles, in
 * the context's arithmetic precision.  Errors: INVALID_ARG, STATE (no
 * temperature known yet), CUDA. */
int ms_get_temperature(ms_ctx* ctx, double* T);

/* Checkpoint: serialise the full device state (fractions, App. A variables,
 * step counter, dt) into blob.  With blob == NULL only *bytes is set to the
 * required size.  Errors: INVALID_ARG (buffer too small), CUDA. */
int ms_get_state(ms_ctx* ctx, void* blob, size_t* bytes);

/* Restore a checkpoint made by ms_get_state on a context with the same
 * n_points and precision.  Errors: INVALID_ARG (size / header mismatch), CUDA. */
int ms_set_state_blob(ms_ctx* ctx, const void* blob, size_t bytes);

/* Throughput probe of one SM pipe, measured on the current device so that
 * roofline fractions use a measured peak (as Sec. 4 measures its CPUs' peak
 * FLOP/s and DAXPY bandwidth before quoting roofline fractions): op 0
 * ex2.approx.f32, 1 lg2.approx.f32, 2 rsqrt.approx.f32, 3 rcp.approx.f32
 * alternating with rsqrt.approx.f32 (both counted), 4 fma.rn.f32.  About 1e10 operations, best of 3 timed repeats.
 * *ops_per_s receives thread-level operations per second, *sm_mhz (may be
 * NULL) the SM clock the probe saw (clock64 cycles per globaltimer ns).
 * Allocates and frees its own small buffers and stream.
 * Errors: INVALID_ARG (op out of range, NULL ops_per_s), CUDA. */
int ms_probe_sfu(int op, double* ops_per_s, double* sm_mhz);

/* ------------------------------------------------ coarsening criterion */
/* The phase-aware coarsening criterion of the paper's adaptive mesh (Sec. 3,
 * the adaptive-mesh passage: an octant made of eight sibling cells of one
 * refinement level may be coarsened only when, for every microstructure
 * phase, all its values are close to each other).  On a grid of points
 * (dims = nx, ny, nz; natural order, x fastest) the finest cells lie between
 * neighbouring points, and octant i of level l >= 1 spans the points
 * i 2^l .. (i + 1) 2^l along an axis of n > 1 points (floor((n - 1) / 2^l)
 * octants per axis) and the single point of an axis with n = 1.  The octant
 * may be coarsened when, for each of X_as, X_am and X_beta, its largest
 * minus its smallest value over the octant's points is <= tol (one FP64
 * subtraction: the decision is exact; a NaN among the points makes the range
 * NaN and the decision false).  A coarsenable octant's children are
 * coarsenable, so the masks nest.  This is the criterion the phases impose;
 * a mesh also coarsens by its own rules (the consolidated fraction, the
 * refinement kept near the active layer), which are not part of it.       */
#define MS_COARSEN_MAX_LEVELS 30

/* Octant counts of levels 1 .. n_levels for grid dims (host only, no CUDA
 * call): counts[l - 1] = octants of level l (0 once an axis runs out), and
 * (scratch_bytes may be NULL) the device scratch ms_coarsen_mask needs: the
 * per-octant minima and maxima of two levels (6 doubles per level-2 and per
 * level-3 octant) and its counters.
 * Errors: INVALID_ARG (dims < 1, n_levels outside [1, MS_COARSEN_MAX_LEVELS],
 * NULL counts). */
int ms_coarsen_sizes(const int32_t* dims, int32_t n_levels, int64_t* counts,
                     size_t* scratch_bytes);

/* The masks of levels 1 .. n_levels for the phase fields x_as, x_am, x_beta
 * (nx ny nz doubles each, natural order).  mask receives the levels in turn,
 * each x fastest, one byte per octant (1 = may be coarsened), sum of
 * ms_coarsen_sizes' counts bytes in all; n_coarse (may be NULL) receives the
 * coarsenable octants per level.  flags MS_PTR_DEVICE: the three fields and
 * mask are device pointers, and scratch (may be NULL) is a device buffer of
 * at least the scratch_bytes ms_coarsen_sizes gives, 16-byte aligned, that
 * the call uses instead of allocating; without MS_PTR_DEVICE they are host
 * pointers, copied through device buffers the call allocates (scratch must
 * be NULL).  stream is a cudaStream_t (NULL = legacy default stream); the
 * call returns when the result is in place.  One kernel reduces levels 1
 * and 2 from the fields (a thread per level-2 slot), the next levels reduce
 * the per-octant ranges of the level below.
 * Errors: INVALID_ARG (NULL field or mask, dims < 1, n_levels out of range,
 * tol negative or not finite, scratch without MS_PTR_DEVICE, too small or
 * misaligned), OOM, CUDA. */
int ms_coarsen_mask(const double* x_as, const double* x_am, const double* x_beta,
                    const int32_t* dims, double tol, int32_t n_levels, uint8_t* mask,
                    int64_t* n_coarse, void* scratch, size_t scratch_bytes, int32_t flags,
                    void* stream);

/* The same criterion on a context's current state: X_as, X_am and X_beta =
 * 1 - X_liq - X_as - X_am at the temperature of its current time level, as
 * ms_get_fractions returns them.  The context must hold one full grid
 * (ms_set_points with one specimen); mask and n_coarse (may be NULL) are
 * host arrays as in ms_coarsen_mask.  Synchronises the context's stream.
 * Errors: INVALID_ARG (NULL mask, n_levels out of range, tol negative or not
 * finite), STATE (no single full grid, or no temperature known yet), OOM,
 * CUDA, NONFINITE (the sticky device error word). */
int ms_coarsen_ctx(ms_ctx* ctx, double tol, int32_t n_levels, uint8_t* mask, int64_t* n_coarse);

/* The device's exp2 and log2 on host arrays, for checking them against the
 * mathematics: which = 0 the FMA-pipe polynomial exp2, 1 the FMA-pipe log2
 * (MS_FLAG_FMA_TRANSCENDENTALS; the paper's fast transcendentals, Sec. 3.3),
 * 2 the SFU's ex2.approx.ftz.f32, 3 the SFU's lg2.approx.ftz.f32, element
 * by element from x to y (n floats each).  Allocates and frees its own
 * device buffers; synchronous.
 * Errors: INVALID_ARG (which outside 0..3, NULL x or y, n < 0), OOM, CUDA. */
int ms_eval_transcendental(int which, const float* x, float* y, int64_t n);

/* ms_run_track_noalloc -- the ms_run_track hot path without allocating.
 * The paper has no counterpart; this is an integration entry point.
 *
 * For callers that cannot allocate device memory at run time.  Applications
 * whose device memory is owned by a pre-sized pool (a framework's caching
 * allocator, a memory budget fixed at start-up) may not allocate outside it.
 * Latency-critical loops cannot afford cudaMalloc / cudaFree, which can
 * synchronise the whole device.  Embeddings that must not grow the GPU
 * footprint while they run cannot allocate either.  ms_create allocates its
 * context buffers with cudaMalloc; this call keeps its scratch (the
 * per-launch source table, the work counters of the persistent kernel, the
 * specimen / track / layer tables and the far-field weights) in one
 * file-scope static device array of 0.77 MiB, which every GPU that loads the
 * library holds until the process exits.
 *
 * It advances one specimen (grid, src) from time level step0 by n_steps
 * explicit steps of dt.  The result is the same as ms_run_track after
 * ms_set_points(grid) from the same state (MS_F32 only, no active-set tile
 * list; the per-step warp vote of T_thr still applies).  The caller owns the
 * state: x_as, x_am and aux are device arrays, 16-byte aligned, each holding
 * at least n_points rounded up to a multiple of 128 floats, in natural
 * order; aux is the library's opaque per-point initiation state, as
 * ms_get_aux returns it (0 means no initiation in progress; keep the array
 * between calls).  The work is queued on cuda_stream (NULL = the legacy
 * default stream); the call returns once that stream has finished it,
 * because it reads the device error word of its launches.
 *
 * Limits: n_points <= 2^24, src->n_tracks <= 128, src->n_layers <= 8,
 * steps_per_launch <= 64, block_threads 0 or 128; larger requests return
 * MS_ERR_INVALID_ARG with a message in ms_last_error.  No cudaMalloc,
 * cudaFree or other allocating call is made.  The first call on a device
 * does a one-time set-up: it looks up the array's device address
 * (cudaGetSymbolAddress), clears the array with cudaMemset and waits for the
 * device (cudaDeviceSynchronize) so that the clear has landed before any
 * stream touches the array; make that first call before any stream capture.
 * Every call shares the array, which keeps the last call's contents (each
 * call resets the error word and the counters it needs); calls whose work
 * overlaps on the GPU (other streams, other host threads) race on it, so the
 * caller must serialise them.
 * farfield_dist applies as in ms_run_track.
 * Errors: INVALID_ARG, UNSUPPORTED (precision other than MS_F32, MS_IMPLICIT,
 * or cuda_stream is capturing: the tables are uploaded from host memory of
 * the call), NONFINITE (a fraction became non-finite in this call's
 * launches), CUDA. */
int ms_run_track_noalloc(const ms_params* p, const ms_grid* grid, const ms_heat_source* src,
                         float* x_as, float* x_am, float* aux, int64_t n_points,
                         int64_t step0, int64_t n_steps, double dt, void* cuda_stream);

/* ------------------------------------------------------ learned surrogate */
/* A small MLP that advances a point's fractions over a window of
 * MS_MLP_WINDOW x r explicit steps in one evaluation, r (1, 2, 4, 8 or 16) being
 * the surrogate's temperature stride: the network sees the temperatures of
 * the window's levels r, 2 r, ..., 8 r.  The paper integrates every step
 * (Sec. 3); the surrogate is an extension of the method, used only where the
 * explicit steps are smooth: a window falls back to the explicit steps when
 * any of its sampled temperatures (the window start and the 8 samples) lies
 * within 40 K of T_am,start, T_as,end, T_as,start or T_as,start + T_reg, or
 * above T_s - 40 K, when two consecutive samples differ by more than 40 K,
 * or when an App. A initiation is running.  With r > 1 the temperatures
 * between samples are not evaluated for the window's MLP points: the
 * sample test stands for them (a window that passes it stays at least 40 K
 * from every switching temperature at its samples and changes by at most
 * 40 K between them).  Points whose samples are all cold and saturated
 * (the test of the plain path's skip, at the samples) keep their state.
 *
 * Network: inputs x[12] = (X_as, X_am, X_beta at the window start, the 8
 * sampled temperatures as (T - 1000 K) / 1000 K, log10(dt) + 5); hidden
 * 64 -> 64 with the surrogate's activation (MS_ACT_GELU: GELU, tanh form;
 * MS_ACT_RELU: max(x, 0)); outputs y[3] = 1e6 x the window's diffusive
 * residual (X_as, X_am, X_beta at the window end minus G(start fractions),
 * where G = g(T_8r, .) o ... o g(T_r, .) applies only the correction g at the
 * 8 sampled temperatures in turn).  An MLP window sets
 * X = g(T_8r, G(X_start) + y / 1e6): the instantaneous part (clamping, the
 * 0.9 bound, the alpha_s cap, martensite dissolution and formation) is taken
 * exactly at the sampled temperatures and the network supplies the rest of
 * the window, the diffusion of Sec. 2.2.  Parameters: MS_MLP_PARAMS floats,
 * W1[64][12], b1[64], W2[64][64], b2[64], W3[3][64], b3[3], weights
 * row-major (out x in).  Inference uses BF16 weights and activations with
 * FP32 accumulation on the tensor cores; training keeps an FP32 master copy
 * (Adam).                                                                  */
#define MS_MLP_IN      12
#define MS_MLP_OUT     3
#define MS_MLP_PARAMS  5187
#define MS_MLP_WINDOW  8      /* temperature samples per window             */
#define MS_ACT_GELU    0
#define MS_ACT_RELU    1

typedef struct ms_surrogate ms_surrogate;

/* Create a surrogate from MS_MLP_PARAMS host floats (copied) with the given
 * hidden activation (MS_ACT_GELU or MS_ACT_RELU) and temperature stride
 * (1, 2, 4, 8 or 16; windows of 8 x stride steps).  Owns its device buffers and a
 * stream.  The activation and the stride are the network's: training and
 * inference use them, and windows for its training must be cut with the
 * same stride.  Errors: INVALID_ARG (NULL, non-finite, another activation
 * or stride), OOM, CUDA. */
int ms_surrogate_create_ex(const float* params, int32_t activation, int32_t stride,
                           ms_surrogate** out);
/* ms_surrogate_create_ex(params, MS_ACT_GELU, 1, out).  Errors: those of
 * ms_surrogate_create_ex. */
int ms_surrogate_create(const float* params, ms_surrogate** out);
/* The surrogate's activation and stride.  Errors: INVALID_ARG (NULL). */
int ms_surrogate_get_config(const ms_surrogate* s, int32_t* activation, int32_t* stride);
/* Free a surrogate (NULL is a no-op).  Detach it from every context first. */
void ms_surrogate_destroy(ms_surrogate* s);
/* Run later calls on cuda_stream (NULL = the surrogate's own stream; pass
 * cudaStreamLegacy for the legacy default stream).  Data written by other
 * streams must be complete before a call reads it.  Errors: INVALID_ARG
 * (NULL surrogate). */
int ms_surrogate_set_stream(ms_surrogate* s, void* cuda_stream);
/* Copy the FP32 master parameters to a host array of MS_MLP_PARAMS floats
 * (synchronises).  Errors: INVALID_ARG (NULL), CUDA. */
int ms_surrogate_get_params(ms_surrogate* s, float* params);
/* Inference on n samples: x device [n][12] FP32, y device [n][3] FP32 (the
 * network output, i.e. 10 x increments).  Asynchronous.  Errors:
 * INVALID_ARG (NULL, n < 0), CUDA (launch). */
int ms_surrogate_forward(ms_surrogate* s, const float* x, float* y, int64_t n);
/* Mean-squared-error gradient over n samples (x device [n][12], targets t
 * device [n][3]): loss = sum (y - t)^2 / (3 n).  The forward pass rounds the
 * weights, inputs and hidden activations to BF16 as inference does.  grad
 * (device, MS_MLP_PARAMS floats, may be NULL) receives dloss/dparams; loss
 * (host, may be NULL; synchronises) the loss before the update.
 * Errors: INVALID_ARG (NULL, n <= 0), OOM (per-sample scratch), CUDA. */
int ms_surrogate_gradient(ms_surrogate* s, const float* x, const float* t, int64_t n,
                          float* grad, double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * gradient of n samples with learning rate lr; refreshes the BF16 copy.
 * Errors: those of ms_surrogate_gradient, INVALID_ARG (lr <= 0 or NaN). */
int ms_surrogate_train_step(ms_surrogate* s, const float* x, const float* t, int64_t n,
                            double lr, double* loss);

/* Apply the correction g of eq:explicit_correction to n independent points
 * at the temperatures T[i][0], ..., T[i][n_T - 1] in turn (T: host array of
 * n x n_T doubles, row-major; x_as, x_am: host arrays updated in place; FP64
 * on the device with the context's parameters).  Not a time step: it forms
 * the surrogate's training targets.  Errors: INVALID_ARG (n_T < 1), OOM,
 * CUDA. */
int ms_apply_correction(ms_ctx* ctx, const double* T, int32_t n_T, double* x_as, double* x_am,
                        int64_t n);

/* Attach a surrogate to a context (NULL detaches): ms_run_track then advances
 * whole windows of MS_MLP_WINDOW x stride steps (counted from the first level
 * of each launch of steps_per_launch steps; a launch's last window, if
 * shorter, takes the explicit steps) with the MLP where the band test allows
 * and with the explicit steps elsewhere.  judge_frac in [0, 1] is the fraction of the 128-point tiles'
 * windows, drawn by a counter-based hash of (tile, level), whose MLP points
 * are also run with the explicit steps to measure the surrogate's error
 * (ms_stats); the MLP result is kept unless the judge's tolerance
 * (ms_set_judge_tol) sends the tile-window back to the explicit steps.
 * The surrogate must outlive its attachment.  Requires MS_F32 or MS_KAHAN.
 * Errors: INVALID_ARG, UNSUPPORTED (other precisions). */
int ms_set_surrogate(ms_ctx* ctx, const ms_surrogate* s, double judge_frac);

#define MS_JUDGE_TOL_DEFAULT 5e-4
/* The judge's tolerance (the paper has no surrogate; this is the hybrid
 * path's own safeguard).  A judged 128-point tile-window whose largest
 * |dX_as| or |dX_am| between the network's result and the explicit steps'
 * exceeds tol takes the explicit steps' result for all its network points
 * (fractions and App. A state), and ms_stats counts it in judge_rejected;
 * tol = +inf keeps the network's result everywhere (the judge only
 * measures).  Default MS_JUDGE_TOL_DEFAULT; applies from the next
 * ms_run_track.  Errors: INVALID_ARG (NULL context, tol NaN or negative). */
int ms_set_judge_tol(ms_ctx* ctx, double tol);

/* ------------------------------------------------- grid thermal solver */
/* An explicit finite-volume solver of the heat equation of Sec. 2.1 on a
 * regular grid, to feed ms_step with T^n and T^{n+1} (the paper's one-way
 * coupling): rho c dT/dt = div(k grad T) + q_vol with
 * k = (1 - r_c) k_p + r_c k_ms (eq:material_parameter_interp, k_m = k_s),
 * r_c the running maximum of g(T) (eq:consolidated_fraction; nodes within
 * h_powder of the top surface start as powder, r_c = 0), harmonic-mean face
 * conductances, the cylindrical laser source eq:heat_soruce_cylindrical in
 * the nodes within h_powder of the top surface (the laser on a track from the
 * track's start to the next track's start, the last track of a layer to the
 * layer's scan end; W_eff = the track's P), radiation eps sigma (T^4 - T_inf^4)
 * from the top layer of nodes, T0 on the bottom layer (Dirichlet), adiabatic
 * sides.  Explicit Euler substeps: ceil(dt / (0.9 dt_stab)) with
 * dt_stab = rho c / (k_ms (2/dx^2 + 2/dy^2 + 2/dz^2)); after each substep T is
 * capped at T_max (the paper's limit T_v + 1000 K, which stands in for the
 * evaporation losses here) and r_c <- max(r_c, g(T)).  FP32 on the device.
 * Fields are float arrays in natural grid order (x fastest). */
typedef struct ms_thermal_params {
  double rho, c;                  /* density, heat capacity (Table 1)            */
  double k_ms, k_p;               /* conductivity of melt/solid and powder       */
  double T_s, T_l;                /* solidus, liquidus [K]                        */
  double T0, T_inf;               /* preheat (initial and Dirichlet), ambient [K] */
  double emissivity;              /* top-surface radiation (Table 1: 0.7)         */
  double T_max;                   /* temperature cap [K] (T_v + 1000 K)           */
  double beam_radius;             /* R of the cylindrical source [m] (Table 5)    */
  double h_powder;                /* powder layer thickness [m]                   */
  int32_t radiation;              /* 1: radiation from the top layer              */
  int32_t dirichlet_bottom;       /* 1: bottom layer held at T0                   */
  int32_t cap;                    /* 1: cap at T_max                              */
  int32_t reserved;
} ms_thermal_params;

typedef struct ms_thermal ms_thermal;

/* Table 1 / Table 5 values, T0 = 353 K, h_powder = 30 um, all options on.
 * Errors: INVALID_ARG (p NULL). */
int ms_thermal_params_default(ms_thermal_params* p);
/* A solver on grid (dims >= 1, finite non-zero spacing); T = T0.  Owns its
 * device fields and a stream.  Errors: INVALID_ARG, OOM, CUDA. */
int ms_thermal_create(const ms_thermal_params* p, const ms_grid* grid, ms_thermal** out);
/* Free a solver (NULL is a no-op). */
void ms_thermal_destroy(ms_thermal* th);
/* Run later calls on cuda_stream (NULL = the solver's own stream).
 * Errors: INVALID_ARG (NULL solver). */
int ms_thermal_set_stream(ms_thermal* th, void* cuda_stream);
/* T = T0, r_c from the powder layer, time 0 (synchronises).
 * Errors: INVALID_ARG (NULL solver), CUDA. */
int ms_thermal_reset(ms_thermal* th);
/* The laser path: src's tracks, sorted by start time within each layer, and
 * layers (copied; the time offset applies).  Errors: INVALID_ARG (NULL, no
 * layer, a track with a bad layer index, v <= 0, P < 0 or a non-finite start,
 * tracks of a layer out of start-time order); the old path is kept then. */
int ms_thermal_set_source(ms_thermal* th, const ms_heat_source* src);
/* Advance by dt (synchronises, adds the device time to ms_thermal_stats).
 * Errors: INVALID_ARG (NULL, dt not finite and positive), CUDA. */
int ms_thermal_step(ms_thermal* th, double dt);
/* Device pointers (valid until the next step or reset) of T at the start
 * and at the end of the last step and of r_c; any may be NULL.  Errors:
 * INVALID_ARG (NULL solver). */
int ms_thermal_fields(ms_thermal* th, const float** T_prev, const float** T_cur, const float** rc);
/* Host copies (n doubles each, natural order); either may be NULL
 * (synchronises).  Errors: INVALID_ARG (NULL solver), CUDA. */
int ms_thermal_get(ms_thermal* th, double* T, double* rc);
/* Simulated time, substeps taken, device time of ms_thermal_step calls;
 * any output may be NULL.  Errors: INVALID_ARG (NULL solver). */
int ms_thermal_stats(ms_thermal* th, double* time_s, int64_t* substeps, double* kernel_ms);
/* n_steps coupled steps of dt on ctx's stream: a thermal step, then
 * ms_step(ctx, T_prev, T_cur, dt, MS_PTR_DEVICE).  ctx must hold one
 * specimen of the same number of points, in the grid's natural order.
 * Errors: INVALID_ARG, the errors of ms_step. */
int ms_thermal_run_coupled(ms_thermal* th, ms_ctx* ctx, int64_t n_steps, double dt);

/* Verification on the device, without copying the state to the host: with
 * j = idx[i] (or i when idx is NULL), compares point j of ctx with point i of
 * ref for i < n over the four fractions X_as, X_am, X_beta, X_liq (each with
 * its context's current temperature) and writes
 *   out[0] = max over i of the largest |X(ctx, j) - X(ref, i)|,
 *   out[1] = max over ctx's points of |X_as + X_am + X_beta + X_liq - 1|,
 *   out[2] = the same for ref's points
 * (NaN reported as +inf).  Typical use: ref an MS_F64 context on a point
 * subset (ms_set_points_subset) of ctx's grid, idx the subset's indices.
 * idx is a host array (copied).  Synchronises both streams.
 * Errors: INVALID_ARG (n larger than ref's points, or than ctx's without idx,
 * an index out of range, contexts on different devices), STATE (no
 * temperature known yet), NONFINITE, CUDA. */
int ms_verify(ms_ctx* ctx, ms_ctx* ref, const int64_t* idx, int64_t n, double* out);

/* Counters and the sticky device error word (synchronises the stream).
 * Errors: INVALID_ARG (NULL), CUDA.  A sticky device error is reported in
 * out->device_error, not as the return value (ms_synchronize returns it). */
int ms_stats(ms_ctx* ctx, ms_stats_t* out);

/* Wait for all work on the context stream; reports a sticky device error.
 * Errors: INVALID_ARG (NULL), DEVICE_TIMEOUT or NONFINITE (the sticky word),
 * CUDA. */
int ms_synchronize(ms_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MS_H */
