// Internal interface between the C-ABI layer (ms_api.cu) and the kernels
// (ms_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ms.h"
#include "ms_device.cuh"

namespace ms {

constexpr int TILE = 128;          // points per tile = one warp x 4 points per thread
constexpr int MAX_LEVELS = 513;    // steps_per_launch <= 512

// device error word bits
constexpr int DEVERR_NONFINITE = 1;
constexpr int DEVERR_TIMEOUT = 2;

// One specimen as the kernels see it.
struct SpecDev {
  double ox, oy, oz;       // grid origin
  double dx, dy, dz;       // grid spacing
  const int64_t* idx;      // optional: the specimen's points are these grid indices
  int32_t nx, ny, nz;
  int32_t n_tracks;        // tracks of this specimen (all layers)
  int64_t n;               // points
  int64_t nat_off;         // offset in natural (user) order
  int64_t pad_off;         // offset in the padded device arrays (multiple of TILE)
  int64_t tile0;           // first tile
  int32_t n_tiles;
  int32_t track0;          // first track in the track table
  int32_t layer0;          // first layer in the layer table
  int32_t n_layers;
  float z_tol;
  float T0, T_max;
  int32_t k_off;           // z-plane offset in the parent grid (ms_grid.k_offset)
  double A, k, alpha, t_offset;
};

struct TrackDev {
  double x0, y0, ux, uy, v, P, t_start;
  int32_t layer;
  int32_t spec;            // specimen of the track
};

// One track over an active-set window [t_a, t_b] (written with the source
// table of the launch): the source's path in the window, absolute.
struct TrackWin {
  double ax, ay;           // position at max(t_a, t_start)
  double bx, by;           // position at t_b
  float ux, uy, v;         // direction and speed
  float cp;                // A P / (2 pi k) (the bound inflates it)
  float z;                 // surface of the track's layer
  int32_t on;              // started by t_b and on a layer current in the window
};

struct LayerDev {
  double z, t_begin, t_scan_end, t_end;
};

// Arguments of the source-table kernel.
struct TableArgs {
  const SpecDev* specs;
  const TrackDev* tracks;
  const LayerDev* layers;
  int32_t n_specs;
  int32_t n_levels;        // levels n0 .. n0 + n_levels - 1
  int32_t slots;           // entries per (specimen, level)
  int32_t pad;
  int64_t n0;              // first level (steps since the time base)
  double t_base;           // time of level 0 of the time base
  double dt;
  void* levels;            // SrcLevelT<AT> [n_specs][n_levels]
  void* entries;           // SrcEntryT<AT> [n_specs][n_levels][slots]
  // optional, for the active set: every track over the window [t_a, t_b]
  TrackWin* win;           // [n_tracks] or nullptr
  int32_t n_tracks;        // tracks of all specimens
  int32_t pad2;
  double t_a, t_b;
  double ff_dist;          // far-field distance of the launches (0: far field off)
};

// Active tiles are handed out heaviest first: the active set sorts them into
// COST_BUCKETS classes by the time k_track last spent on them per level
// (>= 2x, >= 1x, >= 1/2 x the mean of the previous launch, the rest and
// unmeasured tiles), one list region of n_tiles entries per class, and the
// persistent warps pull the classes in order, so the launch's tail is made
// of the cheapest tiles.  The order never changes a result (tiles are
// independent).
constexpr int COST_BUCKETS = 4;

// Work counters of one launch of k_track (device memory, reset per launch).
struct WorkCounters {
  int32_t n_active;            // tiles in the active list
  int32_t next;                // next list position handed to a warp
  unsigned long long tile_steps_active;  // running total of processed tile-steps
  int32_t n_bucket[COST_BUCKETS];        // active tiles per cost class
  uint32_t cost_cnt[2];                  // tiles timed by k_track, by launch parity
  unsigned long long cost_sum[2];        // their cycles per level, summed
};

// Position w of the heaviest-first order -> tile index: the classes' list
// regions (stride entries each) in turn.
__device__ __forceinline__ int list_tile(const int32_t* list, int stride, const int* nb, int w) {
#pragma unroll
  for (int b = 0; b < COST_BUCKETS - 1; ++b) {
    if (w < nb[b]) return list[int64_t(b) * stride + w];
    w -= nb[b];
  }
  return list[int64_t(COST_BUCKETS - 1) * stride + w];
}

// Work done by the plain hot kernel (running totals, reset by
// ms_reset_stats): point x source evaluations of the temperature, and point
// steps on which the model ran (not skipped by the warp vote).
struct OpCounters {
  unsigned long long source_evaluations;
  unsigned long long model_point_steps;
  unsigned long long fp_iterations;    // implicit scheme: fixed-point iterations
  unsigned long long fp_unconverged;   // implicit scheme: substeps that hit the cap
  unsigned long long model_sfu_ex2;    // explicit scheme: the model's exponentials
  unsigned long long model_sfu_slow;   // explicit scheme: the model's logarithms and reciprocals
  unsigned long long farfield_node_evaluations;  // far field: source evaluations at the nodes
  unsigned long long farfield_point_sources;     // far field: point-source pairs interpolated
};

// Far field of the moving sources (ms_params.farfield_dist): 8 Chebyshev
// nodes over a row tile's x-range, Lagrange weights of the 128 points.
constexpr int FF_NODES = 8;
// Device buffer: weights [FF_NODES][TILE] (node-major, so that a warp reads
// one node's weights of its 128 points as one float4 per lane), then the
// nodes' positions as fractions of the range [FF_NODES], padded to 16 bytes.
constexpr int FF_FLOATS = FF_NODES * TILE + FF_NODES;
// A source is interpolated only if it lies at least FF_RANGE_GUARD tile
// x-ranges behind the tile (and at least farfield_dist): the Bernstein
// ellipse of the interpolation then keeps rho >= 17 on any grid spacing.
constexpr float FF_RANGE_GUARD = 4.0f;

// Counters of the hybrid kernel (running totals, reset by ms_reset_stats).
struct HybridCounters {
  unsigned long long surrogate_windows, ode_windows, judge_samples;
  unsigned int judge_err_bits;  // bits of the largest judged |dX| (>= 0, so integer order = float order)
  unsigned int pad;
  unsigned long long judge_rejected;  // judged tile-windows sent back to the explicit steps
};

// Arguments of the run-track kernel (persistent warps pull 128-point tiles).
template <typename AT, typename FT>
struct TrackArgs {
  ModelConstT<AT> m;
  const SpecDev* specs;
  const int32_t* tile_spec;    // tile -> specimen
  const int32_t* tile_list;    // active tiles (nullptr: every tile 0 .. n_tiles-1)
  WorkCounters* work;          // n_active (with a list) and the work cursor
  int32_t n_tiles;             // tiles in the layout
  int32_t n_levels;            // steps + 1
  int32_t slots;
  AT dt;
  const SrcLevelT<AT>* levels;
  const SrcEntryT<AT>* entries;
  FT* xas;
  FT* xam;
  float* aux;
  float* tile_tsat;            // per tile: highest T at which formation still acts (+inf: busy)
  int* err;
  OpCounters* ops;             // work counters of k_track (nullptr: not counted)
  int32_t n_sub;               // implicit scheme: substeps per step
  const float* ff;             // far-field weights and nodes (FF_FLOATS), nullptr: off
  float ff_dist;               // far-field distance [m]
  uint32_t* tile_cost;         // per tile: cycles per level when last processed (nullptr: not timed)
  int32_t cost_slot;           // launch parity: WorkCounters::cost_sum slot this launch adds to
  int32_t count_sfu;           // count the model's transcendentals per branch (MS_FLAG_COUNT_OPS)
  // hybrid kernel only
  const void* mlp;             // MlpDev of the attached surrogate
  HybridCounters* hyb;
  uint64_t judge_thresh;       // a window is judged if hash(point, level) < judge_thresh (2^32 = all)
  float judge_tol;             // a judged tile-window with a larger |dX| takes the explicit result
  int32_t two_rows;            // the layout has tiles across two grid rows (k_track's far field for them)
  int64_t level0;              // global index of the launch's first level
  int32_t mlp_stride;          // levels between a window's temperature samples (1, 2, 4, 8, 16)
};

// Arguments of the active-set builder (reading A9): a tile joins the list
// unless it provably stays below T_thr over [t_a, t_b] and its martensite is
// saturated at the preheat temperature.
struct ActiveArgs {
  const SpecDev* specs;
  const TrackWin* win;         // the tracks over the launch's window (source-table launch)
  const int32_t* tile_spec;
  const float* tile_tsat;
  int32_t n_tiles;
  int32_t pad;
  double T_thr;
  double T_as_end;             // fixed-point tiles are idle below it
  int32_t* tile_list;          // COST_BUCKETS regions of n_tiles entries
  WorkCounters* work;
  const uint32_t* tile_cost;   // per tile: cycles per level when last processed (nullptr: one class)
  int32_t prev_slot;           // the previous launch's cost slot (its mean sets the classes)
  int32_t pad2;
};

// Arguments of the external-temperature step kernel.
template <typename AT, typename FT>
struct StepArgs {
  ModelConstT<AT> m;
  int64_t n;
  AT dt;
  const float* T0;
  const float* T1;
  FT* xas;
  FT* xam;
  float* aux;
  int* err;
  OpCounters* ops;             // implicit iteration counters (nullptr: not counted)
  int32_t n_sub;               // implicit scheme: substeps per step
};

// Parameter checks and derived constants shared by the C-ABI entry points
// (ms_api.cu): validate_params returns MS_OK or an MS_ERR_* code and records
// the message for ms_last_error; record_error records a message and returns
// the code.
int validate_params(const ms_params& p);
template <typename AT>
ModelConstT<AT> model_const(const ms_params& p);
int record_error(int code, const char* msg);

// Launchers (ms_kernels.cu).  All asynchronous on `stream`.
template <typename AT>
cudaError_t launch_src_table(const TableArgs& a, WorkCounters* work, cudaStream_t stream);
cudaError_t launch_active(const ActiveArgs& a, cudaStream_t stream);
cudaError_t launch_fill_f32(float* p, int64_t n, float v, cudaStream_t stream);
// implicit selects the Crank-Nicolson variant (MS_IMPLICIT; only for
// (float, float) and (double, double), cudaErrorNotSupported otherwise).
template <typename AT, typename FT>
cudaError_t launch_track(const TrackArgs<AT, FT>& a, int block_threads, int grid_blocks,
                         cudaStream_t stream, bool implicit = false);
template <typename AT, typename FT>
int track_blocks_per_sm(int block_threads, bool implicit = false);
// The dense launch of one step (no active list, S = 1, FP32 explicit):
// k_track's arithmetic per tile, organised for streaming the state
// (k_track_dense).  cudaErrorInvalidValue unless a.n_levels == 2 and there is
// no tile list.
cudaError_t launch_track_dense(const TrackArgs<float, float>& a, int grid_blocks,
                               cudaStream_t stream);
int track_dense_blocks_per_sm();
int track_dense_grid(int64_t n_tiles, int blocks_per_sm, int sm_count);
// The same FP32 launches with exp2 / log2 on the FMA pipe (ms_kernels_fma.cu,
// MS_FLAG_FMA_TRANSCENDENTALS).
cudaError_t launch_track_fma(const TrackArgs<float, float>& a, int block_threads,
                             int grid_blocks, cudaStream_t stream, bool implicit);
cudaError_t launch_step_ext_fma(const StepArgs<float, float>& a, int block_threads,
                                cudaStream_t stream, bool implicit);
// Verification reductions (k_verify): out[0..2] device doubles.
cudaError_t launch_verify(const double* a, int64_t na, const double* b, int64_t nb, int64_t n,
                          const int64_t* idx, double* out, cudaStream_t stream);

// The correction g on n independent points (device arrays, FP64) at the
// temperatures T[i][0 .. n_T - 1] in turn.
cudaError_t launch_correct(const ModelConstT<double>& m, int64_t n, int n_T, const double* T,
                           double* xas, double* xam, cudaStream_t stream);

// Phase-aware coarsening criterion (ms_coarsen.cu): octants of levels
// 1 .. n_levels (<= MS_COARSEN_MAX_LEVELS) of a grid, their masks (x fastest,
// levels in turn) and the number of coarsenable octants per level (device
// counters).  coarsen_counts fills per_level (may be NULL) and returns the
// total; the scratch holds the per-octant ranges of two levels.
int64_t coarsen_counts(const int32_t dims[3], int n_levels, int64_t* per_level);
size_t coarsen_scratch_bytes(const int32_t dims[3]);
cudaError_t launch_coarsen(const double* xa, const double* xm, const double* xb,
                           const int32_t dims[3], double tol, int n_levels, uint8_t* mask,
                           void* scratch, unsigned long long* n_ok, cudaStream_t stream);

// The stream and the number of points of a context (for the coupled runner).
void* ctx_stream(ms_ctx* c);
int64_t ctx_points(const ms_ctx* c);

// The inference weights of a surrogate (ms_surrogate.cu).
struct MlpDev;
const MlpDev* surrogate_weights(const ms_surrogate* s);
int surrogate_activation(const ms_surrogate* s);   // MS_ACT_GELU or MS_ACT_RELU
int surrogate_stride(const ms_surrogate* s);       // 1, 2, 4, 8 or 16

// Hybrid hot kernel (an attached surrogate; AT = float), one instantiation
// per hidden activation.
template <typename FT>
cudaError_t launch_track_hybrid(const TrackArgs<float, FT>& a, int activation, int grid_blocks,
                                cudaStream_t stream);
template <typename FT>
int hybrid_blocks_per_sm(int activation);
constexpr int HYBRID_THREADS = 256;

template <typename AT, typename FT>
cudaError_t launch_step_ext(const StepArgs<AT, FT>& a, int block_threads, cudaStream_t stream,
                            bool implicit = false);

// Natural-order doubles <-> padded device state (one thread per point).
// xas == nullptr on set fills every point with (xas0, xam0, no initiation).
template <typename FT>
cudaError_t launch_set_state(const SpecDev* specs, const int32_t* tile_spec, int64_t n_tiles,
                             const double* xas, const double* xam, const double* aux,
                             FT* dxas, FT* dxam, float* daux, cudaStream_t stream,
                             double xas0 = 0.9, double xam0 = 0.0);
template <typename FT>
cudaError_t launch_get_state(const SpecDev* specs, const int32_t* tile_spec, int64_t n_tiles,
                             const FT* dxas, const FT* dxam, const float* daux,
                             double* xas, double* xam, double* aux, cudaStream_t stream);

// X_beta and X_liq (and optionally T) in natural order.  Temperatures come
// either from a natural-order array T (external mode) or from level 0 of a
// source table.
template <typename AT, typename FT>
cudaError_t launch_fractions(const ModelConstT<AT>& m, const SpecDev* specs,
                             const int32_t* tile_spec, int64_t n_tiles, const FT* dxas,
                             const FT* dxam, const float* T, const SrcLevelT<AT>* levels,
                             const SrcEntryT<AT>* entries, int32_t slots, double* xbeta,
                             double* xliq, double* T_out, cudaStream_t stream);

}  // namespace ms
