// C ABI of the microstructure point solver (declared in include/ms.h).
//
// The context owns the padded SoA state on the device (X_as, X_am in the
// fraction type, the App. A variable as float), the specimen table, the track
// and layer tables of the moving sources, a per-launch source table and a
// staging buffer for host <-> device copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ms_internal.h"

using ms::LayerDev;
using ms::SpecDev;
using ms::TrackDev;
using ms::TILE;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define MS_CUDA(...)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (__VA_ARGS__);                                                       \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA, "%s: %s (%s:%d)", \
                  #__VA_ARGS__, cudaGetErrorString(e_), __FILE__, __LINE__);              \
  } while (0)

constexpr uint64_t kBlobMagic = 0x4d53434b50543031ull;  // "MSCKPT01"

struct BlobHeader {
  uint64_t magic;
  int64_t n_points;
  int64_t n_pad;
  int32_t precision;
  int32_t reserved;
  int64_t step_n;
  int64_t n_base;
  double t_base;
  double dt;
};

}  // namespace

struct ms_ctx {
  ms_params prm{};
  ms::ModelConstT<float> mc{};     // FP32 arithmetic paths
  ms::ModelConstT<double> mcd{};   // full-FP64 path (MS_F64)
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  int64_t n_points = 0;
  size_t fbytes = 4;  // bytes of the fraction type

  // layout
  std::vector<SpecDev> specs_h;
  SpecDev* specs_d = nullptr;
  int32_t* tile_spec_d = nullptr;
  int64_t n_tiles = 0;
  bool has_grid = false;

  // state (padded)
  void* xas_d = nullptr;
  void* xam_d = nullptr;
  float* aux_d = nullptr;
  int* err_d = nullptr;

  // active set and work distribution of the persistent hot kernel
  int32_t* tile_list_d = nullptr;  // COST_BUCKETS regions of n_tiles entries
  uint32_t* tile_cost_d = nullptr; // per tile: cycles per level when last processed
  int32_t cost_slot = 0;           // parity of the hot-kernel launches
  float* tile_tsat_d = nullptr;
  ms::WorkCounters* work_d = nullptr;
  int sm_count = 0;
  int track_grid = 0;  // persistent grid size for the current layout
  int dense_grid = 0;  // grid of the dense one-step launch (k_track_dense)
  int two_rows = 0;    // some tile lies across two grid rows (k_track's far field for it)

  // attached surrogate (hybrid kernel)
  const ms::MlpDev* mlp = nullptr;
  int32_t mlp_act = MS_ACT_GELU, mlp_stride = 1;
  uint64_t judge_thresh = 0;
  double judge_tol = MS_JUDGE_TOL_DEFAULT;
  ms::HybridCounters* hyb_d = nullptr;
  ms::OpCounters* ops_d = nullptr;       // work done by k_track
  float* ff_d = nullptr;                 // far-field weights and nodes (farfield_dist > 0)
  int hybrid_per_sm = 0;

  // staging
  double* stage_d = nullptr;
  float* Tstage_d = nullptr;
  const float* T_last = nullptr;

  // moving sources
  std::vector<TrackDev> tracks_h;
  std::vector<LayerDev> layers_h;
  TrackDev* tracks_d = nullptr;
  LayerDev* layers_d = nullptr;
  ms::TrackWin* win_d = nullptr;   // the tracks over the current launch's window (active set)
  size_t tracks_cap = 0, layers_cap = 0, win_cap = 0;
  int slots = 0;
  bool src_valid = false;
  void* levels_d = nullptr;        // SrcLevelT<AT> of the context's arithmetic type
  void* entries_d = nullptr;       // SrcEntryT<AT>
  size_t levels_cap = 0, entries_cap = 0;  // bytes
  int64_t* idx_d = nullptr;        // grid indices of a subset specimen

  // time
  int64_t step_n = 0;
  int64_t n_base = 0;
  double t_base = 0.0;
  double dt = 0.0;

  // counters
  ms_stats_t st{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  // per-launch timing of the hot kernel (MS_FLAG_TIME_KERNELS)
  std::vector<cudaEvent_t> kev;  // pairs: start, stop
  size_t kev_used = 0;           // pairs recorded and not yet harvested
  bool capturing = false;        // inside a stream capture (MS_FLAG_GRAPH)

  // captured ms_run_track sequences (MS_FLAG_GRAPH)
  struct Graph {
    int64_t step0, n_steps, n_base;
    double dt, t_base;
    uint64_t epoch;
    size_t kev_pairs;
    int64_t launches;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  uint64_t epoch = 1;            // bumped whenever a captured graph may be stale
};

namespace {

// Calls f with a tag carrying the arithmetic type AT and the fraction type FT
// of the context's precision.
template <typename A, typename F>
struct Tag {
  using at = A;
  using type = F;
};
template <class F>
auto with_ft(const ms_ctx* c, F&& f) {
  switch (c->prm.precision) {
    case MS_F64ACC: return f(Tag<float, double>{});
    case MS_KAHAN: return f(Tag<float, ms::KF>{});
    case MS_F64: return f(Tag<double, double>{});
    default: return f(Tag<float, float>{});
  }
}

template <typename AT>
const ms::ModelConstT<AT>& consts(const ms_ctx* c);
template <>
const ms::ModelConstT<float>& consts<float>(const ms_ctx* c) { return c->mc; }
template <>
const ms::ModelConstT<double>& consts<double>(const ms_ctx* c) { return c->mcd; }

template <typename AT>
ms::ModelConstT<AT> make_const(const ms_params& p) {
  const double l2e = 1.4426950408889634074;
  ms::ModelConstT<AT> m{};
  m.T_s = AT(p.T_s);
  m.T_l = AT(p.T_l);
  m.inv_mushy = AT(1.0 / (p.T_l - p.T_s));
  m.T_as_start = AT(p.T_as_start);
  m.T_as_end = AT(p.T_as_end);
  m.T_am_start = AT(p.T_am_start);
  m.T_inf = AT(p.T_inf);
  m.kaeq_l2 = AT(p.k_alpha_eq * l2e);
  m.kam_l2 = AT(p.k_am_eq * l2e);
  m.k1 = AT(p.k1);
  m.k2 = AT(p.k2);
  m.k3_l2 = AT(p.k3 * l2e);
  m.f = AT(p.f);
  m.c_as = AT(p.c_as);
  m.c_b = AT(p.c_b);
  m.inv_c_as = AT(1.0 / p.c_as);
  m.inv_c_b = AT(1.0 / p.c_b);
  m.pa = AT((p.c_as - 1.0) / p.c_as);
  m.qa = AT((p.c_as + 1.0) / p.c_as);
  m.pb = AT((p.c_b - 1.0) / p.c_b);
  m.qb = AT((p.c_b + 1.0) / p.c_b);
  m.T_cap0 = AT(p.T_as_start + p.T_reg);
  m.inv_T_reg = AT(1.0 / p.T_reg);
  m.init_exit = AT(p.init_exit);
  m.init_exit_floor = AT(p.init_exit_floor);
  m.T_thr = AT(p.T_thr);
  m.martensite_literal = p.martensite_literal ? 1 : 0;
  m.init_ba_steps = p.init_ba_steps ? 1 : 0;
  m.fp_eps_abs = AT(p.fp_eps_abs);
  m.fp_eps_rel = AT(p.fp_eps_rel);
  m.fp_max_iter = p.fp_max_iter;
  return m;
}

int check_params(const ms_params& p) {
  auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
  if (!(pos(p.T_s) && pos(p.T_l) && p.T_l > p.T_s))
    return fail(MS_ERR_INVALID_ARG, "need 0 < T_s < T_l");
  if (!(pos(p.T_as_end) && p.T_as_start > p.T_as_end && pos(p.T_am_start) && pos(p.T_inf)))
    return fail(MS_ERR_INVALID_ARG, "need T_as_end < T_as_start and positive temperatures");
  if (!(pos(p.k_alpha_eq) && pos(p.k_am_eq) && pos(p.k1) && pos(p.k3) && pos(p.f) &&
        std::isfinite(p.k2)))
    return fail(MS_ERR_INVALID_ARG, "rate and equilibrium constants must be positive");
  if (!(p.c_as > 1.0 && p.c_b > 1.0 && std::isfinite(p.c_as) && std::isfinite(p.c_b)))
    return fail(MS_ERR_INVALID_ARG, "c_as and c_b must be > 1");
  if (!pos(p.T_reg)) return fail(MS_ERR_INVALID_ARG, "T_reg must be > 0");
  if (!(std::isfinite(p.init_exit) && p.init_exit >= 0 && std::isfinite(p.init_exit_floor) &&
        p.init_exit_floor >= 0))
    return fail(MS_ERR_INVALID_ARG, "init_exit and init_exit_floor must be >= 0");
  if (!std::isfinite(p.T_thr)) return fail(MS_ERR_INVALID_ARG, "T_thr must be finite");
  if (p.precision != MS_F32 && p.precision != MS_F64ACC && p.precision != MS_KAHAN &&
      p.precision != MS_F64)
    return fail(MS_ERR_INVALID_ARG, "unknown precision %d", p.precision);
  if (p.steps_per_launch < 1 || p.steps_per_launch > ms::MAX_LEVELS - 1)
    return fail(MS_ERR_INVALID_ARG, "steps_per_launch must be in [1, %d]", ms::MAX_LEVELS - 1);
  if (p.block_threads != 0 &&
      (p.block_threads < 32 || p.block_threads > 256 || p.block_threads % 32 != 0))
    return fail(MS_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in [32, 256]");
  if (p.integrator != MS_EXPLICIT && p.integrator != MS_IMPLICIT)
    return fail(MS_ERR_INVALID_ARG, "unknown integrator %d", p.integrator);
  if (p.tile_order != 0 && p.tile_order != 1)
    return fail(MS_ERR_INVALID_ARG, "tile_order must be 0 or 1");
  if ((p.flags & MS_FLAG_FMA_TRANSCENDENTALS) && p.precision != MS_F32)
    return fail(MS_ERR_UNSUPPORTED, "MS_FLAG_FMA_TRANSCENDENTALS needs precision MS_F32");
  if (!(std::isfinite(p.farfield_dist) && p.farfield_dist >= 0.0))
    return fail(MS_ERR_INVALID_ARG, "farfield_dist must be finite and >= 0");
  if (p.integrator == MS_IMPLICIT) {
    if (p.precision != MS_F32 && p.precision != MS_F64)
      return fail(MS_ERR_UNSUPPORTED, "MS_IMPLICIT needs precision MS_F32 or MS_F64");
    if (!(std::isfinite(p.dt_sub) && pos(p.fp_eps_rel) && std::isfinite(p.fp_eps_abs) &&
          p.fp_eps_abs >= 0 && p.fp_max_iter >= 1))
      return fail(MS_ERR_INVALID_ARG, "need finite dt_sub, fp_eps_abs >= 0, fp_eps_rel > 0, fp_max_iter >= 1");
  }
  return MS_OK;
}

// Substeps of the implicit scheme for a step of size dt: ceil(dt / dt_sub),
// at least 1 (the small offset keeps an exact multiple from rounding up).
int32_t n_substeps(const ms_params& p, double dt) {
  if (p.integrator != MS_IMPLICIT || !(p.dt_sub > 0.0)) return 1;
  const double r = std::ceil(dt / p.dt_sub - 1e-9);
  return r < 1.0 ? 1 : (r > 1e9 ? 1000000000 : int32_t(r));
}

int block_threads(const ms_ctx* c) { return c->prm.block_threads ? c->prm.block_threads : 128; }

template <typename T>
int grow(T** p, size_t* cap, size_t n) {
  if (n <= *cap && *p) return MS_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  MS_CUDA(cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T)));
  *cap = n;
  return MS_OK;
}

void drop_graphs(ms_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  c->epoch++;
}

void free_layout(ms_ctx* c) {
  cudaFree(c->tile_list_d);
  cudaFree(c->tile_tsat_d);
  cudaFree(c->tile_cost_d);
  c->tile_cost_d = nullptr;
  c->tile_list_d = nullptr;
  c->tile_tsat_d = nullptr;
  cudaFree(c->specs_d);
  cudaFree(c->tile_spec_d);
  cudaFree(c->xas_d);
  cudaFree(c->xam_d);
  cudaFree(c->aux_d);
  cudaFree(c->stage_d);
  cudaFree(c->Tstage_d);
  c->specs_d = nullptr;
  c->tile_spec_d = nullptr;
  c->xas_d = c->xam_d = nullptr;
  c->aux_d = nullptr;
  c->stage_d = nullptr;
  c->Tstage_d = nullptr;
  c->T_last = nullptr;
}

// (Re)build the padded layout for the current specs_h and reset the state.
int build_layout(ms_ctx* c) {
  drop_graphs(c);
  free_layout(c);
  int64_t tiles = 0, pad = 0, nat = 0;
  for (auto& s : c->specs_h) {
    s.nat_off = nat;
    s.pad_off = pad;
    s.tile0 = tiles;
    s.n_tiles = int32_t((s.n + TILE - 1) / TILE);
    tiles += s.n_tiles;
    pad += int64_t(s.n_tiles) * TILE;
    nat += s.n;
  }
  if (tiles > INT32_MAX / 2) return fail(MS_ERR_INVALID_ARG, "too many points (%lld tiles)", (long long)tiles);
  c->n_tiles = tiles;
  c->two_rows = 0;
  for (const auto& sp : c->specs_h)
    if (!sp.idx && sp.nx % TILE != 0 && int64_t(sp.ny) * sp.nz > 1) c->two_rows = 1;
  std::vector<int32_t> ts(static_cast<size_t>(tiles));
  for (size_t s = 0; s < c->specs_h.size(); ++s)
    for (int32_t t = 0; t < c->specs_h[s].n_tiles; ++t) ts[size_t(c->specs_h[s].tile0 + t)] = int32_t(s);
  const size_t np = size_t(pad);
  MS_CUDA(cudaMalloc(&c->specs_d, c->specs_h.size() * sizeof(SpecDev)));
  MS_CUDA(cudaMalloc(&c->tile_spec_d, ts.size() * sizeof(int32_t)));
  MS_CUDA(cudaMalloc(&c->xas_d, np * c->fbytes));
  MS_CUDA(cudaMalloc(&c->xam_d, np * c->fbytes));
  MS_CUDA(cudaMalloc(&c->aux_d, np * sizeof(float)));
  MS_CUDA(cudaMalloc(&c->stage_d, size_t(c->n_points) * 4 * sizeof(double)));
  MS_CUDA(cudaMalloc(&c->tile_list_d, size_t(tiles) * ms::COST_BUCKETS * sizeof(int32_t)));
  MS_CUDA(cudaMalloc(&c->tile_cost_d, size_t(tiles) * sizeof(uint32_t)));
  MS_CUDA(cudaMemset(c->tile_cost_d, 0, size_t(tiles) * sizeof(uint32_t)));
  MS_CUDA(cudaMalloc(&c->tile_tsat_d, size_t(tiles) * sizeof(float)));
  MS_CUDA(ms::launch_fill_f32(c->tile_tsat_d, tiles, INFINITY, c->stream));
  {
    const int bt = block_threads(c);
    const int per_sm = with_ft(c, [&](auto tag) {
      return ms::track_blocks_per_sm<typename decltype(tag)::at, typename decltype(tag)::type>(
          bt, c->prm.integrator == MS_IMPLICIT);
    });
    const int64_t need = (tiles + bt / 32 - 1) / (bt / 32);
    c->track_grid = int(std::min<int64_t>(int64_t(per_sm) * c->sm_count, need));
    c->dense_grid = ms::track_dense_grid(tiles, ms::track_dense_blocks_per_sm(), c->sm_count);
  }
  MS_CUDA(cudaMemcpy(c->specs_d, c->specs_h.data(), c->specs_h.size() * sizeof(SpecDev),
                     cudaMemcpyHostToDevice));
  MS_CUDA(cudaMemcpy(c->tile_spec_d, ts.data(), ts.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  MS_CUDA(with_ft(c, [&](auto tag) {
      using FT = typename decltype(tag)::type;
      return ms::launch_set_state<FT>(c->specs_d, c->tile_spec_d, c->n_tiles, nullptr, nullptr,
                                        nullptr, (FT*)c->xas_d, (FT*)c->xam_d, c->aux_d,
                                        c->stream);
    }));
  MS_CUDA(cudaStreamSynchronize(c->stream));
  c->step_n = c->n_base = 0;
  c->t_base = 0.0;
  c->src_valid = false;
  return MS_OK;
}

// Record the start (second == false) or stop event of a timed hot-kernel launch.
int kernel_event(ms_ctx* c, bool stop) {
  if (!(c->prm.flags & MS_FLAG_TIME_KERNELS)) return MS_OK;
  const size_t i = 2 * c->kev_used + (stop ? 1 : 0);
  while (c->kev.size() <= i) {
    cudaEvent_t e;
    MS_CUDA(cudaEventCreate(&e));
    c->kev.push_back(e);
  }
  if (c->capturing)
    MS_CUDA(cudaEventRecordWithFlags(c->kev[i], c->stream, cudaEventRecordExternal));
  else
    MS_CUDA(cudaEventRecord(c->kev[i], c->stream));
  if (stop) c->kev_used++;
  return MS_OK;
}


// Add the recorded launch times to the counters (stream already synchronised).
int harvest_kernel_events(ms_ctx* c) {
  for (size_t p = 0; p < c->kev_used; ++p) {
    float ms_ = 0.f;
    MS_CUDA(cudaEventElapsedTime(&ms_, c->kev[2 * p], c->kev[2 * p + 1]));
    c->st.hot_kernel_ms += ms_;
    c->st.hot_kernel_launches++;
  }
  c->kev_used = 0;
  return MS_OK;
}

int check_device_error(ms_ctx* c) {
  int err = 0;
  ms::WorkCounters wc{};
  MS_CUDA(cudaMemcpyAsync(&err, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MS_CUDA(cudaMemcpyAsync(&wc, c->work_d, sizeof(wc), cudaMemcpyDeviceToHost, c->stream));
  MS_CUDA(cudaStreamSynchronize(c->stream));
  c->st.device_error = err;
  c->st.tile_steps_active = int64_t(wc.tile_steps_active);
  if (c->ops_d) {
    ms::OpCounters oc{};
    MS_CUDA(cudaMemcpy(&oc, c->ops_d, sizeof(oc), cudaMemcpyDeviceToHost));
    c->st.source_evaluations = int64_t(oc.source_evaluations);
    c->st.model_point_steps = int64_t(oc.model_point_steps);
    c->st.fp_iterations = int64_t(oc.fp_iterations);
    c->st.fp_unconverged = int64_t(oc.fp_unconverged);
    c->st.model_sfu_ex2 = int64_t(oc.model_sfu_ex2);
    c->st.model_sfu_slow = int64_t(oc.model_sfu_slow);
    c->st.farfield_node_evaluations = int64_t(oc.farfield_node_evaluations);
    c->st.farfield_point_sources = int64_t(oc.farfield_point_sources);
  }
  if (c->hyb_d) {
    ms::HybridCounters hc{};
    MS_CUDA(cudaMemcpy(&hc, c->hyb_d, sizeof(hc), cudaMemcpyDeviceToHost));
    c->st.surrogate_windows = int64_t(hc.surrogate_windows);
    c->st.ode_windows = int64_t(hc.ode_windows);
    c->st.judge_samples = int64_t(hc.judge_samples);
    float e = 0.f;
    std::memcpy(&e, &hc.judge_err_bits, sizeof(e));
    c->st.judge_max_err = double(e);
    c->st.judge_rejected = int64_t(hc.judge_rejected);
  }
  if (c->timed) {
    float ms_ = 0.f;
    if (cudaEventElapsedTime(&ms_, c->ev0, c->ev1) == cudaSuccess) c->st.last_run_ms = ms_;
    c->timed = false;
  }
  int rc = harvest_kernel_events(c);
  if (rc != MS_OK) return rc;
  if (err & ms::DEVERR_NONFINITE) return fail(MS_ERR_NONFINITE, "a fraction became non-finite");
  if (err & ms::DEVERR_TIMEOUT) return fail(MS_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up");
  return MS_OK;
}

// Upload the heat sources if they differ from the cached copy.
int set_sources(ms_ctx* c, const ms_heat_source* src) {
  std::vector<TrackDev> tr;
  std::vector<LayerDev> ly;
  std::vector<SpecDev> specs = c->specs_h;
  int slots = 1;
  for (size_t s = 0; s < specs.size(); ++s) {
    const ms_heat_source& h = src[s];
    if (!(std::isfinite(h.A) && h.A >= 0 && h.k > 0 && h.alpha > 0 && std::isfinite(h.T0) &&
          h.T0 > 0 && h.T_max > h.T0 && std::isfinite(h.t_offset) && h.z_tol >= 0 &&
          h.n_tracks >= 0 && h.n_layers >= 1 && h.layers && (h.n_tracks == 0 || h.tracks)))
      return fail(MS_ERR_INVALID_ARG, "invalid heat source of specimen %zu", s);
    specs[s].A = h.A;
    specs[s].k = h.k;
    specs[s].alpha = h.alpha;
    specs[s].t_offset = h.t_offset;
    specs[s].T0 = float(h.T0);
    specs[s].T_max = float(h.T_max);
    specs[s].z_tol = float(h.z_tol);
    specs[s].track0 = int32_t(tr.size());
    specs[s].n_tracks = h.n_tracks;
    specs[s].layer0 = int32_t(ly.size());
    specs[s].n_layers = h.n_layers;
    std::vector<int> per_layer(size_t(h.n_layers), 0);
    for (int j = 0; j < h.n_tracks; ++j) {
      const ms_track& t = h.tracks[j];
      const double un = std::sqrt(t.ux * t.ux + t.uy * t.uy);
      if (!(t.layer >= 0 && t.layer < h.n_layers && std::fabs(un - 1.0) < 1e-6 && t.v > 0 &&
            std::isfinite(t.v) && t.P >= 0 && std::isfinite(t.P) && std::isfinite(t.x0) &&
            std::isfinite(t.y0) && std::isfinite(t.t_start)))
        return fail(MS_ERR_INVALID_ARG, "invalid track %d of specimen %zu", j, s);
      tr.push_back(TrackDev{t.x0, t.y0, t.ux, t.uy, t.v, t.P, t.t_start, t.layer, int32_t(s)});
      slots = std::max(slots, ++per_layer[size_t(t.layer)]);
    }
    for (int j = 0; j < h.n_layers; ++j) {
      const ms_layer& L = h.layers[j];
      if (!(std::isfinite(L.z_surface) && L.t_scan_end >= L.t_begin && L.t_end >= L.t_scan_end))
        return fail(MS_ERR_INVALID_ARG, "invalid layer %d of specimen %zu", j, s);
      ly.push_back(LayerDev{L.z_surface, L.t_begin, L.t_scan_end, L.t_end});
    }
  }
  const bool same = c->src_valid && slots == c->slots && tr.size() == c->tracks_h.size() &&
                    ly.size() == c->layers_h.size() &&
                    std::memcmp(specs.data(), c->specs_h.data(), specs.size() * sizeof(SpecDev)) == 0 &&
                    (tr.empty() || std::memcmp(tr.data(), c->tracks_h.data(), tr.size() * sizeof(TrackDev)) == 0) &&
                    std::memcmp(ly.data(), c->layers_h.data(), ly.size() * sizeof(LayerDev)) == 0;
  if (same) return MS_OK;
  MS_CUDA(cudaStreamSynchronize(c->stream));  // previous launches may still read the tables
  drop_graphs(c);
  int rc;
  if ((rc = grow(&c->tracks_d, &c->tracks_cap, tr.size())) != MS_OK) return rc;
  if ((rc = grow(&c->win_d, &c->win_cap, tr.size())) != MS_OK) return rc;
  if ((rc = grow(&c->layers_d, &c->layers_cap, ly.size())) != MS_OK) return rc;
  if (!tr.empty())
    MS_CUDA(cudaMemcpy(c->tracks_d, tr.data(), tr.size() * sizeof(TrackDev), cudaMemcpyHostToDevice));
  MS_CUDA(cudaMemcpy(c->layers_d, ly.data(), ly.size() * sizeof(LayerDev), cudaMemcpyHostToDevice));
  MS_CUDA(cudaMemcpy(c->specs_d, specs.data(), specs.size() * sizeof(SpecDev), cudaMemcpyHostToDevice));
  c->specs_h = specs;
  c->tracks_h = tr;
  c->layers_h = ly;
  c->slots = slots;
  c->src_valid = true;
  return MS_OK;
}

int ensure_table(ms_ctx* c, int n_levels) {
  int rc;
  const size_t ns = c->specs_h.size();
  const bool f64 = c->prm.precision == MS_F64;
  const size_t lb = ns * size_t(n_levels) *
                    (f64 ? sizeof(ms::SrcLevelT<double>) : sizeof(ms::SrcLevelT<float>));
  const size_t eb = ns * size_t(n_levels) * size_t(c->slots) *
                    (f64 ? sizeof(ms::SrcEntryT<double>) : sizeof(ms::SrcEntryT<float>));
  if (lb > c->levels_cap || eb > c->entries_cap) drop_graphs(c);
  if ((rc = grow(reinterpret_cast<char**>(&c->levels_d), &c->levels_cap, lb)) != MS_OK) return rc;
  if ((rc = grow(reinterpret_cast<char**>(&c->entries_d), &c->entries_cap, eb)) != MS_OK) return rc;
  return MS_OK;
}

double level_time(const ms_ctx* c, int64_t level) {
  return c->t_base + double(level - c->n_base) * c->dt;
}

// The source table of levels level0 .. level0 + n_levels - 1; with_window
// also writes every track's path over that window for the active set.
int launch_table(ms_ctx* c, int64_t level0, int n_levels, bool with_window = false) {
  ms::TableArgs ta{};
  ta.specs = c->specs_d;
  ta.tracks = c->tracks_d;
  ta.layers = c->layers_d;
  ta.n_specs = int32_t(c->specs_h.size());
  ta.n_levels = n_levels;
  ta.slots = c->slots;
  ta.n0 = level0 - c->n_base;
  ta.t_base = c->t_base;
  ta.dt = c->dt;
  ta.levels = c->levels_d;
  ta.entries = c->entries_d;
  ta.ff_dist = c->ff_d && c->prm.precision != MS_F64 ? c->prm.farfield_dist : 0.0;
  if (with_window && !c->tracks_h.empty()) {
    ta.win = c->win_d;
    ta.n_tracks = int32_t(c->tracks_h.size());
    ta.t_a = level_time(c, level0);
    ta.t_b = level_time(c, level0 + n_levels - 1);
  }
  if (c->prm.precision == MS_F64)
    MS_CUDA(ms::launch_src_table<double>(ta, c->work_d, c->stream));
  else
    MS_CUDA(ms::launch_src_table<float>(ta, c->work_d, c->stream));
  c->st.launches++;
  return MS_OK;
}


template <typename AT, typename FT>
int run_track_impl(ms_ctx* c, int64_t n_steps) {
  const int S = c->prm.steps_per_launch;
  const bool use_list = c->prm.T_thr > 0.0;
  int rc;
  if ((rc = ensure_table(c, S + 1)) != MS_OK) return rc;
  int64_t left = n_steps;
  while (left > 0) {
    const int steps = int(std::min<int64_t>(S, left));
    if ((rc = launch_table(c, c->step_n, steps + 1, use_list)) != MS_OK) return rc;
    if (use_list) {
      ms::ActiveArgs aa{};
      aa.specs = c->specs_d;
      aa.win = c->tracks_h.empty() ? nullptr : c->win_d;
      aa.tile_spec = c->tile_spec_d;
      aa.tile_tsat = c->tile_tsat_d;
      aa.n_tiles = int32_t(c->n_tiles);
      aa.T_thr = c->prm.T_thr;
      aa.T_as_end = c->prm.T_as_end;
      aa.tile_list = c->tile_list_d;
      aa.work = c->work_d;
      aa.tile_cost = c->prm.tile_order == 0 ? c->tile_cost_d : nullptr;
      aa.prev_slot = c->cost_slot ^ 1;
      MS_CUDA(ms::launch_active(aa, c->stream));
      c->st.launches++;
    }
    ms::TrackArgs<AT, FT> a{};
    a.m = consts<AT>(c);
    a.specs = c->specs_d;
    a.tile_spec = c->tile_spec_d;
    a.tile_list = use_list ? c->tile_list_d : nullptr;
    a.work = c->work_d;
    a.n_tiles = int32_t(c->n_tiles);
    a.n_levels = steps + 1;
    a.slots = c->slots;
    a.dt = AT(c->dt);
    a.levels = static_cast<const ms::SrcLevelT<AT>*>(c->levels_d);
    a.entries = static_cast<const ms::SrcEntryT<AT>*>(c->entries_d);
    a.xas = (FT*)c->xas_d;
    a.xam = (FT*)c->xam_d;
    a.aux = c->aux_d;
    a.tile_tsat = c->tile_tsat_d;
    a.err = c->err_d;
    a.ops = c->ops_d;
    if (use_list && c->prm.tile_order == 0) {
      a.tile_cost = c->tile_cost_d;
      a.cost_slot = c->cost_slot;
    }
    a.n_sub = n_substeps(c->prm, c->dt);
    a.count_sfu = (c->prm.flags & MS_FLAG_COUNT_OPS) ? 1 : 0;
    if constexpr (std::is_same<AT, float>::value) {
      a.ff = c->ff_d;
      a.ff_dist = float(c->prm.farfield_dist);
      a.two_rows = c->two_rows;
    }
    if ((rc = kernel_event(c, false)) != MS_OK) return rc;
    bool hybrid = false;
    if constexpr (std::is_same<AT, float>::value &&
                  (std::is_same<FT, float>::value || std::is_same<FT, ms::KF>::value)) {
      if (c->mlp) {
        a.mlp = c->mlp;
        a.hyb = c->hyb_d;
        a.judge_thresh = c->judge_thresh;
        a.judge_tol = c->judge_tol < 3.0e38 ? float(c->judge_tol) : INFINITY;
        a.level0 = c->step_n;
        a.mlp_stride = c->mlp_stride;
        const int64_t need = (c->n_tiles + ms::HYBRID_THREADS / 32 - 1) / (ms::HYBRID_THREADS / 32);
        const int grid = int(std::min<int64_t>(int64_t(c->hybrid_per_sm) * c->sm_count, need));
        MS_CUDA(ms::launch_track_hybrid<FT>(a, c->mlp_act, grid, c->stream));
        hybrid = true;
      }
    }
    if (!hybrid) {
      bool fma = false;
      if constexpr (std::is_same<AT, float>::value && std::is_same<FT, float>::value) {
        if (c->prm.flags & MS_FLAG_FMA_TRANSCENDENTALS) {
          MS_CUDA(ms::launch_track_fma(a, block_threads(c), c->track_grid, c->stream,
                                       c->prm.integrator == MS_IMPLICIT));
          fma = true;
        }
      }
      bool dense = false;
      if constexpr (std::is_same<AT, float>::value && std::is_same<FT, float>::value) {
        // one explicit step over every tile: the streaming form of the same step
        if (!fma && !use_list && steps == 1 && c->prm.integrator != MS_IMPLICIT &&
            !a.count_sfu) {
          MS_CUDA(ms::launch_track_dense(a, c->dense_grid, c->stream));
          dense = true;
        }
      }
      if (!fma && !dense)
        MS_CUDA(ms::launch_track<AT, FT>(a, block_threads(c), c->track_grid, c->stream,
                                         c->prm.integrator == MS_IMPLICIT));
    }
    if ((rc = kernel_event(c, true)) != MS_OK) return rc;
    c->st.launches++;
    c->cost_slot ^= 1;
    c->step_n += steps;
    c->st.steps += steps;
    c->st.point_updates += int64_t(steps) * c->n_points;
    c->st.tile_steps_total += int64_t(steps) * c->n_tiles;
    left -= steps;
  }
  return MS_OK;
}

template <typename AT, typename FT>
int step_impl(ms_ctx* c, const float* T0, const float* T1) {
  ms::StepArgs<AT, FT> a{};
  a.m = consts<AT>(c);
  a.n = c->n_points;
  a.dt = AT(c->dt);
  a.T0 = T0;
  a.T1 = T1;
  a.xas = (FT*)c->xas_d;
  a.xam = (FT*)c->xam_d;
  a.aux = c->aux_d;
  a.err = c->err_d;
  int rc;
  if ((rc = kernel_event(c, false)) != MS_OK) return rc;
  a.ops = c->ops_d;
  a.n_sub = n_substeps(c->prm, c->dt);
  bool fma = false;
  if constexpr (std::is_same<AT, float>::value && std::is_same<FT, float>::value) {
    if (c->prm.flags & MS_FLAG_FMA_TRANSCENDENTALS) {
      MS_CUDA(ms::launch_step_ext_fma(a, block_threads(c), c->stream,
                                      c->prm.integrator == MS_IMPLICIT));
      fma = true;
    }
  }
  if (!fma)
    MS_CUDA(ms::launch_step_ext<AT, FT>(a, block_threads(c), c->stream,
                                        c->prm.integrator == MS_IMPLICIT));
  if ((rc = kernel_event(c, true)) != MS_OK) return rc;
  c->st.launches++;
  return MS_OK;
}

void set_dt(ms_ctx* c, double dt) {
  if (c->dt != dt) {
    c->t_base += double(c->step_n - c->n_base) * c->dt;
    c->n_base = c->step_n;
    c->dt = dt;
  }
}

}  // namespace

namespace {

// Capture (first time) or replay the launch sequence of one ms_run_track call.
int run_track_graph(ms_ctx* c, int64_t n_steps) {
  int rc;
  const bool timing = (c->prm.flags & MS_FLAG_TIME_KERNELS) != 0;
  if (timing && c->kev_used) {  // pending launch timings use the same events
    MS_CUDA(cudaStreamSynchronize(c->stream));
    if ((rc = harvest_kernel_events(c)) != MS_OK) return rc;
  }
  if ((rc = ensure_table(c, c->prm.steps_per_launch + 1)) != MS_OK) return rc;
  ms_ctx::Graph* g = nullptr;
  for (auto& e : c->graphs)
    if (e.step0 == c->step_n && e.n_steps == n_steps && e.n_base == c->n_base && e.dt == c->dt &&
        e.t_base == c->t_base && e.epoch == c->epoch)
      g = &e;
  if (!g) {
    const int64_t step_n = c->step_n;
    const ms_stats_t st = c->st;
    MS_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    c->kev_used = 0;
    rc = with_ft(c, [&](auto tag) { return run_track_impl<typename decltype(tag)::at, typename decltype(tag)::type>(c, n_steps); });
    c->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
    const int64_t launches = c->st.launches - st.launches;
    const size_t pairs = c->kev_used;
    c->step_n = step_n;  // nothing ran yet
    c->st = st;
    c->kev_used = 0;
    if (rc != MS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return fail(MS_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(ec));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(MS_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    if (c->graphs.size() >= 4) {
      cudaGraphExecDestroy(c->graphs.front().exec);
      c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back(ms_ctx::Graph{c->step_n, n_steps, c->n_base, c->dt, c->t_base, c->epoch,
                                      pairs, launches, exec});
    g = &c->graphs.back();
  }
  MS_CUDA(cudaEventRecord(c->ev0, c->stream));
  MS_CUDA(cudaGraphLaunch(g->exec, c->stream));
  MS_CUDA(cudaEventRecord(c->ev1, c->stream));
  c->timed = true;
  c->step_n += n_steps;
  c->st.steps += n_steps;
  c->st.point_updates += n_steps * c->n_points;
  c->st.tile_steps_total += n_steps * c->n_tiles;
  c->st.launches += g->launches;
  if (timing) {
    c->kev_used = g->kev_pairs;  // this replay re-recorded them
    MS_CUDA(cudaStreamSynchronize(c->stream));
    if ((rc = harvest_kernel_events(c)) != MS_OK) return rc;
  }
  return MS_OK;
}

}  // namespace

// Shared with other translation units (declared in ms_internal.h).
namespace ms {
int validate_params(const ms_params& p) { return check_params(p); }
template <typename AT>
ModelConstT<AT> model_const(const ms_params& p) { return make_const<AT>(p); }
template ModelConstT<float> model_const<float>(const ms_params&);
template ModelConstT<double> model_const<double>(const ms_params&);
int record_error(int code, const char* msg) { return fail(code, "%s", msg); }
void* ctx_stream(ms_ctx* c) { return c->stream; }
int64_t ctx_points(const ms_ctx* c) { return c->n_points; }
}  // namespace ms

// =============================================================== C ABI
// Far-field interpolation table: the 8 Chebyshev points of the first kind on
// [0, 1] (the tile's x-range from its first to its 128th point), and for
// each node k and each point i at t_i = i / 127 the Lagrange weight
// l_k(t_i) = prod_{j != k} (t_i - s_j) / (s_k - s_j), computed in double.
static std::vector<float> farfield_weights() {
  constexpr int K = ms::FF_NODES, N = ms::TILE;
  const double pi = 3.14159265358979323846;
  double sn[K];
  for (int k = 0; k < K; ++k) sn[k] = 0.5 * (1.0 - std::cos((2 * k + 1) * pi / (2 * K)));
  std::vector<float> w(ms::FF_FLOATS, 0.0f);
  for (int k = 0; k < K; ++k) {
    for (int i = 0; i < N; ++i) {
      const double t = double(i) / double(N - 1);
      double l = 1.0;
      for (int j = 0; j < K; ++j)
        if (j != k) l *= (t - sn[j]) / (sn[k] - sn[j]);
      w[size_t(k) * N + i] = float(l);
    }
    w[size_t(K) * N + k] = float(sn[k]);
  }
  return w;
}

extern "C" {

const char* ms_version(void) { return "ms-gb300 1.0.0 (sm_103a)"; }

const char* ms_strerror(int code) {
  switch (code) {
    case MS_OK: return "ok";
    case MS_ERR_INVALID_ARG: return "invalid argument";
    case MS_ERR_OOM: return "out of memory";
    case MS_ERR_CUDA: return "CUDA error";
    case MS_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case MS_ERR_NONFINITE: return "non-finite fraction";
    case MS_ERR_STATE: return "call out of order";
    case MS_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

const char* ms_last_error(void) { return g_last_error.c_str(); }

int ms_farfield_table(float* out, int32_t n_out) {
  static_assert(ms::FF_FLOATS == MS_FF_TABLE_FLOATS, "table size");
  if (!out || n_out < ms::FF_FLOATS)
    return fail(MS_ERR_INVALID_ARG, "need a table of at least %d floats", ms::FF_FLOATS);
  const std::vector<float> w = farfield_weights();
  std::copy(w.begin(), w.end(), out);
  return MS_OK;
}

size_t ms_struct_size(int which) {
  switch (which) {
    case 0: return sizeof(ms_params);
    case 1: return sizeof(ms_grid);
    case 2: return sizeof(ms_track);
    case 3: return sizeof(ms_layer);
    case 4: return sizeof(ms_heat_source);
    case 5: return sizeof(ms_stats_t);
    case 6: return sizeof(ms_thermal_params);
    default: return 0;
  }
}

int ms_params_check(const ms_params* p) {
  if (!p) return fail(MS_ERR_INVALID_ARG, "params is NULL");
  return check_params(*p);
}

int ms_params_default(ms_params* p) {
  if (!p) return fail(MS_ERR_INVALID_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->T_s = 1878.0;          // Table 1 / Table 2
  p->T_l = 1928.0;
  p->T_as_start = 1273.0;   // Table 2
  p->T_as_end = 935.0;
  p->T_am_start = 848.0;
  p->T_inf = 293.0;
  p->k_alpha_eq = 0.0068;
  p->k_am_eq = 0.00415;
  p->c_as = 2.51;           // Table 3
  p->c_b = 11.0;
  p->k1 = 0.294;
  p->k2 = 850.0;
  p->k3 = 0.0337;
  p->f = 3.8;
  p->T_reg = 100.0;         // Sec. 2.2
  p->init_exit = 1e-15;     // App. A
  p->init_exit_floor = 1e-3;
  p->T_thr = 0.0;
  p->martensite_literal = 0;
  p->init_ba_steps = 0;
  p->precision = MS_F32;
  p->steps_per_launch = 128;
  p->rebuild_steps = 0;
  p->block_threads = 0;
  p->integrator = MS_EXPLICIT;
  p->dt_sub = 0.01;         // Sec. 3: substeps of at most 0.01 s
  p->fp_eps_abs = 1e-10;    // Sec. 3: WRMS tolerances
  p->fp_eps_rel = 1e-3;
  p->fp_max_iter = 100;
  p->farfield_dist = 5e-3;  // receding sources >= 5 mm behind a row tile: interpolated
  return MS_OK;
}

int ms_create(const ms_params* p, int64_t n_points, ms_ctx** out) {
  if (!p || !out) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (n_points <= 0) return fail(MS_ERR_INVALID_ARG, "n_points must be > 0");
  int rc = check_params(*p);
  if (rc != MS_OK) return rc;
  ms_ctx* c = new (std::nothrow) ms_ctx();
  if (!c) return fail(MS_ERR_OOM, "host allocation failed");
  c->prm = *p;
  c->mc = make_const<float>(*p);
  c->mcd = make_const<double>(*p);
  c->fbytes = p->precision == MS_F32 ? 4 : 8;  // MS_KAHAN stores two floats per fraction
  c->n_points = n_points;
  auto bail = [&](int code) { ms_destroy(c); return code; };
  if (cudaGetDevice(&c->device) != cudaSuccess)
    return bail(fail(MS_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(cudaGetLastError())));
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(MS_ERR_CUDA, "stream creation failed"));
  c->stream = c->own_stream;
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess)
    return bail(fail(MS_ERR_CUDA, "event creation failed"));
  if (cudaMalloc(&c->err_d, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->err_d, 0, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->work_d, sizeof(ms::WorkCounters)) != cudaSuccess ||
      cudaMemset(c->work_d, 0, sizeof(ms::WorkCounters)) != cudaSuccess ||
      cudaMalloc(&c->ops_d, sizeof(ms::OpCounters)) != cudaSuccess ||
      cudaMemset(c->ops_d, 0, sizeof(ms::OpCounters)) != cudaSuccess)
    return bail(fail(MS_ERR_OOM, "device allocation failed"));
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return bail(fail(MS_ERR_CUDA, "cannot query the SM count"));
  if (p->farfield_dist > 0.0 && p->precision != MS_F64) {  // the FP64 path sums directly
    const std::vector<float> w = farfield_weights();
    if (cudaMalloc(&c->ff_d, w.size() * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(c->ff_d, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(MS_ERR_OOM, "device allocation failed"));
  }
  SpecDev s{};
  s.nx = int32_t(std::min<int64_t>(n_points, INT32_MAX));
  s.ny = s.nz = 1;
  s.n = n_points;
  c->specs_h.assign(1, s);
  if ((rc = build_layout(c)) != MS_OK) return bail(rc);
  *out = c;
  return MS_OK;
}

void ms_destroy(ms_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  free_layout(c);
  cudaFree(c->idx_d);
  cudaFree(c->err_d);
  cudaFree(c->work_d);
  cudaFree(c->hyb_d);
  cudaFree(c->ops_d);
  cudaFree(c->ff_d);
  cudaFree(c->tracks_d);
  cudaFree(c->win_d);
  cudaFree(c->layers_d);
  cudaFree(c->levels_d);
  cudaFree(c->entries_d);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (cudaEvent_t e : c->kev) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

int ms_set_stream(ms_ctx* c, void* stream) {
  if (!c) return fail(MS_ERR_INVALID_ARG, "NULL context");
  MS_CUDA(cudaStreamSynchronize(c->stream));
  c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
  return MS_OK;
}

int ms_set_points(ms_ctx* c, const ms_grid* grids, int32_t n_specimens) {
  if (!c || !grids || n_specimens <= 0) return fail(MS_ERR_INVALID_ARG, "NULL grids or n_specimens <= 0");
  std::vector<SpecDev> specs;
  int64_t total = 0;
  for (int32_t s = 0; s < n_specimens; ++s) {
    const ms_grid& g = grids[s];
    if (g.dims[0] < 1 || g.dims[1] < 1 || g.dims[2] < 1 || g.k_offset < 0)
      return fail(MS_ERR_INVALID_ARG, "grid %d: dims must be >= 1 and k_offset >= 0", s);
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(g.origin[a]) || !std::isfinite(g.spacing[a]))
        return fail(MS_ERR_INVALID_ARG, "grid %d: non-finite origin or spacing", s);
    SpecDev d{};
    d.ox = double(float(g.origin[0])); d.oy = double(float(g.origin[1]));
    d.oz = double(float(g.origin[2]));
    d.dx = double(float(g.spacing[0])); d.dy = double(float(g.spacing[1]));
    d.dz = double(float(g.spacing[2]));
    if (c->prm.precision == MS_F64) {  // full-FP64 coordinates
      d.ox = g.origin[0]; d.oy = g.origin[1]; d.oz = g.origin[2];
      d.dx = g.spacing[0]; d.dy = g.spacing[1]; d.dz = g.spacing[2];
    }
    d.nx = g.dims[0]; d.ny = g.dims[1]; d.nz = g.dims[2];
    d.k_off = g.k_offset;
    d.n = int64_t(g.dims[0]) * g.dims[1] * g.dims[2];
    d.n_layers = 1;
    total += d.n;
    specs.push_back(d);
  }
  if (total != c->n_points)
    return fail(MS_ERR_INVALID_ARG, "grids hold %lld points, context has %lld", (long long)total,
                (long long)c->n_points);
  MS_CUDA(cudaStreamSynchronize(c->stream));
  c->specs_h = specs;
  c->has_grid = true;
  return build_layout(c);
}


int ms_set_points_subset(ms_ctx* c, const ms_grid* grid, const int64_t* idx, int64_t n) {
  if (!c || !grid || !idx) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  if (n != c->n_points) return fail(MS_ERR_INVALID_ARG, "subset has %lld points, context %lld",
                                    (long long)n, (long long)c->n_points);
  int rc;
  if ((rc = ms_set_points(c, grid, 1)) == MS_ERR_INVALID_ARG && grid->dims[0] >= 1) {
    // the grid holds more points than the subset: set it up by hand
  } else if (rc != MS_OK && rc != MS_ERR_INVALID_ARG) {
    return rc;
  }
  const int64_t total = int64_t(grid->dims[0]) * grid->dims[1] * grid->dims[2];
  if (grid->dims[0] < 1 || grid->dims[1] < 1 || grid->dims[2] < 1 || grid->k_offset < 0)
    return fail(MS_ERR_INVALID_ARG, "grid dims must be >= 1 and k_offset >= 0");
  for (int64_t i = 0; i < n; ++i)
    if (idx[i] < 0 || idx[i] >= total)
      return fail(MS_ERR_INVALID_ARG, "subset index %lld out of the grid", (long long)idx[i]);
  MS_CUDA(cudaStreamSynchronize(c->stream));
  cudaFree(c->idx_d);
  c->idx_d = nullptr;
  MS_CUDA(cudaMalloc(&c->idx_d, size_t(n) * sizeof(int64_t)));
  MS_CUDA(cudaMemcpy(c->idx_d, idx, size_t(n) * sizeof(int64_t), cudaMemcpyHostToDevice));
  SpecDev d{};
  d.ox = double(float(grid->origin[0])); d.oy = double(float(grid->origin[1]));
  d.oz = double(float(grid->origin[2]));
  d.dx = double(float(grid->spacing[0])); d.dy = double(float(grid->spacing[1]));
  d.dz = double(float(grid->spacing[2]));
  if (c->prm.precision == MS_F64) {
    d.ox = grid->origin[0]; d.oy = grid->origin[1]; d.oz = grid->origin[2];
    d.dx = grid->spacing[0]; d.dy = grid->spacing[1]; d.dz = grid->spacing[2];
  }
  d.nx = grid->dims[0]; d.ny = grid->dims[1]; d.nz = grid->dims[2];
  d.k_off = grid->k_offset;
  d.n = n;
  d.n_layers = 1;
  d.idx = c->idx_d;
  c->specs_h.assign(1, d);
  c->has_grid = true;
  return build_layout(c);
}

int ms_set_state(ms_ctx* c, const double* xas, const double* xam, const double* aux) {
  if (!c || !xas || !xam) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  const int64_t n = c->n_points;
  for (int64_t i = 0; i < n; ++i) {
    const double a = xas[i], m = xam[i];
    if (!std::isfinite(a) || !std::isfinite(m)) return fail(MS_ERR_NONFINITE, "point %lld: non-finite fraction", (long long)i);
    if (a < 0 || m < 0 || a + m > 0.9 + 1e-6)
      return fail(MS_ERR_INVALID_ARG, "point %lld: need X_as, X_am >= 0 and X_as + X_am <= 0.9", (long long)i);
    if (aux) {
      const double v = aux[i];
      if (!(v == 0.0 || v == -1.0 || (v > 0.0 && v < 0.9)))
        return fail(MS_ERR_INVALID_ARG, "point %lld: aux must be 0, -1 or in (0, 0.9)", (long long)i);
    }
  }
  MS_CUDA(cudaStreamSynchronize(c->stream));
  double* d = c->stage_d;
  MS_CUDA(cudaMemcpy(d, xas, size_t(n) * sizeof(double), cudaMemcpyHostToDevice));
  MS_CUDA(cudaMemcpy(d + n, xam, size_t(n) * sizeof(double), cudaMemcpyHostToDevice));
  if (aux) MS_CUDA(cudaMemcpy(d + 2 * n, aux, size_t(n) * sizeof(double), cudaMemcpyHostToDevice));
  MS_CUDA(with_ft(c, [&](auto tag) {
      using FT = typename decltype(tag)::type;
      return ms::launch_set_state<FT>(c->specs_d, c->tile_spec_d, c->n_tiles, d, d + n,
                                        aux ? d + 2 * n : nullptr, (FT*)c->xas_d,
                                        (FT*)c->xam_d, c->aux_d, c->stream);
    }));
  MS_CUDA(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->stream));
  MS_CUDA(ms::launch_fill_f32(c->tile_tsat_d, c->n_tiles, INFINITY, c->stream));
  MS_CUDA(cudaStreamSynchronize(c->stream));
  c->step_n = c->n_base = 0;
  c->t_base = 0.0;
  c->T_last = nullptr;
  return MS_OK;
}

int ms_fill_state(ms_ctx* c, double xas, double xam) {
  if (!c) return fail(MS_ERR_INVALID_ARG, "NULL context");
  if (!(std::isfinite(xas) && std::isfinite(xam) && xas >= 0 && xam >= 0 && xas + xam <= 0.9 + 1e-6))
    return fail(MS_ERR_INVALID_ARG, "need X_as, X_am >= 0 and X_as + X_am <= 0.9");
  MS_CUDA(with_ft(c, [&](auto tag) {
      using FT = typename decltype(tag)::type;
      return ms::launch_set_state<FT>(c->specs_d, c->tile_spec_d, c->n_tiles, nullptr, nullptr,
                                        nullptr, (FT*)c->xas_d, (FT*)c->xam_d, c->aux_d,
                                        c->stream, xas, xam);
    }));
  MS_CUDA(ms::launch_fill_f32(c->tile_tsat_d, c->n_tiles, INFINITY, c->stream));
  c->st.launches += 2;
  c->step_n = c->n_base = 0;
  c->t_base = 0.0;
  c->T_last = nullptr;
  return MS_OK;
}

int ms_reset_stats(ms_ctx* c) {
  if (!c) return fail(MS_ERR_INVALID_ARG, "NULL context");
  MS_CUDA(cudaStreamSynchronize(c->stream));
  MS_CUDA(cudaMemset(c->work_d, 0, sizeof(ms::WorkCounters)));
  if (c->hyb_d) MS_CUDA(cudaMemset(c->hyb_d, 0, sizeof(ms::HybridCounters)));
  MS_CUDA(cudaMemset(c->ops_d, 0, sizeof(ms::OpCounters)));
  const int32_t err = c->st.device_error;
  c->st = ms_stats_t{};
  c->st.device_error = err;
  c->kev_used = 0;
  c->timed = false;
  return MS_OK;
}

int ms_step(ms_ctx* c, const float* T_prev, const float* T_new, double dt, int32_t flags) {
  if (!c || !T_prev || !T_new) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  if (!(std::isfinite(dt) && dt > 0)) return fail(MS_ERR_INVALID_ARG, "dt must be > 0");
  if (c->specs_h.size() != 1) return fail(MS_ERR_STATE, "ms_step needs a single-specimen context");
  const int64_t n = c->n_points;
  const float *t0 = T_prev, *t1 = T_new;
  if (!(flags & MS_PTR_DEVICE)) {
    if (!c->Tstage_d) MS_CUDA(cudaMalloc(&c->Tstage_d, size_t(n) * 2 * sizeof(float)));
    MS_CUDA(cudaMemcpyAsync(c->Tstage_d, T_prev, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    MS_CUDA(cudaMemcpyAsync(c->Tstage_d + n, T_new, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    t0 = c->Tstage_d;
    t1 = c->Tstage_d + n;
  }
  set_dt(c, dt);
  MS_CUDA(cudaEventRecord(c->ev0, c->stream));
  int rc = with_ft(c, [&](auto tag) { return step_impl<typename decltype(tag)::at, typename decltype(tag)::type>(c, t0, t1); });
  if (rc != MS_OK) return rc;
  MS_CUDA(cudaEventRecord(c->ev1, c->stream));
  c->timed = true;
  c->T_last = t1;
  c->step_n += 1;
  c->st.steps += 1;
  c->st.point_updates += n;
  return MS_OK;
}

int ms_run_track(ms_ctx* c, const ms_heat_source* src, int64_t n_steps, double dt) {
  if (!c || !src) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  if (!(std::isfinite(dt) && dt > 0)) return fail(MS_ERR_INVALID_ARG, "dt must be > 0");
  if (n_steps < 0) return fail(MS_ERR_INVALID_ARG, "n_steps must be >= 0");
  if (!c->has_grid) return fail(MS_ERR_STATE, "ms_set_points must come first");
  int rc;
  if ((rc = set_sources(c, src)) != MS_OK) return rc;
  set_dt(c, dt);
  c->T_last = nullptr;
  if ((c->prm.flags & MS_FLAG_GRAPH) && n_steps > 0) return run_track_graph(c, n_steps);
  MS_CUDA(cudaEventRecord(c->ev0, c->stream));
  rc = with_ft(c, [&](auto tag) { return run_track_impl<typename decltype(tag)::at, typename decltype(tag)::type>(c, n_steps); });
  if (rc != MS_OK) return rc;
  MS_CUDA(cudaEventRecord(c->ev1, c->stream));
  c->timed = true;
  return MS_OK;
}

// The four fractions of every point in natural order into the device staging
// buffer (X_as, X_am, then X_beta, X_liq if with_beta), on the context stream.
int stage_fractions(ms_ctx* c, bool with_beta) {
  const int64_t n = c->n_points;
  double* d = c->stage_d;
  int rc;
  if (with_beta) {
    const float* T = nullptr;
    if (c->T_last) {
      T = c->T_last;
    } else if (c->has_grid && c->src_valid) {
      if ((rc = ensure_table(c, 1)) != MS_OK) return rc;
      if ((rc = launch_table(c, c->step_n, 1)) != MS_OK) return rc;
    } else {
      return fail(MS_ERR_STATE, "no temperature known for X_beta / X_liq yet");
    }
    MS_CUDA(with_ft(c, [&](auto tag) {
        using FT = typename decltype(tag)::type;
        using AT = typename decltype(tag)::at;
        return ms::launch_fractions<AT, FT>(
            consts<AT>(c), c->specs_d, c->tile_spec_d, c->n_tiles, (const FT*)c->xas_d,
            (const FT*)c->xam_d, T, static_cast<const ms::SrcLevelT<AT>*>(c->levels_d),
            static_cast<const ms::SrcEntryT<AT>*>(c->entries_d), c->slots, d + 2 * n, d + 3 * n,
            nullptr, c->stream);
      }));
  }
  MS_CUDA(with_ft(c, [&](auto tag) {
      using FT = typename decltype(tag)::type;
      return ms::launch_get_state<FT>(c->specs_d, c->tile_spec_d, c->n_tiles,
                                        (const FT*)c->xas_d, (const FT*)c->xam_d, c->aux_d,
                                        d, d + n, nullptr, c->stream);
    }));
  return MS_OK;
}

int ms_get_fractions(ms_ctx* c, double* xas, double* xam, double* xbeta, double* xliq) {
  if (!c) return fail(MS_ERR_INVALID_ARG, "NULL context");
  const int64_t n = c->n_points;
  double* d = c->stage_d;
  int rc;
  if ((rc = stage_fractions(c, xbeta || xliq)) != MS_OK) return rc;
  const size_t nb = size_t(n) * sizeof(double);
  if (xas) MS_CUDA(cudaMemcpyAsync(xas, d, nb, cudaMemcpyDeviceToHost, c->stream));
  if (xam) MS_CUDA(cudaMemcpyAsync(xam, d + n, nb, cudaMemcpyDeviceToHost, c->stream));
  if (xbeta) MS_CUDA(cudaMemcpyAsync(xbeta, d + 2 * n, nb, cudaMemcpyDeviceToHost, c->stream));
  if (xliq) MS_CUDA(cudaMemcpyAsync(xliq, d + 3 * n, nb, cudaMemcpyDeviceToHost, c->stream));
  return check_device_error(c);
}

int ms_get_aux(ms_ctx* c, double* aux) {
  if (!c || !aux) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  double* d = c->stage_d;
  MS_CUDA(with_ft(c, [&](auto tag) {
      using FT = typename decltype(tag)::type;
      return ms::launch_get_state<FT>(c->specs_d, c->tile_spec_d, c->n_tiles,
                                        (const FT*)c->xas_d, (const FT*)c->xam_d, c->aux_d,
                                        nullptr, nullptr, d, c->stream);
    }));
  MS_CUDA(cudaMemcpyAsync(aux, d, size_t(c->n_points) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check_device_error(c);
}

int ms_get_temperature(ms_ctx* c, double* T) {
  if (!c || !T) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  const int64_t n = c->n_points;
  double* d = c->stage_d;
  int rc;
  const float* Tin = nullptr;
  if (c->T_last) {
    Tin = c->T_last;
  } else if (c->has_grid && c->src_valid) {
    if ((rc = ensure_table(c, 1)) != MS_OK) return rc;
    if ((rc = launch_table(c, c->step_n, 1)) != MS_OK) return rc;
  } else {
    return fail(MS_ERR_STATE, "no temperature known yet");
  }
  MS_CUDA(with_ft(c, [&](auto tag) {
    using AT = typename decltype(tag)::at;
    using FT = typename decltype(tag)::type;
    return ms::launch_fractions<AT, FT>(
        consts<AT>(c), c->specs_d, c->tile_spec_d, c->n_tiles, (const FT*)c->xas_d,
        (const FT*)c->xam_d, Tin, static_cast<const ms::SrcLevelT<AT>*>(c->levels_d),
        static_cast<const ms::SrcEntryT<AT>*>(c->entries_d), c->slots, nullptr, nullptr, d,
        c->stream);
  }));
  MS_CUDA(cudaMemcpyAsync(T, d, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check_device_error(c);
}

int ms_get_state(ms_ctx* c, void* blob, size_t* bytes) {
  if (!c || !bytes) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  const size_t np = size_t(c->n_tiles) * TILE;
  const size_t need = sizeof(BlobHeader) + np * (2 * c->fbytes + sizeof(float));
  if (!blob) {
    *bytes = need;
    return MS_OK;
  }
  if (*bytes < need) return fail(MS_ERR_INVALID_ARG, "blob needs %zu bytes", need);
  BlobHeader h{kBlobMagic, c->n_points, int64_t(np), c->prm.precision, 0, c->step_n, c->n_base,
               c->t_base, c->dt};
  char* p = static_cast<char*>(blob);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  MS_CUDA(cudaMemcpyAsync(p, c->xas_d, np * c->fbytes, cudaMemcpyDeviceToHost, c->stream));
  p += np * c->fbytes;
  MS_CUDA(cudaMemcpyAsync(p, c->xam_d, np * c->fbytes, cudaMemcpyDeviceToHost, c->stream));
  p += np * c->fbytes;
  MS_CUDA(cudaMemcpyAsync(p, c->aux_d, np * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  *bytes = need;
  return check_device_error(c);
}

int ms_set_state_blob(ms_ctx* c, const void* blob, size_t bytes) {
  if (!c || !blob) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  const size_t np = size_t(c->n_tiles) * TILE;
  const size_t need = sizeof(BlobHeader) + np * (2 * c->fbytes + sizeof(float));
  BlobHeader h;
  if (bytes < sizeof(h)) return fail(MS_ERR_INVALID_ARG, "blob too small");
  std::memcpy(&h, blob, sizeof(h));
  if (h.magic != kBlobMagic || h.n_points != c->n_points || h.n_pad != int64_t(np) ||
      h.precision != c->prm.precision || bytes != need)
    return fail(MS_ERR_INVALID_ARG, "checkpoint does not match this context");
  MS_CUDA(cudaStreamSynchronize(c->stream));
  const char* p = static_cast<const char*>(blob) + sizeof(h);
  MS_CUDA(cudaMemcpy(c->xas_d, p, np * c->fbytes, cudaMemcpyHostToDevice));
  p += np * c->fbytes;
  MS_CUDA(cudaMemcpy(c->xam_d, p, np * c->fbytes, cudaMemcpyHostToDevice));
  p += np * c->fbytes;
  MS_CUDA(cudaMemcpy(c->aux_d, p, np * sizeof(float), cudaMemcpyHostToDevice));
  MS_CUDA(ms::launch_fill_f32(c->tile_tsat_d, c->n_tiles, INFINITY, c->stream));
  MS_CUDA(cudaStreamSynchronize(c->stream));
  c->step_n = h.step_n;
  c->n_base = h.n_base;
  c->t_base = h.t_base;
  c->dt = h.dt;
  c->T_last = nullptr;
  return MS_OK;
}

int ms_verify(ms_ctx* c, ms_ctx* ref, const int64_t* idx, int64_t n, double* out) {
  if (!c || !ref || !out || n < 0) return fail(MS_ERR_INVALID_ARG, "bad argument");
  if (n > ref->n_points || (!idx && n > c->n_points))
    return fail(MS_ERR_INVALID_ARG, "n exceeds the points of a context");
  if (c->device != ref->device) return fail(MS_ERR_INVALID_ARG, "contexts on different devices");
  for (int64_t i = 0; idx && i < n; ++i)
    if (idx[i] < 0 || idx[i] >= c->n_points) return fail(MS_ERR_INVALID_ARG, "idx[%lld] out of range", (long long)i);
  int rc;
  if ((rc = stage_fractions(ref, true)) != MS_OK) return rc;
  MS_CUDA(cudaStreamSynchronize(ref->stream));
  if ((rc = stage_fractions(c, true)) != MS_OK) return rc;
  int64_t* idx_d = nullptr;
  double* out_d = nullptr;
  cudaError_t e = cudaMalloc(&out_d, 3 * sizeof(double));
  if (e == cudaSuccess && idx && n > 0) e = cudaMalloc(&idx_d, size_t(n) * sizeof(int64_t));
  if (e == cudaSuccess && idx_d)
    e = cudaMemcpyAsync(idx_d, idx, size_t(n) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = ms::launch_verify(c->stage_d, c->n_points, ref->stage_d, ref->n_points, n, idx_d, out_d,
                          c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, out_d, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(idx_d);
  cudaFree(out_d);
  if (e != cudaSuccess) return fail(MS_ERR_CUDA, "%s", cudaGetErrorString(e));
  return check_device_error(c);
}

int ms_apply_correction(ms_ctx* c, const double* T, int32_t n_T, double* x_as, double* x_am,
                        int64_t n) {
  if (!c || !T || !x_as || !x_am || n < 0 || n_T < 1) return fail(MS_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return MS_OK;
  double* d = nullptr;
  MS_CUDA(cudaMalloc(&d, size_t(n) * (2 + size_t(n_T)) * sizeof(double)));
  const size_t b = size_t(n) * sizeof(double);
  double* dT = d + 2 * n;
  cudaError_t e = cudaMemcpyAsync(dT, T, b * size_t(n_T), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, x_as, b, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + n, x_am, b, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = ms::launch_correct(c->mcd, n, n_T, dT, d, d + n, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x_as, d, b, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x_am, d + n, b, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (e != cudaSuccess) return fail(MS_ERR_CUDA, "%s", cudaGetErrorString(e));
  return MS_OK;
}

int ms_set_surrogate(ms_ctx* c, const ms_surrogate* s, double judge_frac) {
  if (!c) return fail(MS_ERR_INVALID_ARG, "NULL context");
  if (!(judge_frac >= 0.0 && judge_frac <= 1.0))
    return fail(MS_ERR_INVALID_ARG, "judge_frac must be in [0, 1]");
  if (s && c->prm.precision != MS_F32 && c->prm.precision != MS_KAHAN)
    return fail(MS_ERR_UNSUPPORTED, "the hybrid path needs precision MS_F32 or MS_KAHAN");
  if (s && c->prm.integrator != MS_EXPLICIT)
    return fail(MS_ERR_UNSUPPORTED, "the hybrid path uses the explicit scheme");
  MS_CUDA(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  if (!s) {
    c->mlp = nullptr;
    return MS_OK;
  }
  if (!c->hyb_d) {
    MS_CUDA(cudaMalloc(&c->hyb_d, sizeof(ms::HybridCounters)));
    MS_CUDA(cudaMemset(c->hyb_d, 0, sizeof(ms::HybridCounters)));
  }
  const int act = ms::surrogate_activation(s);
  const int per_sm = c->prm.precision == MS_KAHAN ? ms::hybrid_blocks_per_sm<ms::KF>(act)
                                                  : ms::hybrid_blocks_per_sm<float>(act);
  if (per_sm <= 0) return fail(MS_ERR_CUDA, "hybrid kernel cannot be made resident");
  c->hybrid_per_sm = per_sm;
  c->mlp = ms::surrogate_weights(s);
  c->mlp_act = act;
  c->mlp_stride = ms::surrogate_stride(s);
  c->judge_thresh = uint64_t(std::llround(judge_frac * 4294967296.0));
  return MS_OK;
}

int ms_set_judge_tol(ms_ctx* c, double tol) {
  if (!c) return fail(MS_ERR_INVALID_ARG, "NULL context");
  if (!(tol >= 0.0)) return fail(MS_ERR_INVALID_ARG, "judge tolerance must be >= 0");
  if (tol != c->judge_tol) {
    MS_CUDA(cudaStreamSynchronize(c->stream));
    drop_graphs(c);  // captured launches hold the old value
    c->judge_tol = tol;
  }
  return MS_OK;
}

int ms_coarsen_ctx(ms_ctx* c, double tol, int32_t n_levels, uint8_t* mask, int64_t* n_coarse) {
  if (!c || !mask) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  if (n_levels < 1 || n_levels > MS_COARSEN_MAX_LEVELS)
    return fail(MS_ERR_INVALID_ARG, "n_levels must be in [1, MS_COARSEN_MAX_LEVELS]");
  if (!(tol >= 0.0 && tol <= 1e300)) return fail(MS_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (!c->has_grid || c->specs_h.size() != 1 || c->specs_h[0].idx)
    return fail(MS_ERR_STATE, "the coarsening criterion needs one full grid (ms_set_points)");
  const SpecDev& sp = c->specs_h[0];
  const int32_t dims[3] = {sp.nx, sp.ny, sp.nz};
  int rc;
  if ((rc = stage_fractions(c, true)) != MS_OK) return rc;
  const int64_t n = c->n_points;
  const int64_t total = ms::coarsen_counts(dims, n_levels, nullptr);
  const size_t sb = ms::coarsen_scratch_bytes(dims);   // ranges, then the counters
  char* buf = nullptr;
  MS_CUDA(cudaMalloc(&buf, sb + size_t(total) + 64 * sizeof(unsigned long long)));
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(buf + sb);
  uint8_t* dmask = reinterpret_cast<uint8_t*>(buf + sb + 64 * sizeof(unsigned long long));
  const double* d = c->stage_d;
  unsigned long long hc[64] = {};
  cudaError_t e = ms::launch_coarsen(d, d + n, d + 2 * n, dims, tol, n_levels, dmask, buf, cnt,
                                     c->stream);
  if (e == cudaSuccess && total > 0)
    e = cudaMemcpyAsync(mask, dmask, size_t(total), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hc, cnt, sizeof(unsigned long long) * size_t(n_levels),
                        cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(MS_ERR_CUDA, "%s", cudaGetErrorString(e));
  if (n_coarse)
    for (int l = 0; l < n_levels; ++l) n_coarse[l] = int64_t(hc[l]);
  return check_device_error(c);
}

int ms_stats(ms_ctx* c, ms_stats_t* out) {
  if (!c || !out) return fail(MS_ERR_INVALID_ARG, "NULL argument");
  int rc = check_device_error(c);
  *out = c->st;
  return rc == MS_ERR_CUDA ? rc : MS_OK;
}

int ms_synchronize(ms_ctx* c) {
  if (!c) return fail(MS_ERR_INVALID_ARG, "NULL context");
  return check_device_error(c);
}

}  // extern "C"
