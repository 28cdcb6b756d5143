// ms_run_track_noalloc: the ms_run_track hot path for callers that cannot
// allocate device memory.
//
// Its scratch (the per-launch source table, the work counters of the
// persistent kernel, the specimen / track / layer tables and the
// tile -> specimen map) lives in one file-scope static device array of a fixed
// size instead of context-owned cudaMalloc'd buffers.  The caller passes the
// state arrays (inputs and outputs) and the source; nothing is allocated, on
// the device or on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "ms_internal.h"

namespace {

constexpr int kMaxTracks = 128;                 // tracks of the specimen
constexpr int kMaxLayers = 8;                   // layers of the specimen
constexpr int kMaxSteps = 64;                   // steps per launch
constexpr int kMaxLevels = kMaxSteps + 1;
constexpr int64_t kMaxTiles = int64_t(1) << 17; // 2^24 points
constexpr int kMaxDevices = 64;

struct Scratch {
  ms::WorkCounters work;
  int32_t err;
  int32_t pad0;
  ms::SpecDev spec;
  ms::TrackDev tracks[kMaxTracks];
  ms::LayerDev layers[kMaxLayers];
  ms::SrcLevelT<float> levels[kMaxLevels];
  ms::SrcEntryT<float> entries[kMaxLevels * kMaxTracks];
  float ff[ms::FF_FLOATS];                      // far-field weights and nodes (set-up)
  int32_t tile_spec[kMaxTiles];                 // all zero: one specimen
};

// The shared scratch: 0.77 MiB on every device that loads the library, held
// until the process exits.  Calls whose work overlaps on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(Scratch)];

// Host-side copy of the small tables, uploaded in one copy per call.
struct Upload {
  ms::SpecDev spec;
  ms::TrackDev tracks[kMaxTracks];
  ms::LayerDev layers[kMaxLayers];
};
static_assert(offsetof(Scratch, tracks) - offsetof(Scratch, spec) == offsetof(Upload, tracks),
              "Upload must mirror the spec / tracks / layers part of Scratch");
static_assert(offsetof(Scratch, layers) - offsetof(Scratch, spec) == offsetof(Upload, layers),
              "Upload must mirror the spec / tracks / layers part of Scratch");
static_assert(offsetof(Scratch, spec) % 8 == 0, "spec must be 8-byte aligned");
static_assert(offsetof(Scratch, levels) % 16 == 0 && offsetof(Scratch, entries) % 16 == 0,
              "the source table is read with 16-byte vector loads");
static_assert(offsetof(Scratch, ff) % 16 == 0, "far-field table alignment");
static_assert(sizeof(Scratch) < (1u << 20), "the no-alloc scratch stays below 1 MiB");

std::mutex g_setup_mu;
Scratch* g_scratch_ptr[kMaxDevices] = {};
int g_track_grid[kMaxDevices] = {};

// Once per device, with that device current: the device address of the static
// array (its name in host code is only a host-side stand-in), a cleared tile
// map and the far-field interpolation table.  Not allocation: the array is
// part of the loaded module.  The clear and the table copy go to the legacy
// default stream, which does not order against streams created non-blocking
// (torch's side streams, for one), so the set-up waits for them before any
// work of the caller's stream can touch the array.
int setup_device(int dev, Scratch** out, int* grid_per_device) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return ms::record_error(MS_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
    static float table[ms::FF_FLOATS];
    if (ms_farfield_table(table, ms::FF_FLOATS) != MS_OK) return MS_ERR_INVALID_ARG;
    Scratch* sp = static_cast<Scratch*>(p);
    if (cudaMemset(p, 0, sizeof(Scratch)) != cudaSuccess ||
        cudaMemcpy(sp->ff, table, sizeof(table), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
      return ms::record_error(MS_ERR_CUDA, "clearing the no-alloc scratch failed");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return ms::record_error(MS_ERR_CUDA, "cannot query the SM count");
    g_track_grid[dev] = ms::track_blocks_per_sm<float, float>(128) * sms;
    g_scratch_ptr[dev] = static_cast<Scratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  *grid_per_device = g_track_grid[dev];
  return MS_OK;
}

}  // namespace

extern "C" int ms_run_track_noalloc(const ms_params* p, const ms_grid* grid,
                                    const ms_heat_source* src, float* x_as, float* x_am,
                                    float* aux, int64_t n_points, int64_t step0, int64_t n_steps,
                                    double dt, void* stream) {
  if (!p || !grid || !src || !x_as || !x_am || !aux)
    return ms::record_error(MS_ERR_INVALID_ARG, "NULL argument");
  int rc = ms::validate_params(*p);
  if (rc != MS_OK) return rc;
  if (p->precision != MS_F32)
    return ms::record_error(MS_ERR_UNSUPPORTED, "ms_run_track_noalloc computes in MS_F32 only");
  if (p->integrator != MS_EXPLICIT)
    return ms::record_error(MS_ERR_UNSUPPORTED, "ms_run_track_noalloc takes explicit steps only");
  if (p->steps_per_launch > kMaxSteps)
    return ms::record_error(MS_ERR_INVALID_ARG, "steps_per_launch above 64 (no-alloc limit)");
  if (p->block_threads != 0 && p->block_threads != 128)
    return ms::record_error(MS_ERR_INVALID_ARG, "the no-alloc path runs 128-thread blocks");
  if (!(std::isfinite(dt) && dt > 0) || n_steps < 0 || step0 < 0)
    return ms::record_error(MS_ERR_INVALID_ARG, "need dt > 0, n_steps >= 0, step0 >= 0");
  if (((reinterpret_cast<uintptr_t>(x_as) | reinterpret_cast<uintptr_t>(x_am) |
        reinterpret_cast<uintptr_t>(aux)) & 15) != 0)
    return ms::record_error(MS_ERR_INVALID_ARG, "state arrays must be 16-byte aligned");
  if (grid->dims[0] < 1 || grid->dims[1] < 1 || grid->dims[2] < 1 || grid->k_offset < 0 ||
      int64_t(grid->dims[0]) * grid->dims[1] * grid->dims[2] != n_points)
    return ms::record_error(MS_ERR_INVALID_ARG, "grid dims do not give n_points");
  const int64_t n_tiles = (n_points + ms::TILE - 1) / ms::TILE;
  if (n_tiles > kMaxTiles)
    return ms::record_error(MS_ERR_INVALID_ARG, "more than 2^24 points (no-alloc limit)");
  if (src->n_tracks < 0 || src->n_tracks > kMaxTracks || src->n_layers < 1 ||
      src->n_layers > kMaxLayers || !src->layers || (src->n_tracks > 0 && !src->tracks))
    return ms::record_error(MS_ERR_INVALID_ARG, "more than 128 tracks or 8 layers (no-alloc limit)");
  if (!(std::isfinite(src->A) && src->A >= 0 && src->k > 0 && src->alpha > 0 && src->T0 > 0 &&
        src->T_max > src->T0 && std::isfinite(src->t_offset) && src->z_tol >= 0))
    return ms::record_error(MS_ERR_INVALID_ARG, "invalid heat source");

  Upload up;
  std::memset(&up, 0, sizeof(up));
  int per_layer[kMaxLayers] = {};
  int slots = 1;
  for (int j = 0; j < src->n_tracks; ++j) {
    const ms_track& t = src->tracks[j];
    const double un = std::sqrt(t.ux * t.ux + t.uy * t.uy);
    if (!(t.layer >= 0 && t.layer < src->n_layers && std::fabs(un - 1.0) < 1e-6 && t.v > 0 &&
          std::isfinite(t.v) && t.P >= 0 && std::isfinite(t.P) && std::isfinite(t.x0) &&
          std::isfinite(t.y0) && std::isfinite(t.t_start)))
      return ms::record_error(MS_ERR_INVALID_ARG, "invalid track");
    up.tracks[j] = ms::TrackDev{t.x0, t.y0, t.ux, t.uy, t.v, t.P, t.t_start, t.layer, 0};  // one specimen
    if (++per_layer[t.layer] > slots) slots = per_layer[t.layer];
  }
  for (int j = 0; j < src->n_layers; ++j) {
    const ms_layer& L = src->layers[j];
    if (!(std::isfinite(L.z_surface) && L.t_scan_end >= L.t_begin && L.t_end >= L.t_scan_end))
      return ms::record_error(MS_ERR_INVALID_ARG, "invalid layer");
    up.layers[j] = ms::LayerDev{L.z_surface, L.t_begin, L.t_scan_end, L.t_end};
  }
  ms::SpecDev& s = up.spec;
  s.ox = double(float(grid->origin[0])); s.oy = double(float(grid->origin[1]));
  s.oz = double(float(grid->origin[2]));
  s.dx = double(float(grid->spacing[0])); s.dy = double(float(grid->spacing[1]));
  s.dz = double(float(grid->spacing[2]));
  s.nx = grid->dims[0]; s.ny = grid->dims[1]; s.nz = grid->dims[2];
  s.k_off = grid->k_offset;
  s.n = n_points;
  s.n_tiles = int32_t(n_tiles);
  s.n_tracks = src->n_tracks;
  s.n_layers = src->n_layers;
  s.z_tol = float(src->z_tol);
  s.T0 = float(src->T0);
  s.T_max = float(src->T_max);
  s.A = src->A; s.k = src->k; s.alpha = src->alpha; s.t_offset = src->t_offset;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return ms::record_error(MS_ERR_CUDA, "no usable CUDA device");
  Scratch* sc = nullptr;
  int grid_cap = 0;
  if ((rc = setup_device(dev, &sc, &grid_cap)) != MS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The tables are copied from this call's stack frame: a captured copy would
  // read that frame again on every replay, long after the call returned.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess)
    return ms::record_error(MS_ERR_CUDA, "cannot query the stream's capture status");
  if (cap != cudaStreamCaptureStatusNone)
    return ms::record_error(MS_ERR_UNSUPPORTED,
                            "ms_run_track_noalloc uploads its tables from host memory of the "
                            "call and refuses a capturing stream");
  if (cudaMemsetAsync(&sc->err, 0, sizeof(int32_t), st) != cudaSuccess ||
      cudaMemcpyAsync(&sc->spec, &up, sizeof(Upload), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return ms::record_error(MS_ERR_CUDA, "uploading the source tables failed");

  const ms::ModelConstT<float> mc = ms::model_const<float>(*p);
  const int S = p->steps_per_launch;
  const int grid_blocks = int(std::min<int64_t>(grid_cap, (n_tiles + 3) / 4));
  int64_t done = 0;
  while (done < n_steps) {
    const int steps = int(std::min<int64_t>(S, n_steps - done));
    ms::TableArgs ta{};
    ta.specs = &sc->spec;
    ta.tracks = sc->tracks;
    ta.layers = sc->layers;
    ta.n_specs = 1;
    ta.n_levels = steps + 1;
    ta.slots = slots;
    ta.n0 = step0 + done;
    ta.t_base = 0.0;
    ta.dt = dt;
    ta.levels = sc->levels;
    ta.entries = sc->entries;
    ta.ff_dist = p->farfield_dist > 0.0 ? p->farfield_dist : 0.0;
    if (ms::launch_src_table<float>(ta, &sc->work, st) != cudaSuccess)
      return ms::record_error(MS_ERR_CUDA, "source-table launch failed");
    ms::TrackArgs<float, float> a{};
    a.m = mc;
    a.specs = &sc->spec;
    a.tile_spec = sc->tile_spec;
    a.tile_list = nullptr;
    a.work = &sc->work;
    a.n_tiles = int32_t(n_tiles);
    a.n_levels = steps + 1;
    a.slots = slots;
    a.dt = float(dt);
    a.levels = sc->levels;
    a.entries = sc->entries;
    a.xas = x_as;
    a.xam = x_am;
    a.aux = aux;
    a.tile_tsat = nullptr;
    a.err = &sc->err;
    if (p->farfield_dist > 0.0) {
      a.ff = sc->ff;
      a.ff_dist = float(p->farfield_dist);
      // tiles across two grid rows: the instantiation ms_run_track takes
      a.two_rows = grid->dims[0] % ms::TILE != 0 && int64_t(grid->dims[1]) * grid->dims[2] > 1;
    }
    if (ms::launch_track<float, float>(a, 128, grid_blocks, st) != cudaSuccess)
      return ms::record_error(MS_ERR_CUDA, "hot-kernel launch failed");
    done += steps;
  }
  // The device error word of this call's launches: wait for them and report a
  // non-finite fraction as ms_run_track's contexts do at their sync points.
  int32_t err = 0;
  if (cudaMemcpyAsync(&err, &sc->err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ms::record_error(MS_ERR_CUDA, "reading the device error word failed");
  if (err & ms::DEVERR_NONFINITE)
    return ms::record_error(MS_ERR_NONFINITE, "a fraction became non-finite");
  return MS_OK;
}
