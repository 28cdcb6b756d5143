// Grid thermal solver feeding the phase model (one-way coupling of Sec. 3:
// the temperature field comes from a thermal model, the phase model takes
// T^n and T^{n+1} of every point).
//
// The heat equation of Sec. 2.1, rho c dT/dt = div(k grad T) + q_vol, on the
// points' own regular grid: one finite volume per node, conductance
// k_f A / d between neighbours with the harmonic mean k_f of the two nodes'
// conductivities k = (1 - r_c) k_p + r_c k_ms (eq:material_parameter_interp
// with k_m = k_s), the cylindrical laser source eq:heat_soruce_cylindrical
// in the powder layer below the top surface, radiation eps sigma (T^4 -
// T_inf^4) from the top layer, T0 held on the bottom layer, adiabatic sides,
// explicit Euler substeps within the stability limit, T capped at T_max and
// r_c <- max(r_c, g(T)) (eq:consolidated_fraction) after each substep.
//
// k_heat: one thread per node, FP32, neighbours read through the caches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ms_internal.h"

namespace {

constexpr double kPiD = 3.14159265358979323846;
constexpr double kSigmaSB = 5.670374419e-8;
constexpr float kLog2eF = 1.4426950408889634f;

struct HeatArgs {
  int nx, ny, nz, top, bottom;
  float gx, gy, gz;          // face area / node distance per direction [m]
  float inv_cap;             // h / (rho c V) [K / J]
  float V, area_top;         // node volume, top face area
  float k_ms, k_p;
  float T0, T_inf4, eps_sigma, T_max, T_s, inv_mushy;
  int radiation, dirichlet, cap, laser_on;
  float sx, sy;              // laser centre relative to the grid origin [m]
  float q_peak;              // 2 W / (pi R^2 h_p) [W/m^3]
  float neg2_over_R2_l2;     // -2 / R^2 * log2(e)
  float ox_rel_dx, oy_rel_dy;  // unused padding
  float dx, dy;
  const float* z_depth;      // per layer: depth below the top surface [m]
  float h_powder;
  const float* T;
  const float* rc;
  float* Tn;
  float* rcn;
};

__device__ __forceinline__ float cond(const HeatArgs& a, float rc) {
  return (1.0f - rc) * a.k_p + rc * a.k_ms;
}

__device__ __forceinline__ float harm(float ka, float kb) {
  const float s = ka + kb;
  return s > 0.0f ? 2.0f * ka * kb / s : 0.0f;
}

__global__ void __launch_bounds__(128) k_heat(const HeatArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= a.nx) return;
  const int64_t nxy = int64_t(a.nx) * a.ny;
  const int64_t id = i + int64_t(a.nx) * j + nxy * k;
  const float Tc = a.T[id];
  const float rcc = a.rc[id];
  const float kc = cond(a, rcc);
  float flux = 0.0f;
  if (i > 0) flux += harm(kc, cond(a, a.rc[id - 1])) * a.gx * (a.T[id - 1] - Tc);
  if (i + 1 < a.nx) flux += harm(kc, cond(a, a.rc[id + 1])) * a.gx * (a.T[id + 1] - Tc);
  if (j > 0) flux += harm(kc, cond(a, a.rc[id - a.nx])) * a.gy * (a.T[id - a.nx] - Tc);
  if (j + 1 < a.ny) flux += harm(kc, cond(a, a.rc[id + a.nx])) * a.gy * (a.T[id + a.nx] - Tc);
  if (k > 0) flux += harm(kc, cond(a, a.rc[id - nxy])) * a.gz * (a.T[id - nxy] - Tc);
  if (k + 1 < a.nz) flux += harm(kc, cond(a, a.rc[id + nxy])) * a.gz * (a.T[id + nxy] - Tc);
  if (a.laser_on) {
    const float depth = a.z_depth[k];
    if (depth >= 0.0f && depth < a.h_powder) {
      const float rx = float(i) * a.dx - a.sx, ry = float(j) * a.dy - a.sy;
      float e;
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(a.neg2_over_R2_l2 * (rx * rx + ry * ry)));
      flux += a.q_peak * e * a.V;
    }
  }
  if (a.radiation && k == a.top) {
    const float T2 = Tc * Tc;
    flux -= a.eps_sigma * (T2 * T2 - a.T_inf4) * a.area_top;
  }
  float Tn = fmaf(flux, a.inv_cap, Tc);
  if (a.dirichlet && k == a.bottom) Tn = a.T0;
  if (a.cap) Tn = fminf(Tn, a.T_max);
  const float g = fminf(fmaxf((Tn - a.T_s) * a.inv_mushy, 0.0f), 1.0f);
  a.Tn[id] = Tn;
  a.rcn[id] = fmaxf(rcc, g);
}

__global__ void k_thermal_init(float* T, float* rc, const float* z_depth, int64_t nxy, int nz,
                               float T0, float h_powder) {
  const int64_t id = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (id >= nxy * nz) return;
  const int k = int(id / nxy);
  const float d = z_depth[k];
  T[id] = T0;
  rc[id] = (d >= 0.0f && d < h_powder) ? 0.0f : 1.0f;
}

struct Track {
  double x0, y0, ux, uy, v, P, t_start, t_end;
};

}  // namespace

struct ms_thermal {
  ms_thermal_params p{};
  ms_grid grid{};
  int nx = 0, ny = 0, nz = 0, top = 0, bottom = 0;
  int64_t n = 0;
  float* T[3] = {nullptr, nullptr, nullptr};
  float* rc[2] = {nullptr, nullptr};
  float* z_depth = nullptr;
  int prev = 0, cur = 0, rcur = 0;
  double t = 0.0;
  std::vector<Track> tracks;
  cudaStream_t own = nullptr, stream = nullptr;
  int64_t substeps = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double kernel_ms = 0.0;
};

namespace {

#define TH_CUDA(...)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (__VA_ARGS__);                                                           \
    if (e_ != cudaSuccess)                                                                    \
      return ms::record_error(e_ == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA,     \
                              cudaGetErrorString(e_));                                        \
  } while (0)

int n_substeps(const ms_thermal* th, double dt) {
  const double dx = std::fabs(th->grid.spacing[0]), dy = std::fabs(th->grid.spacing[1]),
               dz = std::fabs(th->grid.spacing[2]);
  const double dt_stab =
      th->p.rho * th->p.c / (th->p.k_ms * (2.0 / (dx * dx) + 2.0 / (dy * dy) + 2.0 / (dz * dz)));
  const double r = std::ceil(dt / (0.9 * dt_stab) - 1e-9);
  return r < 1.0 ? 1 : int(std::min(r, 1e8));
}

// The laser at time t: on from a track's start to its end (the next track's
// start, or the layer's scan end for the last track of a layer).
bool laser_at(const ms_thermal* th, double t, double* x, double* y, double* W) {
  for (const Track& tr : th->tracks) {
    if (tr.t_start <= t && t < tr.t_end) {
      const double d = tr.v * (t - tr.t_start);
      *x = tr.x0 + tr.ux * d;
      *y = tr.y0 + tr.uy * d;
      *W = tr.P;
      return true;
    }
  }
  return false;
}

int step_on(ms_thermal* th, double dt, cudaStream_t st) {
  const int ns = n_substeps(th, dt);
  const double h = dt / ns;
  const double dx = std::fabs(th->grid.spacing[0]), dy = std::fabs(th->grid.spacing[1]),
               dz = std::fabs(th->grid.spacing[2]);
  const double V = dx * dy * dz;
  HeatArgs a{};
  a.nx = th->nx;
  a.ny = th->ny;
  a.nz = th->nz;
  a.top = th->top;
  a.bottom = th->bottom;
  a.gx = float(dy * dz / dx);
  a.gy = float(dx * dz / dy);
  a.gz = float(dx * dy / dz);
  a.inv_cap = float(h / (th->p.rho * th->p.c * V));
  a.V = float(V);
  a.area_top = float(dx * dy);
  a.k_ms = float(th->p.k_ms);
  a.k_p = float(th->p.k_p);
  a.T0 = float(th->p.T0);
  a.T_inf4 = float(std::pow(th->p.T_inf, 4.0));
  a.eps_sigma = float(th->p.emissivity * kSigmaSB);
  a.T_max = float(th->p.T_max);
  a.T_s = float(th->p.T_s);
  a.inv_mushy = float(1.0 / (th->p.T_l - th->p.T_s));
  a.radiation = th->p.radiation;
  a.dirichlet = th->p.dirichlet_bottom;
  a.cap = th->p.cap;
  a.q_peak = 0.0f;
  a.neg2_over_R2_l2 =
      float(-2.0 / (th->p.beam_radius * th->p.beam_radius)) * kLog2eF;
  a.dx = float(th->grid.spacing[0]);
  a.dy = float(th->grid.spacing[1]);
  a.z_depth = th->z_depth;
  a.h_powder = float(th->p.h_powder);
  const dim3 grid(unsigned((th->nx + 127) / 128), unsigned(th->ny), unsigned(th->nz));
  // substeps read T[prev] first, then ping-pong between the other two
  // buffers; the last one written becomes the new current field
  int src = th->prev;
  const int o1 = (th->prev + 1) % 3, o2 = (th->prev + 2) % 3;
  int dst = o1;
  for (int s = 0; s < ns; ++s) {
    double x = 0, y = 0, W = 0;
    a.laser_on = laser_at(th, th->t + s * h, &x, &y, &W) ? 1 : 0;
    a.sx = float(x - th->grid.origin[0]);
    a.sy = float(y - th->grid.origin[1]);
    a.q_peak = float(2.0 * W / (kPiD * th->p.beam_radius * th->p.beam_radius * th->p.h_powder));
    a.T = th->T[src];
    a.Tn = th->T[dst];
    a.rc = th->rc[th->rcur];
    a.rcn = th->rc[1 - th->rcur];
    k_heat<<<grid, 128, 0, st>>>(a);
    TH_CUDA(cudaGetLastError());
    th->rcur = 1 - th->rcur;
    src = dst;
    dst = (dst == o1) ? o2 : o1;
  }
  th->cur = src;
  th->t += dt;
  th->substeps += ns;
  return MS_OK;
}

}  // namespace

extern "C" {

int ms_thermal_params_default(ms_thermal_params* p) {
  if (!p) return ms::record_error(MS_ERR_INVALID_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->rho = 4090.0;       // Table 1
  p->c = 1130.0;
  p->k_ms = 28.6;
  p->k_p = 0.286;
  p->T_s = 1878.0;
  p->T_l = 1928.0;
  p->T0 = 353.0;
  p->T_inf = 293.0;
  p->emissivity = 0.7;
  p->T_max = 4130.0;     // T_v + 1000 K
  p->beam_radius = 0.06e-3;  // Table 5
  p->h_powder = 30e-6;
  p->radiation = 1;
  p->dirichlet_bottom = 1;
  p->cap = 1;
  return MS_OK;
}

int ms_thermal_create(const ms_thermal_params* p, const ms_grid* g, ms_thermal** out) {
  if (!p || !g || !out) return ms::record_error(MS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
  if (!(pos(p->rho) && pos(p->c) && pos(p->k_ms) && p->k_p >= 0 && std::isfinite(p->k_p) &&
        pos(p->T0) && pos(p->T_s) && p->T_l > p->T_s && pos(p->T_max) && p->emissivity >= 0 &&
        pos(p->beam_radius) && pos(p->h_powder) && std::isfinite(p->T_inf)))
    return ms::record_error(MS_ERR_INVALID_ARG, "invalid thermal parameters");
  for (int d = 0; d < 3; ++d)
    if (g->dims[d] < 1 || !(std::isfinite(g->spacing[d]) && g->spacing[d] != 0.0) ||
        !std::isfinite(g->origin[d]))
      return ms::record_error(MS_ERR_INVALID_ARG, "invalid grid");
  if (g->k_offset != 0)
    return ms::record_error(MS_ERR_INVALID_ARG, "the thermal solver takes k_offset = 0 only");
  ms_thermal* th = new (std::nothrow) ms_thermal();
  if (!th) return ms::record_error(MS_ERR_OOM, "host allocation failed");
  auto bail = [&](int rc) { ms_thermal_destroy(th); return rc; };
  th->p = *p;
  th->grid = *g;
  th->nx = g->dims[0];
  th->ny = g->dims[1];
  th->nz = g->dims[2];
  th->n = int64_t(th->nx) * th->ny * th->nz;
  // top = the layer with the largest z, bottom = the smallest
  th->top = g->spacing[2] < 0 ? 0 : th->nz - 1;
  th->bottom = g->spacing[2] < 0 ? th->nz - 1 : 0;
  std::vector<float> depth(size_t(th->nz));
  const double ztop = g->origin[2] + g->spacing[2] * th->top;
  for (int k = 0; k < th->nz; ++k) depth[size_t(k)] = float(ztop - (g->origin[2] + g->spacing[2] * k));
  if (cudaStreamCreateWithFlags(&th->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&th->ev0) != cudaSuccess || cudaEventCreate(&th->ev1) != cudaSuccess)
    return bail(ms::record_error(MS_ERR_CUDA, "stream or event creation failed"));
  th->stream = th->own;
  for (int b = 0; b < 3; ++b)
    if (cudaMalloc(&th->T[b], size_t(th->n) * sizeof(float)) != cudaSuccess)
      return bail(ms::record_error(MS_ERR_OOM, "device allocation failed"));
  for (int b = 0; b < 2; ++b)
    if (cudaMalloc(&th->rc[b], size_t(th->n) * sizeof(float)) != cudaSuccess)
      return bail(ms::record_error(MS_ERR_OOM, "device allocation failed"));
  if (cudaMalloc(&th->z_depth, size_t(th->nz) * sizeof(float)) != cudaSuccess ||
      cudaMemcpy(th->z_depth, depth.data(), depth.size() * sizeof(float), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return bail(ms::record_error(MS_ERR_OOM, "device allocation failed"));
  int rc = ms_thermal_reset(th);
  if (rc != MS_OK) return bail(rc);
  *out = th;
  return MS_OK;
}

void ms_thermal_destroy(ms_thermal* th) {
  if (!th) return;
  if (th->stream) cudaStreamSynchronize(th->stream);
  for (float* b : th->T) cudaFree(b);
  for (float* b : th->rc) cudaFree(b);
  cudaFree(th->z_depth);
  if (th->ev0) cudaEventDestroy(th->ev0);
  if (th->ev1) cudaEventDestroy(th->ev1);
  if (th->own) cudaStreamDestroy(th->own);
  delete th;
}

int ms_thermal_set_stream(ms_thermal* th, void* stream) {
  if (!th) return ms::record_error(MS_ERR_INVALID_ARG, "NULL thermal solver");
  TH_CUDA(cudaStreamSynchronize(th->stream));
  th->stream = stream ? static_cast<cudaStream_t>(stream) : th->own;
  return MS_OK;
}

int ms_thermal_reset(ms_thermal* th) {
  if (!th) return ms::record_error(MS_ERR_INVALID_ARG, "NULL thermal solver");
  const int64_t nxy = int64_t(th->nx) * th->ny;
  th->prev = th->cur = 0;
  th->rcur = 0;
  th->t = 0.0;
  k_thermal_init<<<unsigned((th->n + 255) / 256), 256, 0, th->stream>>>(
      th->T[0], th->rc[0], th->z_depth, nxy, th->nz, float(th->p.T0), float(th->p.h_powder));
  TH_CUDA(cudaGetLastError());
  TH_CUDA(cudaStreamSynchronize(th->stream));
  return MS_OK;
}

int ms_thermal_set_source(ms_thermal* th, const ms_heat_source* src) {
  if (!th || !src || (src->n_tracks > 0 && !src->tracks) || src->n_layers < 1 || !src->layers)
    return ms::record_error(MS_ERR_INVALID_ARG, "bad heat source");
  std::vector<Track> tr;
  for (int j = 0; j < src->n_tracks; ++j) {
    const ms_track& t = src->tracks[j];
    if (t.layer < 0 || t.layer >= src->n_layers || !(t.v > 0) || !(t.P >= 0) ||
        !std::isfinite(t.t_start))
      return ms::record_error(MS_ERR_INVALID_ARG, "invalid track");
    double t_end = src->layers[t.layer].t_scan_end;
    if (j + 1 < src->n_tracks && src->tracks[j + 1].layer == t.layer) {
      // the laser leaves a track when the next one of its layer starts
      if (src->tracks[j + 1].t_start < t.t_start)
        return ms::record_error(MS_ERR_INVALID_ARG, "tracks of a layer must be sorted by start time");
      t_end = src->tracks[j + 1].t_start;
    }
    tr.push_back(Track{t.x0, t.y0, t.ux, t.uy, t.v, t.P, t.t_start + src->t_offset,
                       t_end + src->t_offset});
  }
  th->tracks = tr;
  return MS_OK;
}

int ms_thermal_step(ms_thermal* th, double dt) {
  if (!th || !(std::isfinite(dt) && dt > 0)) return ms::record_error(MS_ERR_INVALID_ARG, "bad argument");
  TH_CUDA(cudaEventRecord(th->ev0, th->stream));
  th->prev = th->cur;
  int rc = step_on(th, dt, th->stream);
  if (rc != MS_OK) return rc;
  TH_CUDA(cudaEventRecord(th->ev1, th->stream));
  TH_CUDA(cudaEventSynchronize(th->ev1));
  float ms_ = 0.f;
  TH_CUDA(cudaEventElapsedTime(&ms_, th->ev0, th->ev1));
  th->kernel_ms += ms_;
  return MS_OK;
}

int ms_thermal_fields(ms_thermal* th, const float** T_prev, const float** T_cur, const float** rc) {
  if (!th) return ms::record_error(MS_ERR_INVALID_ARG, "NULL thermal solver");
  if (T_prev) *T_prev = th->T[th->prev];
  if (T_cur) *T_cur = th->T[th->cur];
  if (rc) *rc = th->rc[th->rcur];
  return MS_OK;
}

int ms_thermal_get(ms_thermal* th, double* T, double* rc_out) {
  if (!th) return ms::record_error(MS_ERR_INVALID_ARG, "NULL thermal solver");
  std::vector<float> buf(size_t(th->n));
  for (int w = 0; w < 2; ++w) {
    double* out = w == 0 ? T : rc_out;
    if (!out) continue;
    const float* src = w == 0 ? th->T[th->cur] : th->rc[th->rcur];
    TH_CUDA(cudaMemcpyAsync(buf.data(), src, size_t(th->n) * sizeof(float), cudaMemcpyDeviceToHost,
                            th->stream));
    TH_CUDA(cudaStreamSynchronize(th->stream));
    for (int64_t i = 0; i < th->n; ++i) out[i] = double(buf[size_t(i)]);
  }
  return MS_OK;
}

int ms_thermal_stats(ms_thermal* th, double* time_s, int64_t* substeps, double* kernel_ms) {
  if (!th) return ms::record_error(MS_ERR_INVALID_ARG, "NULL thermal solver");
  if (time_s) *time_s = th->t;
  if (substeps) *substeps = th->substeps;
  if (kernel_ms) *kernel_ms = th->kernel_ms;
  return MS_OK;
}

int ms_thermal_run_coupled(ms_thermal* th, ms_ctx* ctx, int64_t n_steps, double dt) {
  if (!th || !ctx || n_steps < 0 || !(std::isfinite(dt) && dt > 0))
    return ms::record_error(MS_ERR_INVALID_ARG, "bad argument");
  void* cs = ms::ctx_stream(ctx);
  if (ms::ctx_points(ctx) != th->n)
    return ms::record_error(MS_ERR_INVALID_ARG, "context and thermal grid differ in size");
  TH_CUDA(cudaStreamSynchronize(th->stream));
  cudaStream_t st = static_cast<cudaStream_t>(cs);
  for (int64_t s = 0; s < n_steps; ++s) {
    th->prev = th->cur;
    int rc = step_on(th, dt, st);
    if (rc != MS_OK) return rc;
    rc = ms_step(ctx, th->T[th->prev], th->T[th->cur], dt, MS_PTR_DEVICE);
    if (rc != MS_OK) return rc;
  }
  return ms_synchronize(ctx);
}

}  // extern "C"
