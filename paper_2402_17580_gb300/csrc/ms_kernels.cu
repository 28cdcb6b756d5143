// sm_103a kernels of the microstructure point solver.
//
//  k_src_table   per (specimen, time level): positions and constants of the
//                started moving sources (FP64 -> FP32), so the hot kernel
//                reads one 32-byte entry per source and level.
//  k_track       the hot path of ms_run_track: one warp per 128-point tile,
//                4 points per thread (128-bit SoA loads), S steps per state
//                load; the temperature of every point and level is computed
//                in the kernel from the source table, so only the phase state
//                touches memory.  Warp vote skips the model when every lane is
//                cold and saturated (active set, reading A9).
//  k_step_ext    ms_step: one explicit step with temperatures read from memory
//                (Algorithm 1 with the local step of Algorithm 2).
//  k_set_state / k_get_state / k_fractions   natural order <-> padded layout.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ms_internal.h"

namespace ms {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kLog2e = 1.4426950408889634074;

// --------------------------------------------------------- source table
__global__ void k_src_table(const TableArgs a) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= a.n_specs * a.n_levels) return;
  const int s = id / a.n_levels;
  const int lv = id - s * a.n_levels;
  const SpecDev& sp = a.specs[s];
  const double tl = a.t_base + double(a.n0 + lv) * a.dt - sp.t_offset;
  int l = 0;
  for (int j = 0; j < sp.n_layers; ++j)
    if (a.layers[sp.layer0 + j].t_begin <= tl) l = j;
  const LayerDev L = a.layers[sp.layer0 + l];
  double scale = 1.0;
  if (tl > L.t_scan_end) {
    const double span = L.t_end - L.t_scan_end;
    scale = span > 0.0 ? 1.0 - (tl - L.t_scan_end) / span : 0.0;
    if (scale < 0.0) scale = 0.0;
  }
  const double C0 = sp.A / (2.0 * kPi * sp.k) * scale;
  const double cv = -kLog2e / (2.0 * sp.alpha);
  SrcEntry* out = a.entries + (int64_t(s) * a.n_levels + lv) * a.slots;
  int n = 0;
  for (int j = 0; j < sp.n_tracks && n < a.slots; ++j) {
    const TrackDev tr = a.tracks[sp.track0 + j];
    if (tr.layer != l || tl < tr.t_start) continue;
    const double travel = tr.v * (tl - tr.t_start);
    const double sx = tr.x0 + tr.ux * travel, sy = tr.y0 + tr.uy * travel;
    const double C = C0 * tr.P;
    SrcEntry e;
    e.s_xi = float(sx * tr.ux + sy * tr.uy);
    e.s_pp = float(sx * tr.uy - sy * tr.ux);
    e.ux = float(tr.ux);
    e.uy = float(tr.uy);
    e.cR = float(cv * tr.v);
    e.lC = C > 0.0 ? float(log2(C)) : -INFINITY;
    e.pad0 = e.pad1 = 0.0f;
    out[n++] = e;
  }
  SrcLevel r;
  r.n = n;
  r.z_surf = float(L.z);
  r.T0 = sp.T0;
  r.T_max = sp.T_max;
  a.levels[id] = r;
}

__device__ __forceinline__ SrcEntry load_entry(const SrcEntry* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  SrcEntry e;
  e.s_xi = a.x; e.s_pp = a.y; e.ux = a.z; e.uy = a.w;
  e.cR = b.x; e.lC = b.y; e.pad0 = b.z; e.pad1 = b.w;
  return e;
}

__device__ __forceinline__ float depth2(float pz, float z_surf) {
  const float dz = pz - z_surf;
  return fmaf(dz, dz, 1e-30f);
}

// Temperatures of 4 points at one level (4 independent chains per source).
__device__ __forceinline__ void temps4(const SrcLevel& L, const SrcEntry* en, const float* px,
                                       const float* py, const float* pz, float* T) {
  float acc[4] = {0.f, 0.f, 0.f, 0.f}, dz2[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) dz2[q] = depth2(pz[q], L.z_surf);
  for (int j = 0; j < L.n; ++j) {
    const SrcEntry e = load_entry(en + j);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += source_term(e, px[q], py[q], dz2[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) T[q] = fminf(L.T0 + acc[q], L.T_max);
}

__device__ __forceinline__ float temp1(const SrcLevel& L, const SrcEntry* en, float px, float py,
                                       float pz) {
  float acc = 0.f;
  const float dz2 = depth2(pz, L.z_surf);
  for (int j = 0; j < L.n; ++j) acc += source_term(load_entry(en + j), px, py, dz2);
  return fminf(L.T0 + acc, L.T_max);
}

// ---------------------------------------------------------- state access
template <typename FT>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  static __device__ __forceinline__ void store(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void load(const double* p, double* v) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void store(double* p, const double* v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

template <typename FT>
__device__ __forceinline__ bool finite_pair(FT a, FT b) {
  return isfinite(a) && isfinite(b);
}

// ------------------------------------------------------------ hot kernel
template <typename FT>
// Minimum resident 256-thread blocks per SM for k_track: 3 caps it at 85
// registers (24 resident warps at 128 threads per block), measured fastest on
// the 256x256x64 block against 1 (107 registers) and 4 (64, with spills).
#ifndef MS_TRACK_MINB
#define MS_TRACK_MINB 3
#endif
__global__ void __launch_bounds__(256, MS_TRACK_MINB) k_track(const TrackArgs<FT> a) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.n_work) return;
  const int tile = a.tile_list ? a.tile_list[w] : int(w);
  const int s = a.tile_spec[tile];
  const SpecDev& sp = a.specs[s];
  const int64_t local0 = int64_t(tile - sp.tile0) * TILE + lane * 4;
  const int64_t g0 = sp.pad_off + local0;

  float px[4], py[4], pz[4];
  bool valid[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t li = local0 + q;
    valid[q] = li < sp.n;
    const int64_t ii = valid[q] ? li : 0;
    const int64_t r = ii / sp.nx;
    const int64_t i = ii - r * sp.nx;
    const int64_t k = r / sp.ny;
    const int64_t j = r - k * sp.ny;
    px[q] = sp.ox + float(i) * sp.dx;
    py[q] = sp.oy + float(j) * sp.dy;
    pz[q] = sp.oz + float(k) * sp.dz;
  }

  FT xs[4], xm[4];
  float ax[4];
  Vec4<FT>::load(a.xas + g0, xs);
  Vec4<FT>::load(a.xam + g0, xm);
  Vec4<float>::load(a.aux + g0, ax);

  const SrcLevel* lv = a.levels + int64_t(s) * a.n_levels;
  const SrcEntry* en = a.entries + int64_t(s) * a.n_levels * a.slots;
  const float z_tol = sp.z_tol;
  const bool skipping = a.m.T_thr > 0.0f;

  float T0[4];
  temps4(lv[0], en, px, py, pz, T0);
  for (int l = 1; l < a.n_levels; ++l) {
    const SrcLevel L = lv[l];
    float T1[4];
    temps4(L, en + int64_t(l) * a.slots, px, py, pz, T1);
    const float zlim = L.z_surf + z_tol;
    bool noop = true;
    if (skipping) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        noop = noop && (!valid[q] || !(pz[q] <= zlim) ||
                        step_is_noop<FT>(a.m, T0[q], T1[q], xs[q], xm[q], ax[q]));
    }
    if (!(skipping && __all_sync(0xffffffffu, noop))) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (valid[q] && pz[q] <= zlim) point_step<FT>(a.m, T0[q], T1[q], a.dt, xs[q], xm[q], ax[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) T0[q] = T1[q];
  }

  Vec4<FT>::store(a.xas + g0, xs);
  Vec4<FT>::store(a.xam + g0, xm);
  Vec4<float>::store(a.aux + g0, ax);
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) ok = ok && finite_pair(xs[q], xm[q]);
  if (!ok) atomicOr(a.err, DEVERR_NONFINITE);
}

// ---------------------------------------------------- external T (ms_step)
template <typename FT>
__global__ void __launch_bounds__(256) k_step_ext(const StepArgs<FT> a, int vec_T) {
  const int64_t i0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 4;
  if (i0 >= a.n) return;
  FT xs[4], xm[4];
  float ax[4], T0[4], T1[4];
  Vec4<FT>::load(a.xas + i0, xs);  // state arrays are padded to whole tiles
  Vec4<FT>::load(a.xam + i0, xm);
  Vec4<float>::load(a.aux + i0, ax);
  const int cnt = a.n - i0 < 4 ? int(a.n - i0) : 4;
  if (vec_T && cnt == 4) {
    const float4 t0 = __ldcs(reinterpret_cast<const float4*>(a.T0 + i0));
    const float4 t1 = __ldcs(reinterpret_cast<const float4*>(a.T1 + i0));
    T0[0] = t0.x; T0[1] = t0.y; T0[2] = t0.z; T0[3] = t0.w;
    T1[0] = t1.x; T1[1] = t1.y; T1[2] = t1.z; T1[3] = t1.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T0[q] = q < cnt ? a.T0[i0 + q] : 300.0f;
      T1[q] = q < cnt ? a.T1[i0 + q] : 300.0f;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < cnt) point_step<FT>(a.m, T0[q], T1[q], a.dt, xs[q], xm[q], ax[q]);
  Vec4<FT>::store(a.xas + i0, xs);
  Vec4<FT>::store(a.xam + i0, xm);
  Vec4<float>::store(a.aux + i0, ax);
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) ok = ok && finite_pair(xs[q], xm[q]);
  if (!ok) atomicOr(a.err, DEVERR_NONFINITE);
}

// --------------------------------------------------------- layout kernels
__device__ __forceinline__ bool padded_to_natural(const SpecDev* specs, const int32_t* tile_spec,
                                                  int64_t g, int& s, int64_t& nat) {
  s = tile_spec[g / TILE];
  const SpecDev& sp = specs[s];
  const int64_t local = g - sp.pad_off;
  nat = sp.nat_off + local;
  return local < sp.n;
}

template <typename FT>
__global__ void k_set_state(const SpecDev* specs, const int32_t* tile_spec, int64_t n_pad,
                            const double* xas, const double* xam, const double* aux, FT* dxas,
                            FT* dxam, float* daux, double xas0, double xam0) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= n_pad) return;
  int s;
  int64_t nat;
  if (padded_to_natural(specs, tile_spec, g, s, nat)) {
    dxas[g] = xas ? FT(xas[nat]) : FT(xas0);
    dxam[g] = xam ? FT(xam[nat]) : FT(xam0);
    const double v = aux ? aux[nat] : 0.0;
    daux[g] = v > 0.0 ? float(log2(v)) : (v < 0.0 ? 1.0f : 0.0f);
  } else {
    dxas[g] = FT(0.9);
    dxam[g] = FT(0);
    daux[g] = 0.0f;
  }
}

template <typename FT>
__global__ void k_get_state(const SpecDev* specs, const int32_t* tile_spec, int64_t n_pad,
                            const FT* dxas, const FT* dxam, const float* daux, double* xas,
                            double* xam, double* aux) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= n_pad) return;
  int s;
  int64_t nat;
  if (!padded_to_natural(specs, tile_spec, g, s, nat)) return;
  if (xas) xas[nat] = double(dxas[g]);
  if (xam) xam[nat] = double(dxam[g]);
  if (aux) {
    const float L = daux[g];
    aux[nat] = L < 0.0f ? exp2(double(L)) : (L > 0.0f ? -1.0 : 0.0);
  }
}

template <typename FT>
__global__ void k_fractions(const ModelConst m, const SpecDev* specs, const int32_t* tile_spec,
                            int64_t n_pad, const FT* dxas, const FT* dxam, const float* T,
                            const SrcLevel* levels, const SrcEntry* entries, int32_t slots,
                            double* xbeta, double* xliq) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= n_pad) return;
  int s;
  int64_t nat;
  if (!padded_to_natural(specs, tile_spec, g, s, nat)) return;
  float Tp;
  if (T) {
    Tp = T[nat];
  } else {
    const SpecDev& sp = specs[s];
    const int64_t li = g - sp.pad_off;
    const int64_t r = li / sp.nx;
    const int64_t i = li - r * sp.nx;
    const int64_t k = r / sp.ny;
    const int64_t j = r - k * sp.ny;
    Tp = temp1(levels[s], entries + int64_t(s) * slots, sp.ox + float(i) * sp.dx,
               sp.oy + float(j) * sp.dy, sp.oz + float(k) * sp.dz);
  }
  const double gl = double(liquid_fraction(m, Tp));
  if (xbeta) xbeta[nat] = (1.0 - gl) - double(dxas[g]) - double(dxam[g]);
  if (xliq) xliq[nat] = gl;
}

inline unsigned blocks_for(int64_t n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

}  // namespace

// ------------------------------------------------------------- launchers
cudaError_t launch_src_table(const TableArgs& a, cudaStream_t stream) {
  const int n = a.n_specs * a.n_levels;
  if (n <= 0) return cudaSuccess;
  k_src_table<<<blocks_for(n, 128), 128, 0, stream>>>(a);
  return cudaGetLastError();
}

template <typename FT>
cudaError_t launch_track(const TrackArgs<FT>& a, int block_threads, cudaStream_t stream) {
  if (a.n_work <= 0) return cudaSuccess;
  const int warps_per_block = block_threads / 32;
  const unsigned grid = unsigned((a.n_work + warps_per_block - 1) / warps_per_block);
  k_track<FT><<<grid, block_threads, 0, stream>>>(a);
  return cudaGetLastError();
}

template <typename FT>
cudaError_t launch_step_ext(const StepArgs<FT>& a, int block_threads, cudaStream_t stream) {
  if (a.n <= 0) return cudaSuccess;
  const int vec = ((reinterpret_cast<uintptr_t>(a.T0) | reinterpret_cast<uintptr_t>(a.T1)) & 15) == 0;
  k_step_ext<FT><<<blocks_for((a.n + 3) / 4, block_threads), block_threads, 0, stream>>>(a, vec);
  return cudaGetLastError();
}

template <typename FT>
cudaError_t launch_set_state(const SpecDev* specs, const int32_t* tile_spec, int64_t n_tiles,
                             const double* xas, const double* xam, const double* aux, FT* dxas,
                             FT* dxam, float* daux, cudaStream_t stream, double xas0, double xam0) {
  const int64_t n_pad = n_tiles * TILE;
  k_set_state<FT><<<blocks_for(n_pad, 256), 256, 0, stream>>>(specs, tile_spec, n_pad, xas, xam,
                                                              aux, dxas, dxam, daux, xas0, xam0);
  return cudaGetLastError();
}

template <typename FT>
cudaError_t launch_get_state(const SpecDev* specs, const int32_t* tile_spec, int64_t n_tiles,
                             const FT* dxas, const FT* dxam, const float* daux, double* xas,
                             double* xam, double* aux, cudaStream_t stream) {
  const int64_t n_pad = n_tiles * TILE;
  k_get_state<FT><<<blocks_for(n_pad, 256), 256, 0, stream>>>(specs, tile_spec, n_pad, dxas, dxam,
                                                              daux, xas, xam, aux);
  return cudaGetLastError();
}

template <typename FT>
cudaError_t launch_fractions(const ModelConst& m, const SpecDev* specs, const int32_t* tile_spec,
                             int64_t n_tiles, const FT* dxas, const FT* dxam, const float* T,
                             const SrcLevel* levels, const SrcEntry* entries, int32_t slots,
                             double* xbeta, double* xliq, cudaStream_t stream) {
  const int64_t n_pad = n_tiles * TILE;
  k_fractions<FT><<<blocks_for(n_pad, 256), 256, 0, stream>>>(
      m, specs, tile_spec, n_pad, dxas, dxam, T, levels, entries, slots, xbeta, xliq);
  return cudaGetLastError();
}

#define MS_INSTANTIATE(FT)                                                                        \
  template cudaError_t launch_track<FT>(const TrackArgs<FT>&, int, cudaStream_t);                \
  template cudaError_t launch_step_ext<FT>(const StepArgs<FT>&, int, cudaStream_t);              \
  template cudaError_t launch_set_state<FT>(const SpecDev*, const int32_t*, int64_t,             \
                                            const double*, const double*, const double*, FT*,    \
                                            FT*, float*, cudaStream_t, double, double);          \
  template cudaError_t launch_get_state<FT>(const SpecDev*, const int32_t*, int64_t, const FT*,  \
                                            const FT*, const float*, double*, double*, double*,  \
                                            cudaStream_t);                                       \
  template cudaError_t launch_fractions<FT>(const ModelConst&, const SpecDev*, const int32_t*,   \
                                            int64_t, const FT*, const FT*, const float*,         \
                                            const SrcLevel*, const SrcEntry*, int32_t, double*,  \
                                            double*, cudaStream_t);

MS_INSTANTIATE(float)
MS_INSTANTIATE(double)

}  // namespace ms
