// Per-tile helpers shared by the plain and the hybrid hot kernels: point
// coordinates, source-table reads, the superposed moving-source temperature
// of 4 points per thread, 128-bit state access and the martensite saturation
// temperature that drives the active set.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ms_internal.h"

namespace ms {

// Coordinates of local point li of a specimen (a grid point, or the grid
// point idx[li] for a subset specimen).
template <typename AT>
__device__ __forceinline__ void point_coords(const SpecDev& sp, int64_t li, AT& x, AT& y, AT& z) {
  const int64_t ii = sp.idx ? sp.idx[li] : li;
  const int64_t r = ii / sp.nx;
  const int64_t i = ii - r * sp.nx;
  const int64_t k = r / sp.ny;
  const int64_t j = r - k * sp.ny;
  x = AT(sp.ox) + AT(i) * AT(sp.dx);
  y = AT(sp.oy) + AT(j) * AT(sp.dy);
  z = AT(sp.oz) + AT(k) * AT(sp.dz);
}

// Every point of the tile lies in one grid row (shares y and z): a full-grid
// specimen whose first and last point of the tile have the same row index.
// The tile's padding points take point 0's coordinates; their temperatures
// are never used.
__device__ __forceinline__ bool tile_in_one_row(const SpecDev& sp, int tile) {
  if (sp.idx) return false;
  const int64_t li0 = int64_t(tile - sp.tile0) * TILE;
  const int64_t li1 = li0 + TILE - 1 < sp.n - 1 ? li0 + TILE - 1 : sp.n - 1;
  return li0 / sp.nx == li1 / sp.nx;
}

__device__ __forceinline__ SrcEntryT<float> load_entry(const SrcEntryT<float>* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  SrcEntryT<float> e;
  e.s_xi = a.x; e.s_pp = a.y; e.ux = a.z; e.uy = a.w;
  e.cR = b.x; e.lC = b.y; e.pad0 = b.z; e.pad1 = b.w;
  return e;
}
__device__ __forceinline__ SrcEntryT<double> load_entry(const SrcEntryT<double>* p) {
  return *p;
}

template <typename AT>
__device__ __forceinline__ AT depth2(AT pz, AT z_surf) {
  const AT dz = pz - z_surf;
  return Fn<AT>::fma(dz, dz, AT(1e-30));
}

// Temperatures of 4 points at one level: two sources per iteration, so each
// thread runs 8 independent chains; the sum runs in source order.
//
// row (warp-uniform) says that every point of the tile shares py[0] and pz[0]
// (a tile inside one grid row).  Then the parts of a source's offsets that do
// not depend on x, and for a level whose sources all move along +-x the whole
// perp^2, are computed once per source instead of once per point: the same
// operations on the same operands, so the bits do not change (see
// source_term).  Per point and source that leaves 12 instructions instead of
// 16 when the level is axis-aligned.
template <typename AT>
__device__ __forceinline__ void temps4(const SrcLevelT<AT>& L, const SrcEntryT<AT>* en,
                                       const AT* px, const AT* py, const AT* pz, bool row,
                                       AT* T) {
  AT acc[4] = {AT(0), AT(0), AT(0), AT(0)};
  int j = 0;
  if (row && L.axis) {
    const AT dz2 = depth2<AT>(pz[0], L.z_surf);
    for (; j + 1 < L.n; j += 2) {
      const SrcEntryT<AT> e0 = load_entry(en + j), e1 = load_entry(en + j + 1);
      AT x0, p0, x1, p1;
      source_offsets<AT>(e0, py[0], x0, p0);
      source_offsets<AT>(e1, py[0], x1, p1);
      const AT q0 = Fn<AT>::fma(p0, p0, dz2), q1 = Fn<AT>::fma(p1, p1, dz2);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] += source_term_x<AT>(e0, Fn<AT>::fma(px[q], e0.ux, x0), q0);
        acc[q] += source_term_x<AT>(e1, Fn<AT>::fma(px[q], e1.ux, x1), q1);
      }
    }
  } else if (row) {
    const AT dz2 = depth2<AT>(pz[0], L.z_surf);
    for (; j + 1 < L.n; j += 2) {
      const SrcEntryT<AT> e0 = load_entry(en + j), e1 = load_entry(en + j + 1);
      AT x0, p0, x1, p1;
      source_offsets<AT>(e0, py[0], x0, p0);
      source_offsets<AT>(e1, py[0], x1, p1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const AT pp0 = Fn<AT>::fma(px[q], e0.uy, p0), pp1 = Fn<AT>::fma(px[q], e1.uy, p1);
        acc[q] += source_term_x<AT>(e0, Fn<AT>::fma(px[q], e0.ux, x0), Fn<AT>::fma(pp0, pp0, dz2));
        acc[q] += source_term_x<AT>(e1, Fn<AT>::fma(px[q], e1.ux, x1), Fn<AT>::fma(pp1, pp1, dz2));
      }
    }
  } else {
    AT dz2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) dz2[q] = depth2<AT>(pz[q], L.z_surf);
    for (; j + 1 < L.n; j += 2) {
      const SrcEntryT<AT> e0 = load_entry(en + j), e1 = load_entry(en + j + 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] += source_term<AT>(e0, px[q], py[q], dz2[q]);
        acc[q] += source_term<AT>(e1, px[q], py[q], dz2[q]);
      }
    }
  }
  if (j < L.n) {
    const SrcEntryT<AT> e0 = load_entry(en + j);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      acc[q] += source_term<AT>(e0, px[q], py[q], depth2<AT>(pz[q], L.z_surf));
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) T[q] = Fn<AT>::min(L.T0 + acc[q], L.T_max);
}

// Temperature of one point; the same arithmetic and order as temps4.
template <typename AT>
__device__ __forceinline__ AT temp1(const SrcLevelT<AT>& L, const SrcEntryT<AT>* en, AT px, AT py,
                                    AT pz) {
  AT acc = AT(0);
  const AT dz2 = depth2<AT>(pz, L.z_surf);
  for (int j = 0; j < L.n; ++j) acc += source_term<AT>(load_entry(en + j), px, py, dz2);
  return Fn<AT>::min(L.T0 + acc, L.T_max);
}

// Highest T1 at which martensite formation would still change this point
// (formation is a no-op for T1 >= the returned value); +inf while an App. A
// initiation runs (never skip), -inf if formation can never act.
template <typename AT, typename FT>
__device__ __forceinline__ float point_tsat(const ModelConstT<AT>& m, FT xas, FT xam, float aux) {
  if (aux != 0.0f) return INFINITY;
  const FT q = FT(0.9) - xas;
  if (!(q > FT(0))) return -INFINITY;
  const float r = float(xam * FT(0.9) / q);
  if (r >= XMAX) return -INFINITY;
  return float(m.T_am_start) + sfu_lg2(1.0f - r) / float(m.kam_l2);
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
template <>
struct Vec4<KF> {
  static __device__ __forceinline__ void load(const KF* p, KF* v) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    v[0] = KF(a.x, a.y); v[1] = KF(a.z, a.w); v[2] = KF(b.x, b.y); v[3] = KF(b.z, b.w);
  }
  static __device__ __forceinline__ void store(KF* p, const KF* v) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
  }
};

__device__ __forceinline__ bool finite1(float a) { return ::isfinite(a); }
__device__ __forceinline__ bool finite1(double a) { return ::isfinite(a); }
__device__ __forceinline__ bool finite1(KF a) { return ::isfinite(a.hi) && ::isfinite(a.lo); }

template <typename FT>
__device__ __forceinline__ bool finite_pair(FT a, FT b) {
  return finite1(a) && finite1(b);
}

}  // namespace ms
