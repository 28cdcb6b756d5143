// Per-tile helpers shared by the plain and the hybrid hot kernels: point
// coordinates, source-table reads, the superposed moving-source temperature
// of 4 points per thread, 128-bit state access and the martensite saturation
// temperature that drives the active set.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "ms_internal.h"

namespace ms {

// A grid coordinate o + i d as one explicit FMA, so that every kernel and
// every index path (32- or 64-bit, grid or subset) rounds it the same way
// (a multiply and an add may be fused or not, depending on the code around
// them).
template <typename AT>
__device__ __forceinline__ AT grid_coord(AT o, AT i, AT d) {
  return Fn<AT>::fma(i, d, o);
}

// Coordinates of local point li of a specimen (a grid point, or the grid
// point idx[li] for a subset specimen).
template <typename AT>
__device__ __forceinline__ void point_coords(const SpecDev& sp, int64_t li, AT& x, AT& y, AT& z) {
  const int64_t ii = sp.idx ? sp.idx[li] : li;
  const int64_t r = ii / sp.nx;
  const int64_t i = ii - r * sp.nx;
  const int64_t k = r / sp.ny;
  const int64_t j = r - k * sp.ny;
  x = grid_coord<AT>(AT(sp.ox), AT(i), AT(sp.dx));
  y = grid_coord<AT>(AT(sp.oy), AT(j), AT(sp.dy));
  z = grid_coord<AT>(AT(sp.oz), AT(k + sp.k_off), AT(sp.dz));
}

// Coordinates of the four consecutive local points li0 .. li0 + 3 of a
// specimen; points with valid[q] false take point 0's, as point_coords(sp, 0)
// gives them.  One index decomposition per thread, then a carry per point
// instead of a division: the same integer indices, so the same coordinates.
// When the specimen's indices fit in 32 bits (every specimen below 2^31
// points) the indices stay 32-bit integers: a conversion from a 64-bit
// integer to floating point runs on the FP64 pipe.  col returns the column of
// point li0 (0 for a subset specimen).
template <typename AT>
__device__ __forceinline__ void point_coords4(const SpecDev& sp, int64_t li0, const bool* valid,
                                              AT* x, AT* y, AT* z, int64_t& col) {
  col = 0;
  if (sp.idx) {
#pragma unroll
    for (int q = 0; q < 4; ++q) point_coords<AT>(sp, valid[q] ? li0 + q : 0, x[q], y[q], z[q]);
    return;
  }
  const AT ox = AT(sp.ox), oy = AT(sp.oy), oz = AT(sp.oz);
  const AT dx = AT(sp.dx), dy = AT(sp.dy), dz = AT(sp.dz);
  if (sp.n + 4 < (int64_t(1) << 31) && sp.nz + sp.k_off < (1 << 30)) {
    const int32_t nx = sp.nx, ny = sp.ny;
    const uint32_t l = uint32_t(li0);
    const uint32_t r = l / uint32_t(nx);
    int32_t i = int32_t(l - r * uint32_t(nx));
    int32_t k = int32_t(r / uint32_t(ny));
    int32_t j = int32_t(r) - k * ny;
    col = i;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q > 0 && ++i == nx) {
        i = 0;
        if (++j == ny) {
          j = 0;
          ++k;
        }
      }
      const int32_t ii = valid[q] ? i : 0, jj = valid[q] ? j : 0, kk = valid[q] ? k : 0;
      x[q] = grid_coord<AT>(ox, AT(ii), dx);
      y[q] = grid_coord<AT>(oy, AT(jj), dy);
      z[q] = grid_coord<AT>(oz, AT(kk + sp.k_off), dz);
    }
    return;
  }
  const int64_t r = li0 / sp.nx;
  int64_t i = li0 - r * sp.nx;
  int64_t k = r / sp.ny;
  int64_t j = r - k * sp.ny;
  col = i;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q > 0 && ++i == sp.nx) {
      i = 0;
      if (++j == sp.ny) {
        j = 0;
        ++k;
      }
    }
    const int64_t ii = valid[q] ? i : 0, jj = valid[q] ? j : 0, kk = valid[q] ? k : 0;
    x[q] = grid_coord<AT>(ox, AT(ii), dx);
    y[q] = grid_coord<AT>(oy, AT(jj), dy);
    z[q] = grid_coord<AT>(oz, AT(kk + sp.k_off), dz);
  }
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
  e.cR = b.x; e.lC = b.y; e.hcR = b.z; e.pad1 = b.w;
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
// source_term).  Per point and source that leaves 11 instructions instead of
// 15 when the level is axis-aligned.  An odd last source takes the same form.
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
        acc[q] = source_term_x<AT>(e0, Fn<AT>::fma(px[q], e0.ux, x0), q0, acc[q]);
        acc[q] = source_term_x<AT>(e1, Fn<AT>::fma(px[q], e1.ux, x1), q1, acc[q]);
      }
    }
    if (j < L.n) {
      const SrcEntryT<AT> e0 = load_entry(en + j);
      AT x0, p0;
      source_offsets<AT>(e0, py[0], x0, p0);
      const AT q0 = Fn<AT>::fma(p0, p0, dz2);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = source_term_x<AT>(e0, Fn<AT>::fma(px[q], e0.ux, x0), q0, acc[q]);
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
        acc[q] = source_term_x<AT>(e0, Fn<AT>::fma(px[q], e0.ux, x0), Fn<AT>::fma(pp0, pp0, dz2), acc[q]);
        acc[q] = source_term_x<AT>(e1, Fn<AT>::fma(px[q], e1.ux, x1), Fn<AT>::fma(pp1, pp1, dz2), acc[q]);
      }
    }
    if (j < L.n) {
      const SrcEntryT<AT> e0 = load_entry(en + j);
      AT x0, p0;
      source_offsets<AT>(e0, py[0], x0, p0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const AT pp0 = Fn<AT>::fma(px[q], e0.uy, p0);
        acc[q] = source_term_x<AT>(e0, Fn<AT>::fma(px[q], e0.ux, x0), Fn<AT>::fma(pp0, pp0, dz2), acc[q]);
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
        acc[q] = source_term<AT>(e0, px[q], py[q], dz2[q], acc[q]);
        acc[q] = source_term<AT>(e1, px[q], py[q], dz2[q], acc[q]);
      }
    }
    if (j < L.n) {
      const SrcEntryT<AT> e0 = load_entry(en + j);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = source_term<AT>(e0, px[q], py[q], dz2[q], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) T[q] = Fn<AT>::min(L.T0 + acc[q], L.T_max);
}

// temps4 at two levels with the same number of sources, for a row tile
// whose levels both move along +-x (temps4's first form): one loop over the
// sources evaluates both levels, each level summing its sources in order as
// temps4 does, so each level gets temps4's bits.
__device__ __forceinline__ void temps4_x2(const SrcLevelT<float>& La, const SrcEntryT<float>* ea,
                                          const SrcLevelT<float>& Lb, const SrcEntryT<float>* eb,
                                          const float* px, float py, float pz, float* Ta,
                                          float* Tb) {
  float acc_a[4] = {0.0f, 0.0f, 0.0f, 0.0f}, acc_b[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float dza = depth2<float>(pz, La.z_surf), dzb = depth2<float>(pz, Lb.z_surf);
  for (int j = 0; j < La.n; ++j) {
    const SrcEntryT<float> e0 = load_entry(ea + j), e1 = load_entry(eb + j);
    float x0, p0, x1, p1;
    source_offsets<float>(e0, py, x0, p0);
    source_offsets<float>(e1, py, x1, p1);
    const float q0 = fmaf(p0, p0, dza), q1 = fmaf(p1, p1, dzb);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc_a[q] = source_term_x<float>(e0, fmaf(px[q], e0.ux, x0), q0, acc_a[q]);
      acc_b[q] = source_term_x<float>(e1, fmaf(px[q], e1.ux, x1), q1, acc_b[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    Ta[q] = fminf(La.T0 + acc_a[q], La.T_max);
    Tb[q] = fminf(Lb.T0 + acc_b[q], Lb.T_max);
  }
}

// Dynamic shared memory of the far-field kernel: the interpolation weights
// and node positions (FF_FLOATS floats, see ms_internal.h).
extern __shared__ float4 ms_ff_smem[];

// temps4 with the far field (ms_params.farfield_dist > 0) for a tile inside
// one grid row at a level whose sources all move along +-x.  A source that
// lies at least dist behind every point of the tile's x-range [x_first,
// x_first + x_span] is summed at the range's FF_NODES Chebyshev nodes
// instead of at the 128 points: lane (k, g) = (lane & 7, lane >> 3) evaluates
// node k (at x_first + x_span s_node) for every fourth far source, the four
// groups' partial sums are added across the warp, and each lane interpolates
// its four points with the Lagrange weights [k][point] of the table ffw
// (FF_FLOATS floats: k_track keeps it in shared memory, ms_ff_smem; the
// hybrid kernel, whose shared memory holds the network, reads it through the
// caches).  The other sources are summed point by point as in temps4.
// n_near and n_far return the level's two counts (warp-uniform).  py and pz
// are the row's y and z in every lane (lane 0's first point, broadcast): a
// lane whose four points all lie past the specimen's end (a ragged last
// tile) holds point 0's coordinates, and the node sums of all lanes are added
// across the warp.
__device__ __forceinline__ void temps4_far(const SrcLevelT<float>& L, const SrcEntryT<float>* en,
                                           const float* px, float py, float pz, float x_first,
                                           float x_span, float dist, int lane, float* T,
                                           int& n_near, int& n_far, const float* ffw) {
  constexpr unsigned FULL = 0xffffffffu;
  const float dz2 = depth2<float>(pz, L.z_surf);
  const int g = lane >> 3;
  const float xk = fmaf(x_span, ffw[FF_NODES * TILE + (lane & (FF_NODES - 1))], x_first);
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  float fk = 0.0f;
  int nn = 0, nf = 0;
  for (int j0 = 0; j0 < L.n; j0 += 32) {
    const int cnt = L.n - j0 < 32 ? L.n - j0 : 32;
    bool far = false;
    if (lane < cnt) {
      // xi = x u_x - s_xi (u_y = 0 at this level); its largest value on the range
      const SrcEntryT<float> e = load_entry(en + j0 + lane);
      const float xa = fmaf(x_first, e.ux, -e.s_xi), xb = fmaf(x_first + x_span, e.ux, -e.s_xi);
      far = fmaxf(xa, xb) <= -dist;
    }
    const unsigned fm = __ballot_sync(FULL, far);
    const unsigned all = cnt == 32 ? FULL : (1u << cnt) - 1u;
    nf += __popc(fm);
    nn += cnt - __popc(fm);
    for (unsigned m = all & ~fm; m; m &= m - 1) {
      const SrcEntryT<float> e0 = load_entry(en + j0 + __ffs(m) - 1);
      float x0, p0;
      source_offsets<float>(e0, py, x0, p0);
      const float q0 = fmaf(p0, p0, dz2);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = source_term_x<float>(e0, fmaf(px[q], e0.ux, x0), q0, acc[q]);
    }
    for (int j = g; j < cnt; j += 4)
      if ((fm >> j) & 1u) {
        const SrcEntryT<float> e0 = load_entry(en + j0 + j);
        float x0, p0;
        source_offsets<float>(e0, py, x0, p0);
        fk = source_term_x<float>(e0, fmaf(xk, e0.ux, x0), fmaf(p0, p0, dz2), fk);
      }
  }
  if (nf > 0) {
    fk += __shfl_xor_sync(FULL, fk, 8);
    fk += __shfl_xor_sync(FULL, fk, 16);
#pragma unroll
    for (int k = 0; k < FF_NODES; ++k) {
      const float F = __shfl_sync(FULL, fk, k);
      const float4 w = reinterpret_cast<const float4*>(ffw + k * TILE)[lane];
      acc[0] = fmaf(w.x, F, acc[0]);
      acc[1] = fmaf(w.y, F, acc[1]);
      acc[2] = fmaf(w.z, F, acc[2]);
      acc[3] = fmaf(w.w, F, acc[3]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) T[q] = fminf(L.T0 + acc[q], L.T_max);
  n_near = nn;
  n_far = nf;
}

// For a tile whose points lie in two consecutive grid rows, points 0 .. m - 1
// in the first: the second row's y and z, point m's (every lane must call
// this with the same m; point m is always a point of the specimen).
__device__ __forceinline__ void second_row_yz(const float* py, const float* pz, int m, float& y_b,
                                              float& z_b) {
  const int q = m & 3;
  const float y = q == 0 ? py[0] : (q == 1 ? py[1] : (q == 2 ? py[2] : py[3]));
  const float z = q == 0 ? pz[0] : (q == 1 ? pz[1] : (q == 2 ? pz[2] : pz[3]));
  y_b = __shfl_sync(0xffffffffu, y, m >> 2);
  z_b = __shfl_sync(0xffffffffu, z, m >> 2);
}

// temps4_far for a tile whose points lie in two consecutive grid rows: the
// first m points in row A (y_a, z_a) from x_first_a on, the others in row B
// (y_b, z_b) from the grid's first column on.  Row B's points take the
// range [x_first_b, x_first_b + x_span] with x_first_b = x_first_a of B's
// first point minus m columns, so that point p of the tile sits at position
// p / 127 of its own row's range and one table of weights serves both.  A
// source is far when it is far from both ranges; its node sums are taken at
// 8 nodes of each range (lane (k, r, g) = (lane & 7, lane >> 3 & 1, lane >>
// 4): node k of range r for every second far source), and each point
// interpolates from its own row's nodes.  The near sources are summed point
// by point at each point's row (as temps4 sums them for such a tile: the same
// bits where no source is far).  n_near, n_far: the level's counts
// (warp-uniform); the node evaluations are 2 FF_NODES per far source.
__device__ __forceinline__ void temps4_far2(const SrcLevelT<float>& L, const SrcEntryT<float>* en,
                                            const float* px, float y_a, float z_a, float y_b,
                                            float z_b, int m, float x_first_a, float x_first_b,
                                            float x_span, float dist, int lane, float* T,
                                            int& n_near, int& n_far, const float* ffw) {
  constexpr unsigned FULL = 0xffffffffu;
  const float dza = depth2<float>(z_a, L.z_surf), dzb = depth2<float>(z_b, L.z_surf);
  bool in_b[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) in_b[q] = lane * 4 + q >= m;
  const int r = (lane >> 3) & 1, g = lane >> 4;
  const float s_k = ffw[FF_NODES * TILE + (lane & (FF_NODES - 1))];
  const float xk = fmaf(x_span, s_k, r ? x_first_b : x_first_a);
  const float yk = r ? y_b : y_a, dzk = r ? dzb : dza;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  float fk = 0.0f;
  int nn = 0, nf = 0;
  for (int j0 = 0; j0 < L.n; j0 += 32) {
    const int cnt = L.n - j0 < 32 ? L.n - j0 : 32;
    bool far = false;
    if (lane < cnt) {
      const SrcEntryT<float> e = load_entry(en + j0 + lane);
      const float xa = fmaf(x_first_a, e.ux, -e.s_xi), xb = fmaf(x_first_a + x_span, e.ux, -e.s_xi);
      const float xc = fmaf(x_first_b, e.ux, -e.s_xi), xd = fmaf(x_first_b + x_span, e.ux, -e.s_xi);
      far = fmaxf(fmaxf(xa, xb), fmaxf(xc, xd)) <= -dist;
    }
    const unsigned fm = __ballot_sync(FULL, far);
    const unsigned all = cnt == 32 ? FULL : (1u << cnt) - 1u;
    nf += __popc(fm);
    nn += cnt - __popc(fm);
    for (unsigned mm = all & ~fm; mm; mm &= mm - 1) {
      const SrcEntryT<float> e0 = load_entry(en + j0 + __ffs(mm) - 1);
      float x0a, p0a, x0b, p0b;
      source_offsets<float>(e0, y_a, x0a, p0a);
      source_offsets<float>(e0, y_b, x0b, p0b);
      const float qa = fmaf(p0a, p0a, dza), qb = fmaf(p0b, p0b, dzb);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        acc[q] = source_term_x<float>(e0, fmaf(px[q], e0.ux, in_b[q] ? x0b : x0a),
                                      in_b[q] ? qb : qa, acc[q]);
    }
    for (int j = g; j < cnt; j += 2)
      if ((fm >> j) & 1u) {
        const SrcEntryT<float> e0 = load_entry(en + j0 + j);
        float x0, p0;
        source_offsets<float>(e0, yk, x0, p0);
        fk = source_term_x<float>(e0, fmaf(xk, e0.ux, x0), fmaf(p0, p0, dzk), fk);
      }
  }
  if (nf > 0) {
    fk += __shfl_xor_sync(FULL, fk, 16);
#pragma unroll
    for (int k = 0; k < FF_NODES; ++k) {
      const float Fa = __shfl_sync(FULL, fk, k), Fb = __shfl_sync(FULL, fk, k + FF_NODES);
      const float4 w = reinterpret_cast<const float4*>(ffw + k * TILE)[lane];
      acc[0] = fmaf(w.x, in_b[0] ? Fb : Fa, acc[0]);
      acc[1] = fmaf(w.y, in_b[1] ? Fb : Fa, acc[1]);
      acc[2] = fmaf(w.z, in_b[2] ? Fb : Fa, acc[2]);
      acc[3] = fmaf(w.w, in_b[3] ? Fb : Fa, acc[3]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) T[q] = fminf(L.T0 + acc[q], L.T_max);
  n_near = nn;
  n_far = nf;
}

// Temperature of one point; the same arithmetic and order as temps4.
template <typename AT>
__device__ __forceinline__ AT temp1(const SrcLevelT<AT>& L, const SrcEntryT<AT>* en, AT px, AT py,
                                    AT pz) {
  AT acc = AT(0);
  const AT dz2 = depth2<AT>(pz, L.z_surf);
  for (int j = 0; j < L.n; ++j) acc = source_term<AT>(load_entry(en + j), px, py, dz2, acc);
  return Fn<AT>::min(L.T0 + acc, L.T_max);
}

// Highest T1 at which martensite formation would still change this point
// (formation is a no-op for T1 >= the returned value); +inf while an App. A
// initiation runs (never skip), -FLT_MAX if formation can never act, and
// -inf only on the alpha_s plateau's fixed point (X_as = 0.9, X_am = 0, no
// initiation): below T_as,end its step is the identity, since X_alpha^eq =
// 0.9 there, no rate acts and g changes nothing.  A tile's maximum is -inf
// exactly when all its points sit on that fixed point.
template <typename AT, typename FT>
__device__ __forceinline__ float point_tsat(const ModelConstT<AT>& m, FT xas, FT xam, float aux) {
  if (aux != 0.0f) return INFINITY;
  const FT q = FT(0.9) - xas;
  if (!(q > FT(0))) return xam == FT(0) ? -INFINITY : -FLT_MAX;
  const float r = float(xam * FT(0.9) / q);
  if (r >= XMAX) return -FLT_MAX;
  return float(m.T_am_start) + sfu_lg2(1.0f - r) / float(m.kam_l2);
}

// ------------------------------------------------ four points in lockstep
// The explicit step of a thread's four points in the FP32 path.  point_step
// is one dependent chain with branches for every point, so the four points of
// a thread run one after another.  Here the model's common branch is written
// as straight-line code over the four points, so their chains interleave.
// The common branch: no App. A initiation running (aux = 0) or starting
// (reading A5: X_alpha > X_alpha^eq on the bound 0.9 with no martensite;
// reading A6: X_as = 0 below X_alpha^eq).  If any point of the warp leaves
// it, the warp takes point_step for its points.  The optional parts (the
// exponentials of the equilibria, the alpha_s -> beta rate, alpha_m ->
// alpha_s, the rescale of X_alpha > 0.9, the regularisation cap, martensite
// formation) run when any point of the warp needs them.  Every value is the
// same operation on the same operands as in point_step and correct, so the
// two give the same bits (a subset specimen, whose warps hold other points,
// checks that).  run[q] marks the points to advance; every lane of the warp
// must call this.
//
// xeq carries X_alpha^eq between consecutive steps: the correction of step n
// evaluates it at T^{n+1}, and the rates of step n + 1 need it at the same
// temperature, so with have_xeq (warp-uniform: the previous level took the
// lockstep step) the step reads it instead of evaluating it again (the same
// operation on the same operand, so the same bits).  Returns whether xeq
// holds X_alpha^eq(T1) on return.
//
// With IDLE (the dense one-step launch, where most warps hold points at rest)
// a warp whose points have X_alpha = X_alpha^eq and no martensite skips the
// rate constants, and one whose forming points all have X_as = 0.9 skips
// X_am^eq: both give exactly what the full evaluation gives (no rate acts;
// formation adds X_am^eq (0.9 - X_as) / 0.9 = 0), at two more votes per step,
// which the other launches, whose warps are mostly busy, do not pay.  With
// COLD (on with IDLE) a warp whose points all lie in the cold regime takes
// point_step4_cold (the same bits); k_track's busy warps measured 1 % slower
// with it, so k_track leaves it off.
//
// With INC (the wide fraction types, whose state the caller keeps in FP64 or
// as a compensated pair and passes here rounded to FP32) the step also
// returns the Euler increments dt * rate of both fractions (du) and, in mod,
// which of them the correction g changed (bit 2q for X_as, 2q + 1 for X_am):
// the caller adds an increment to its wide state, or takes g's FP32 value
// where g set it.  If a point of the warp takes an initiation (the rare
// branch), nothing is stepped and false is returned: the caller steps its
// wide state point by point.
// point_step4 for a warp whose points all lie in the cold regime
// T^n < T_as,end and T_inf <= T^{n+1} < T_am,start (room temperature up to
// the martensite start: most points of a part most of the time).  There
// X_alpha^eq = 0.9 at both levels, App. A's alpha_s -> beta entry cannot
// hold, the regularisation cap does not act and martensite formation takes
// its middle branch; this is point_step4's common branch with those choices
// made once for the warp instead of per point, so it gives the same bits.
// Used by point_step4's IDLE form; returns as point_step4 does.
template <typename OC>
__device__ __forceinline__ bool point_step4_cold(const ModelConstT<float>& m, const float* T0,
                                                 const float* T1, float dt, const bool* run,
                                                 float* xs, float* xm, float* ax, OC& oc,
                                                 float* xeq) {
  constexpr unsigned FULL = 0xffffffffu;
  using F = Fn<float>;
  float xa[4];
  // a warp whose points all have no initiation, X_alpha = 0.9 and no
  // martensite has no initiation to start either (that needs X_alpha <
  // 0.9): one vote tells both
  bool busy = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    xa[q] = xs[q] + xm[q];
    busy = busy || (run[q] && (ax[q] != 0.0f || xa[q] != 0.9f || xm[q] > 0.0f));
  }
  bool any_rate = __any_sync(FULL, busy);
  if (any_rate) {
    bool rare = false;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      rare = rare || (run[q] && (ax[q] != 0.0f || (xa[q] < 0.9f && xs[q] == 0.0f)));
    if (__any_sync(FULL, rare)) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (run[q]) point_step<float, float>(m, T0[q], T1[q], dt, xs[q], xm[q], ax[q], oc);
      return false;
    }
    any_rate = false;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      any_rate = any_rate || (run[q] && (xa[q] != 0.9f || xm[q] > 0.0f));
    any_rate = __any_sync(FULL, any_rate);
  }
  float nas[4], nam[4];
  if (!any_rate) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float d0 = 0.0f;
      nas[q] = euler_add<float, float>(xs[q], dt, d0);
      nam[q] = euler_add<float, float>(xm[q], dt, d0);
      if (run[q]) oc.add(1, 1);  // k_as
    }
  } else {
    float k[4], las[4], lg[4];
    bool any_hi = false, any_am = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      k[q] = k_alpha_s<float>(m, T0[q]);
      las[q] = F::lg2(xs[q]);
      lg[q] = 0.0f;
      any_hi = any_hi || (run[q] && xa[q] > 0.9f);
      any_am = any_am || (run[q] && xm[q] > 0.0f);
    }
    any_hi = __any_sync(FULL, any_hi);
    if (any_hi) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float gap = 0.9f - xa[q];
        lg[q] = gap > 0.0f ? F::lg2(gap) : -INFINITY;
      }
    }
    any_am = __any_sync(FULL, any_am);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool lo = xa[q] < 0.9f, hi = xa[q] > 0.9f;
      float d_as;
      if (any_hi) {
        const float kb = m.f * k[q];
        const float r = pow_rate<float>(lo ? k[q] : -kb, lo ? m.pa : m.pb, lo ? las[q] : lg[q],
                                        lo ? m.qa : m.qb, lo ? 0.9f - xa[q] : xa[q] - 0.9f);
        d_as = lo || hi ? r : 0.0f;
      } else {
        const float r = pow_rate<float>(k[q], m.pa, las[q], m.qa, 0.9f - xa[q]);
        d_as = lo ? r : 0.0f;
      }
      float d_am = 0.0f;
      if (any_am && xm[q] > 0.0f) {
        const float r2 = pow_rate<float>(k[q], m.pa, las[q], m.qa, xm[q]);
        d_as += r2;
        d_am = -r2;
      }
      nas[q] = euler_add<float, float>(xs[q], dt, d_as);
      nam[q] = euler_add<float, float>(xm[q], dt, d_am);
      if (run[q]) {
        oc.add(1, 1);  // k_as
        if (lo) oc.add(1, 2);
        if (hi) oc.add(1, 0.9f - xa[q] > 0.0f ? 2 : 1);
        if (xm[q] > 0.0f) oc.add(1, lo ? 1 : 2);
      }
    }
  }
  // eq:explicit_correction at T^{n+1}: no cap, X_alpha^eq = 0.9
  bool any_big = false, any_run = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    nas[q] = nas[q] > 0.0f ? nas[q] : 0.0f;
    nam[q] = nam[q] > 0.0f ? nam[q] : 0.0f;
    any_big = any_big || (run[q] && nas[q] + nam[q] > 0.9f);
    any_run = any_run || run[q];
  }
  if (__any_sync(FULL, any_big)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x = nas[q] + nam[q];
      if (x > 0.9f) {
        const float sc = 0.9f / x;
        nas[q] *= sc;
        nam[q] *= sc;
      }
    }
  }
  bool any_room = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (nas[q] + nam[q] > 0.9f) {
      const float v = 0.9f - nas[q];
      nam[q] = v > 0.0f ? v : 0.0f;
    }
    any_room = any_room || (run[q] && nas[q] != 0.9f);
  }
  // martensite formation, middle branch (T_inf <= T^{n+1} <= T_am,start)
  if (__any_sync(FULL, any_run)) {
    if (!__any_sync(FULL, any_room)) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (m.martensite_literal) nam[q] = 0.0f;
        if (run[q]) oc.add(1, 0);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float x0 = F::min(1.0f - F::ex2(m.kam_l2 * (T1[q] - m.T_am_start)), 0.9f);
        const float e = x0 * (0.9f - nas[q]) * float(1.0 / 0.9);
        if (m.martensite_literal) nam[q] = e;
        else if (e > nam[q]) nam[q] = e;
        if (run[q]) oc.add(1, 0);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (run[q]) {
      xs[q] = nas[q];
      xm[q] = nam[q];
    }
    xeq[q] = 0.9f;
  }
  return true;
}

template <typename OC, bool INC = false, bool IDLE = false, bool COLD = IDLE>
__device__ __forceinline__ bool point_step4(const ModelConstT<float>& m, const float* T0,
                                            const float* T1, float dt, const bool* run,
                                            float* xs, float* xm, float* ax, OC& oc, float* xeq,
                                            bool have_xeq, float* du_as = nullptr,
                                            float* du_am = nullptr, unsigned* mod = nullptr) {
  constexpr unsigned FULL = 0xffffffffu;
  using F = Fn<float>;
  if constexpr (COLD) {
    static_assert(!INC, "the cold-regime form is for the FP32 state");
    bool cold = true;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      cold = cold && T0[q] < m.T_as_end && T1[q] < m.T_am_start && !(T1[q] < m.T_inf);
    if (__all_sync(FULL, cold) && m.T_am_start < m.T_as_end && m.T_am_start <= m.T_as_start)
      return point_step4_cold(m, T0, T1, dt, run, xs, xm, ax, oc, xeq);
  }
  float xa[4], xeq0[4];
  bool mid0[4], any = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    xa[q] = xs[q] + xm[q];
    mid0[q] = !(T0[q] < m.T_as_end) && T0[q] <= m.T_as_start;
    any = any || (run[q] && mid0[q]);
  }
  // X_alpha^eq(T^n) (eq:equilibrium_phase_as)
  if (have_xeq) {
#pragma unroll
    for (int q = 0; q < 4; ++q) xeq0[q] = xeq[q];
  } else if (__any_sync(FULL, any)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float e = 1.0f - F::ex2(m.kaeq_l2 * (T0[q] - m.T_as_start));
      xeq0[q] = T0[q] < m.T_as_end ? 0.9f : (mid0[q] ? e : 0.0f);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) xeq0[q] = T0[q] < m.T_as_end ? 0.9f : 0.0f;
  }
  bool rare = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    // point_step's entry test of A5: X_alpha^eq < 0.9 <= X_alpha (the sign of
    // 0.9 - X_alpha is exact, and X_alpha > X_alpha^eq follows) with X_am = 0
    const bool enter5 = xm[q] == 0.0f && xa[q] >= 0.9f && xeq0[q] < 0.9f;
    const bool enter6 = xa[q] < xeq0[q] && xs[q] == 0.0f;
    rare = rare || (run[q] && (ax[q] != 0.0f || enter5 || enter6));
  }
  if (__any_sync(FULL, rare)) {
    if constexpr (!INC) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (run[q]) point_step<float, float>(m, T0[q], T1[q], dt, xs[q], xm[q], ax[q], oc);
    }
    return false;
  }

  // eq:explicit_integration with the rates at T^n; r1 and r3 exclude each
  // other and share one lg2 / lg2 / ex2 triple.  r1 and r3 carry a power of
  // |X_alpha^eq - X_alpha| and r2 one of X_am, so where every point of the
  // warp has X_alpha = X_alpha^eq and no martensite no rate acts: with IDLE
  // the warp then skips the rate constants and takes d = 0, as the rates give.
  float nas[4], nam[4];
  bool any_rate = !IDLE;
  if constexpr (IDLE) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      any_rate = any_rate || (run[q] && (xa[q] != xeq0[q] || xm[q] > 0.0f));
    any_rate = __any_sync(FULL, any_rate);
  }
  if (!any_rate) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float d0 = 0.0f;
      if constexpr (INC) {
        du_as[q] = __fmul_rn(dt, d0);
        du_am[q] = __fmul_rn(dt, d0);
        nas[q] = __fadd_rn(xs[q], du_as[q]);
        nam[q] = __fadd_rn(xm[q], du_am[q]);
      } else {
        nas[q] = euler_add<float, float>(xs[q], dt, d0);
        nam[q] = euler_add<float, float>(xm[q], dt, d0);
      }
      if (run[q]) {
        if (mid0[q]) oc.add(1, 0);
        oc.add(1, 1);  // k_as
      }
    }
  } else {
  float k[4], las[4], lg[4];
  bool any_hi = false, any_am = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    k[q] = k_alpha_s<float>(m, T0[q]);
    las[q] = F::lg2(xs[q]);
    lg[q] = 0.0f;
    any_hi = any_hi || (run[q] && xa[q] > xeq0[q]);
    any_am = any_am || (run[q] && xm[q] > 0.0f);
  }
  any_hi = __any_sync(FULL, any_hi);
  if (any_hi) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float gap = 0.9f - xa[q];
      lg[q] = gap > 0.0f ? F::lg2(gap) : -INFINITY;
    }
  }
  any_am = __any_sync(FULL, any_am);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool lo = xa[q] < xeq0[q], hi = xa[q] > xeq0[q];
    float d_as;
    if (any_hi) {  // r1 or r3 per point
      const float kb = m.f * k[q];
      const float r = pow_rate<float>(lo ? k[q] : -kb, lo ? m.pa : m.pb, lo ? las[q] : lg[q],
                                      lo ? m.qa : m.qb, lo ? xeq0[q] - xa[q] : xa[q] - xeq0[q]);
      d_as = lo || hi ? r : 0.0f;
    } else {       // no point of the warp above X_alpha^eq: r1 only
      const float r = pow_rate<float>(k[q], m.pa, las[q], m.qa, xeq0[q] - xa[q]);
      d_as = lo ? r : 0.0f;
    }
    float d_am = 0.0f;
    if (any_am && xm[q] > 0.0f) {
      const float r2 = pow_rate<float>(k[q], m.pa, las[q], m.qa, xm[q]);
      d_as += r2;
      d_am = -r2;
    }
    if constexpr (INC) {  // rounded product, then rounded sum: the caller adds du exactly so
      du_as[q] = __fmul_rn(dt, d_as);
      du_am[q] = __fmul_rn(dt, d_am);
      nas[q] = __fadd_rn(xs[q], du_as[q]);
      nam[q] = __fadd_rn(xm[q], du_am[q]);
    } else {
      nas[q] = euler_add<float, float>(xs[q], dt, d_as);
      nam[q] = euler_add<float, float>(xm[q], dt, d_am);
    }
    if (run[q]) {
      if (mid0[q]) oc.add(1, 0);
      oc.add(1, 1);                                      // k_as
      if (lo) oc.add(1, 2);
      if (hi) oc.add(1, 0.9f - xa[q] > 0.0f ? 2 : 1);
      if (xm[q] > 0.0f) oc.add(1, lo ? 1 : 2);
    }
  }
  }

  // eq:explicit_correction at T^{n+1}
  bool any_big = false, any_cap = false, any_mid1 = false, any_form = false;
  bool mid1[4], form[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    nas[q] = nas[q] > 0.0f ? nas[q] : 0.0f;
    nam[q] = nam[q] > 0.0f ? nam[q] : 0.0f;
    mid1[q] = !(T1[q] < m.T_as_end) && T1[q] <= m.T_as_start;
    form[q] = T1[q] < m.T_am_start;
    any_big = any_big || (run[q] && nas[q] + nam[q] > 0.9f);
    any_cap = any_cap || (run[q] && T1[q] > m.T_as_start);
    any_mid1 = any_mid1 || (run[q] && mid1[q]);
    any_form = any_form || (run[q] && form[q]);
  }
  if (__any_sync(FULL, any_big)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x = nas[q] + nam[q];
      if (x > 0.9f) {
        const float sc = 0.9f / x;
        nas[q] *= sc;
        nam[q] *= sc;
      }
    }
  }
  if (__any_sync(FULL, any_cap)) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (T1[q] > m.T_as_start) {
        const float cap = F::max(0.9f * (m.T_cap0 - T1[q]) * m.inv_T_reg, 0.0f);
        if (nas[q] > cap) nas[q] = cap;
      }
  }
  float xeq1[4];
  if (__any_sync(FULL, any_mid1)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float e = 1.0f - F::ex2(m.kaeq_l2 * (T1[q] - m.T_as_start));
      xeq1[q] = T1[q] < m.T_as_end ? 0.9f : (mid1[q] ? e : 0.0f);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) xeq1[q] = T1[q] < m.T_as_end ? 0.9f : 0.0f;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (nas[q] + nam[q] > xeq1[q]) {
      const float v = xeq1[q] - nas[q];
      nam[q] = v > 0.0f ? v : 0.0f;
    }
    if (run[q] && mid1[q]) oc.add(1, 0);
  }
  // Formation adds X_am^eq(T) (0.9 - X_as) / 0.9: nothing where X_as = 0.9,
  // whatever X_am^eq, so with IDLE a warp whose forming points all sit there
  // skips it (reading A3's literal form still sets X_am to that 0).
  bool any_room = !IDLE;
  const bool vote_form = __any_sync(FULL, any_form);
  if constexpr (IDLE) {
#pragma unroll
    for (int q = 0; q < 4; ++q) any_room = any_room || (run[q] && form[q] && nas[q] != 0.9f);
    any_room = __any_sync(FULL, any_room);
  }
  if (vote_form && !any_room) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (form[q]) {
        if (m.martensite_literal) nam[q] = 0.0f;
        if (run[q] && !(T1[q] < m.T_inf) && T1[q] <= m.T_am_start) oc.add(1, 0);
      }
  } else if (vote_form) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool ex = !(T1[q] < m.T_inf) && T1[q] <= m.T_am_start;
      const float x0 = T1[q] < m.T_inf
                           ? 0.9f
                           : (ex ? F::min(1.0f - F::ex2(m.kam_l2 * (T1[q] - m.T_am_start)), 0.9f)
                                 : 0.0f);
      if (form[q]) {
        const float e = x0 * (0.9f - nas[q]) * float(1.0 / 0.9);
        if (m.martensite_literal) nam[q] = e;
        else if (e > nam[q]) nam[q] = e;
        if (run[q] && ex) oc.add(1, 0);
      }
    }
  }
  if constexpr (INC) {
    unsigned mk = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nas[q] != __fadd_rn(xs[q], du_as[q])) mk |= 1u << (2 * q);
      if (nam[q] != __fadd_rn(xm[q], du_am[q])) mk |= 2u << (2 * q);
    }
    *mod = mk;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (run[q]) {
      xs[q] = nas[q];
      xm[q] = nam[q];
    }
    xeq[q] = xeq1[q];
  }
  return true;
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
