// sm_103a kernels of the microstructure point solver.
//
//  k_src_table   per (specimen, time level): positions and constants of the
//                started moving sources (computed in FP64, stored in the
//                arithmetic type), so the hot kernel reads one entry per
//                source and level.
//  (k_active, the active-set compaction of reading A9, is in ms_active.cu)
//  k_track       the hot path of ms_run_track: persistent warps pull 128-point
//                tiles, 4 points per thread (128-bit SoA loads), S steps per
//                state load; the temperature of every point and level is
//                computed in the kernel from the source table, so only the
//                phase state touches memory.  A warp vote skips the model
//                when every lane is cold and saturated.
//  k_step_ext    ms_step: one explicit step with temperatures read from memory
//                (Algorithm 1 with the local step of Algorithm 2).
//  k_set_state / k_get_state / k_fractions   natural order <-> padded layout.
//  k_correct     the correction g alone on independent points (FP64), for the
//                surrogate's training targets.
//  k_verify      max |dX| between two contexts' fractions and max |sum - 1|.
//
// Kernels are templated on the arithmetic type AT (float on the SFU, double
// for the full-FP64 path) and the fraction type FT (float, double, KF).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "ms_internal.h"
#include "ms_tile.cuh"

namespace ms {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kLog2e = 1.4426950408889634074;


// --------------------------------------------------------- source table
// One warp per (specimen, level): the lanes take the specimen's tracks 32 at
// a time, a ballot numbers the started ones of the current layer in track
// order (their table slots), and each lane computes its own entry in FP64.
// Warps past the table write the active set's per-track window (TrackWin),
// one thread per track.
template <typename AT>
__device__ __forceinline__ void table_level(const TableArgs& a, int id, int lane) {
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
  SrcEntryT<AT>* out =
      static_cast<SrcEntryT<AT>*>(a.entries) + (int64_t(s) * a.n_levels + lv) * a.slots;
  int n = 0;
  bool axis = true, far = false;
  // the far field's test (a source at least ff_dist behind every point of a
  // row tile's x-range) against the whole x-range that row tiles can span:
  // where no source passes it here, none passes it for any tile
  double x_lo = 0.0, x_hi = 0.0, ffd = 0.0;
  if (a.ff_dist > 0.0) {
    const double ext = double(TILE - 1) * fabs(sp.dx);
    const double xe = sp.ox + double(sp.nx - 1) * sp.dx;
    x_lo = fmin(sp.ox, xe) - ext;
    x_hi = fmax(sp.ox, xe) + ext;
    ffd = fmax(a.ff_dist, double(FF_RANGE_GUARD) * ext) - 1e-6;  // margin over FP32 rounding
  }
  for (int j0 = 0; j0 < sp.n_tracks && n < a.slots; j0 += 32) {
    const int j = j0 + lane;
    TrackDev tr{};
    bool on = false;
    if (j < sp.n_tracks) {
      tr = a.tracks[sp.track0 + j];
      on = tr.layer == l && !(tl < tr.t_start);
    }
    const unsigned m = __ballot_sync(0xffffffffu, on);
    const int slot = n + __popc(m & ((1u << lane) - 1u));
    if (on && slot < a.slots) {
      const double travel = tr.v * (tl - tr.t_start);
      const double sx = tr.x0 + tr.ux * travel, sy = tr.y0 + tr.uy * travel;
      const double C = C0 * tr.P;
      SrcEntryT<AT> e;
      e.s_xi = AT(sx * tr.ux + sy * tr.uy);
      e.s_pp = AT(sx * tr.uy - sy * tr.ux);
      e.ux = AT(tr.ux);
      e.uy = AT(tr.uy);
      e.cR = AT(cv * tr.v);
      e.lC = C > 0.0 ? AT(log2(C)) : AT(-INFINITY);
      e.hcR = AT(-0.5 * cv * tr.v);
      e.pad1 = AT(0);
      out[slot] = e;
      axis = axis && e.uy == AT(0);
      if (a.ff_dist > 0.0) {
        const double sxi = sx * tr.ux + sy * tr.uy;
        far = far || fmin(x_lo * tr.ux - sxi, x_hi * tr.ux - sxi) <= -ffd;
      }
    }
    axis = __all_sync(0xffffffffu, axis);
    n += __popc(m);
  }
  far = __any_sync(0xffffffffu, far);
  if (lane == 0) {
    SrcLevelT<AT> r;
    r.n = n < a.slots ? n : a.slots;
    r.axis = axis ? (a.ff_dist > 0.0 && !far ? LEVEL_AXIS_NEAR : LEVEL_AXIS) : 0;
    r.z_surf = AT(L.z);
    r.T0 = AT(sp.T0);
    r.T_max = AT(sp.T_max);
    static_cast<SrcLevelT<AT>*>(a.levels)[id] = r;
  }
}

__device__ __forceinline__ void track_window(const TableArgs& a, int t) {
  const TrackDev tr = a.tracks[t];
  const SpecDev& sp = a.specs[tr.spec];
  const double tla = a.t_a - sp.t_offset, tlb = a.t_b - sp.t_offset;
  int la = 0, lb = 0;
  for (int j = 0; j < sp.n_layers; ++j) {
    if (a.layers[sp.layer0 + j].t_begin <= tla) la = j;
    if (a.layers[sp.layer0 + j].t_begin <= tlb) lb = j;
  }
  TrackWin w;
  w.on = !(tr.layer < la || tr.layer > lb || tr.t_start > tlb);
  const double ta = fmax(tla, tr.t_start);
  const double pa = tr.v * (ta - tr.t_start), pb = tr.v * (tlb - tr.t_start);
  w.ax = tr.x0 + tr.ux * pa;
  w.ay = tr.y0 + tr.uy * pa;
  w.bx = tr.x0 + tr.ux * pb;
  w.by = tr.y0 + tr.uy * pb;
  w.ux = float(tr.ux);
  w.uy = float(tr.uy);
  w.v = float(tr.v);
  w.cp = float(sp.A / (2.0 * kPi * sp.k) * tr.P);
  w.z = float(a.layers[sp.layer0 + tr.layer].z);
  a.win[t] = w;
}

template <typename AT>
__global__ void k_src_table(const TableArgs a, WorkCounters* work) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  if (gt == 0 && work) {
    work->n_active = 0;
    work->next = 0;
#pragma unroll
    for (int b = 0; b < COST_BUCKETS; ++b) work->n_bucket[b] = 0;
  }
  const int warp = gt >> 5, lane = threadIdx.x & 31;
  const int n_table = a.n_specs * a.n_levels;
  if (warp < n_table) {
    table_level<AT>(a, warp, lane);
  } else if (a.win) {
    const int t = gt - n_table * 32;
    if (t < a.n_tracks) track_window(a, t);
  }
}


__global__ void k_fill_f32(float* p, int64_t n, float v) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}



// ------------------------------------------------------------ hot kernel
// The FP32 explicit path advances a thread's four points in lockstep
// (point_step4); the other paths call point_step point by point.
template <typename AT, typename FT, bool IMPL>
constexpr bool kLockstep = std::is_same<AT, float>::value && std::is_same<FT, float>::value && !IMPL;
// The wide fraction types (MS_F64ACC, MS_KAHAN) take the same lockstep step on
// their state rounded to FP32 and add its Euler increments to the wide state
// (the FP32 arithmetic of the rates and the correction, the wide type only
// for the accumulation); where g sets a fraction, its FP32 value is taken.
template <typename AT, typename FT, bool IMPL>
constexpr bool kLockstepWide = std::is_same<AT, float>::value && !IMPL &&
                               (std::is_same<FT, double>::value || std::is_same<FT, KF>::value);

// One 128-point tile for the launch's S steps (4 points per lane).  OC counts
// the model's transcendentals per branch (SfuCount, MS_FLAG_COUNT_OPS) or
// compiles the counting away (NoCount).
template <typename AT, typename FT, bool IMPL, bool FAR, typename OC, bool TWO = false>
__device__ __forceinline__ void track_tile(const TrackArgs<AT, FT>& a, int tile, int lane,
                                           unsigned long long& n_src, unsigned long long& n_model,
                                           unsigned& fp_it, unsigned& fp_unconv, OC& oc,
                                           unsigned& n_ex2, unsigned& n_slow,
                                           unsigned long long& ff_nodes,
                                           unsigned long long& ff_pairs) {
  const int s = a.tile_spec[tile];
  const SpecDev& sp = a.specs[s];
  const int64_t local0 = int64_t(tile - sp.tile0) * TILE + lane * 4;
  const int64_t g0 = sp.pad_off + local0;

  AT px[4], py[4], pz[4];
  bool valid[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) valid[q] = local0 + q < sp.n;
  int64_t col;
  point_coords4<AT>(sp, local0, valid, px, py, pz, col);
  // the tile lies in one grid row when its first point's column (lane 0's)
  // plus its span stays inside the row (tile_in_one_row without dividing)
  const int64_t col0 = __shfl_sync(0xffffffffu, col, 0);
  const int64_t li_first = int64_t(tile - sp.tile0) * TILE;
  const int64_t span = sp.n - 1 - li_first < TILE - 1 ? sp.n - 1 - li_first : TILE - 1;
  const bool row = !sp.idx && col0 + span < sp.nx;
  // far field: the tile's x-range, first to 128th point (a row tile)
  AT x_first = AT(0), x_span = AT(0), ff_dist = AT(0), py_row = AT(0), pz_row = AT(0);
  if constexpr (FAR) {
    x_first = grid_coord<AT>(AT(sp.ox), AT(int32_t(col0)), AT(sp.dx));  // col0 < nx: 32-bit
    x_span = Fn<AT>::mul_rn(AT(TILE - 1), AT(sp.dx));  // rounded: never fused into x_first + x_span
    // never closer than FF_RANGE_GUARD tile ranges, whatever the grid spacing
    ff_dist = Fn<AT>::max(a.ff_dist, AT(FF_RANGE_GUARD) * Fn<AT>::abs(x_span));
    py_row = __shfl_sync(0xffffffffu, py[0], 0);  // lane 0's first point is always valid
    pz_row = __shfl_sync(0xffffffffu, pz[0], 0);
  }
  // a tile across two rows: the far field over both rows' ranges
  bool two = false;
  int m_two = 0;
  AT x_first_b = AT(0), y_b = AT(0), z_b = AT(0);
  if constexpr (FAR && TWO) {
    two = !sp.idx && !row && col0 + span < 2 * int64_t(sp.nx);
    if (two) {
      m_two = int(sp.nx - col0);
      x_first_b = grid_coord<AT>(AT(sp.ox), AT(-m_two), AT(sp.dx));
      second_row_yz(py, pz, m_two, y_b, z_b);
    }
  }

  FT xs[4], xm[4];
  float ax[4];
  Vec4<FT>::load(a.xas + g0, xs);
  Vec4<FT>::load(a.xam + g0, xm);
  Vec4<float>::load(a.aux + g0, ax);

  const SrcLevelT<AT>* lv = a.levels + int64_t(s) * a.n_levels;
  const SrcEntryT<AT>* en = a.entries + int64_t(s) * a.n_levels * a.slots;
  const AT z_tol = AT(sp.z_tol);
  const bool skipping = a.m.T_thr > AT(0);

  // valid points of this tile (all lanes agree): the work counters count them
  const int64_t rest = sp.n - int64_t(tile - sp.tile0) * TILE;
  const unsigned long long nv = (unsigned long long)(rest < TILE ? rest : TILE);
  unsigned srcs = 0, models = 0, fsrcs = 0, fsrcs2 = 0;  // per tile: <= 513 levels x slots
  AT T0[4];
  float xeq[4];          // lockstep path: X_alpha^eq at T0, when have_xeq
  bool have_xeq = false;
  for (int l = 0; l < a.n_levels; ++l) {  // level 0 only sets T0 (one inlined temps4)
    const SrcLevelT<AT> L = lv[l];
    AT T1[4];
    bool done_far = false;
    if constexpr (FAR) {
      if (row && L.axis == LEVEL_AXIS) {
        int nn, nf;
        temps4_far(L, en + int64_t(l) * a.slots, px, py_row, pz_row, x_first, x_span, ff_dist,
                   lane, T1, nn, nf, reinterpret_cast<const float*>(ms_ff_smem));
        srcs += nn;
        fsrcs += nf;
        done_far = true;
      } else if (TWO && two && L.axis == LEVEL_AXIS) {
        int nn, nf;
        temps4_far2(L, en + int64_t(l) * a.slots, px, py_row, pz_row, y_b, z_b, m_two, x_first,
                    x_first_b, x_span, ff_dist, lane, T1, nn, nf,
                    reinterpret_cast<const float*>(ms_ff_smem));
        srcs += nn;
        fsrcs += nf;
        fsrcs2 += nf;
        done_far = true;
      }
    }
    if (!done_far) {
      temps4<AT>(L, en + int64_t(l) * a.slots, px, py, pz, row, T1);
      srcs += L.n;
    }
    if (l == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) T0[q] = T1[q];
      continue;
    }
    const AT zlim = L.z_surf + z_tol;
    bool noop = true;
    if (skipping) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        noop = noop && (!valid[q] || !(pz[q] <= zlim) ||
                        step_is_noop<AT, FT>(a.m, T0[q], T1[q], xs[q], xm[q], ax[q]));
    }
    if (skipping && __all_sync(0xffffffffu, noop)) {
      have_xeq = false;
    } else {
      ++models;
      if constexpr (kLockstep<AT, FT, IMPL>) {
        bool run[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) run[q] = valid[q] && pz[q] <= zlim;
        have_xeq = point_step4(a.m, T0, T1, a.dt, run, xs, xm, ax, oc, xeq, have_xeq);
      } else if constexpr (kLockstepWide<AT, FT, IMPL>) {
        bool run[4];
        float fs[4], fm[4], du_s[4], du_m[4];
        unsigned mod = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          run[q] = valid[q] && pz[q] <= zlim;
          fs[q] = float(xs[q]);
          fm[q] = float(xm[q]);
        }
        have_xeq = point_step4<decltype(oc), true>(a.m, T0, T1, a.dt, run, fs, fm, ax, oc, xeq,
                                                   have_xeq, du_s, du_m, &mod);
        if (have_xeq) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (run[q]) {
              xs[q] = (mod >> (2 * q)) & 1u ? FT(fs[q]) : xs[q] + FT(du_s[q]);
              xm[q] = (mod >> (2 * q)) & 2u ? FT(fm[q]) : xm[q] + FT(du_m[q]);
            }
        } else {  // an initiation in the warp: the per-point step on the wide state
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (run[q]) point_step<AT, FT>(a.m, T0[q], T1[q], a.dt, xs[q], xm[q], ax[q], oc);
        }
      } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (valid[q] && pz[q] <= zlim) {
          if constexpr (IMPL)
            point_step_implicit<AT, FT>(a.m, T0[q], T1[q], a.dt, a.n_sub, xs[q], xm[q], ax[q],
                                        fp_it, fp_unconv);
          else
            point_step<AT, FT>(a.m, T0[q], T1[q], a.dt, xs[q], xm[q], ax[q], oc);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) T0[q] = T1[q];
  }

  Vec4<FT>::store(a.xas + g0, xs);
  Vec4<FT>::store(a.xam + g0, xm);
  Vec4<float>::store(a.aux + g0, ax);
  if constexpr (std::is_same<OC, SfuCount>::value) {
    n_ex2 += oc.packed & 0xffffu;
    n_slow += oc.packed >> 16;
    oc.packed = 0;
  }
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) ok = ok && finite_pair(xs[q], xm[q]);
  n_src += (unsigned long long)srcs * nv;
  n_model += (unsigned long long)models * nv;
  ff_nodes += (unsigned long long)(fsrcs + fsrcs2) * FF_NODES;  // two rows: 2 x 8 nodes
  ff_pairs += (unsigned long long)fsrcs * nv;
  if (!ok) atomicOr(a.err, DEVERR_NONFINITE);
  if (a.tile_tsat && skipping) {  // read by the active set, which runs only with T_thr > 0
    float ts = -INFINITY;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (valid[q]) ts = fmaxf(ts, point_tsat<AT, FT>(a.m, xs[q], xm[q], ax[q]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ts = fmaxf(ts, __shfl_xor_sync(0xffffffffu, ts, o));
    if (lane == 0) a.tile_tsat[tile] = ts + 0.5f;  // margin against FP32 rounding
  }
}

// The state of one tile (X_as, X_am, aux) into L2 with bulk prefetches: the
// padded arrays hold whole tiles, 16-byte aligned.
template <typename AT, typename FT>
__device__ __forceinline__ void prefetch_tile_state(const TrackArgs<AT, FT>& a, int tile) {
  const SpecDev& sp = a.specs[a.tile_spec[tile]];
  const int64_t g0 = sp.pad_off + int64_t(tile - sp.tile0) * TILE;
  const unsigned fb = unsigned(TILE * sizeof(FT)), ab = unsigned(TILE * sizeof(float));
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.xas + g0), "r"(fb) : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.xam + g0), "r"(fb) : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.aux + g0), "r"(ab) : "memory");
}

// Minimum resident 256-thread blocks per SM for k_track: 3 caps it at 85
// registers (24 resident warps at 128 threads per block), measured fastest on
// the 256x256x64 block against 1 (107 registers) and 4 (64, with spills).
#ifndef MS_TRACK_MINB
#define MS_TRACK_MINB 3
#endif
#ifndef MS_TRACK_MINB_FAR
#define MS_TRACK_MINB_FAR 3
#endif

// Persistent hot kernel: every warp pulls tiles (from the active list, or all
// tiles) through an atomic cursor until the work runs out, so the grid is
// sized to the resident capacity and no launch tail is left idle.
template <typename AT, typename FT, bool IMPL, bool FAR = false, bool CNT = false, bool TWO = false>
__global__ void __launch_bounds__(256, FAR ? MS_TRACK_MINB_FAR : MS_TRACK_MINB)
    k_track(const TrackArgs<AT, FT> a) {
  const int lane = threadIdx.x & 31;
  const int n_work = a.tile_list ? a.work->n_active : a.n_tiles;
  unsigned long long done = 0, n_src = 0, n_model = 0;
  unsigned fp_it = 0, fp_unconv = 0;
  std::conditional_t<CNT, SfuCount, NoCount> oc;
  unsigned n_ex2 = 0, n_slow = 0;
  unsigned long long ff_nodes = 0, ff_pairs = 0;
  // far field: every block copies the interpolation weights to shared memory
  if constexpr (FAR) {
    float* sm = reinterpret_cast<float*>(ms_ff_smem);
    for (int i = threadIdx.x; i < FF_FLOATS; i += blockDim.x) sm[i] = a.ff[i];
    __syncthreads();
  }
  int nb[COST_BUCKETS];
#pragma unroll
  for (int b = 0; b < COST_BUCKETS; ++b) nb[b] = a.tile_list ? a.work->n_bucket[b] : 0;
  unsigned long long cost_sum = 0;
  unsigned cost_n = 0;
  // Work is taken in chunks of consecutive positions, so that a launch with
  // many tiles per warp (one step per launch over a large grid) does not
  // queue on the cursor's atomic; with about one tile per warp (the active
  // set of a long launch) the chunk is one tile.  While a tile computes, the
  // next tile of the chunk has its state prefetched into L2.
  const int n_warps = int(gridDim.x) * int(blockDim.x >> 5);
  const int chunk = max(1, min(16, n_work / (8 * n_warps)));
  for (;;) {
    int w0 = 0;
    if (lane == 0) w0 = atomicAdd(&a.work->next, chunk);
    w0 = __shfl_sync(0xffffffffu, w0, 0);
    if (w0 >= n_work) break;
    const int w1 = min(w0 + chunk, n_work);
    int tile = a.tile_list ? list_tile(a.tile_list, a.n_tiles, nb, w0) : w0;
    for (int w = w0; w < w1; ++w) {
      const int next = w + 1 < w1 ? (a.tile_list ? list_tile(a.tile_list, a.n_tiles, nb, w + 1)
                                                  : w + 1)
                                  : -1;
      if (next >= 0 && lane == 0) prefetch_tile_state(a, next);
      const long long t0 = clock64();
      track_tile<AT, FT, IMPL, FAR, decltype(oc), TWO>(a, tile, lane, n_src, n_model, fp_it,
                                                         fp_unconv, oc, n_ex2,
                                    n_slow, ff_nodes, ff_pairs);
      if (a.tile_cost && lane == 0) {  // cycles per level, the next launch's ordering hint
        const long long dc = clock64() - t0;
        const unsigned per = unsigned(min(dc / (a.n_levels - 1 > 0 ? a.n_levels - 1 : 1),
                                          (long long)0x7fffffff));
        a.tile_cost[tile] = per;
        cost_sum += per;
        ++cost_n;
      }
      ++done;
      tile = next;
    }
  }
  if (a.tile_cost && lane == 0 && cost_n) {
    atomicAdd(&a.work->cost_sum[a.cost_slot & 1], cost_sum);
    atomicAdd(&a.work->cost_cnt[a.cost_slot & 1], cost_n);
  }
  if (CNT && a.ops) {
    unsigned long long e = n_ex2, sl = n_slow;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      sl += __shfl_xor_sync(0xffffffffu, sl, o);
    }
    if (lane == 0 && (e || sl)) {
      atomicAdd(&a.ops->model_sfu_ex2, e);
      atomicAdd(&a.ops->model_sfu_slow, sl);
    }
  }
  if constexpr (IMPL) {
    unsigned long long it = fp_it, un = fp_unconv;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      it += __shfl_xor_sync(0xffffffffu, it, o);
      un += __shfl_xor_sync(0xffffffffu, un, o);
    }
    if (lane == 0 && a.ops && it) {
      atomicAdd(&a.ops->fp_iterations, it);
      if (un) atomicAdd(&a.ops->fp_unconverged, un);
    }
  }
  if (lane == 0 && done) {
    atomicAdd(&a.work->tile_steps_active, done * (unsigned long long)(a.n_levels - 1));
    if (a.ops) {
      atomicAdd(&a.ops->source_evaluations, n_src);
      atomicAdd(&a.ops->model_point_steps, n_model);
      if (ff_nodes) {
        atomicAdd(&a.ops->farfield_node_evaluations, ff_nodes);
        atomicAdd(&a.ops->farfield_point_sources, ff_pairs);
      }
    }
  }
}

// ------------------------------------------------- dense one-step launches
// Exact division of a 32-bit unsigned by a runtime divisor d >= 1 through a
// multiply-high and two shifts (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Fig. 4.1): with
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
//   t = mulhi(m, n),  n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct UDiv {
  uint32_t m;
  uint32_t s1, s2;
  __device__ __forceinline__ void init(uint32_t d) {
    uint32_t l = 0;
    while (l < 32 && (uint64_t(1) << l) < d) ++l;
    m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    s1 = l < 1 ? l : 1;
    s2 = l > 1 ? l - 1 : 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

// The dense launch of one step: no active list (T_thr = 0), S = 1, the FP32
// explicit path.  Per tile it is k_track's arithmetic, in the same order and
// through the same helpers (temps4 / temps4_far at both levels, point_step4),
// so the two give the same bits; what differs is the organisation around it,
// for a launch that streams every tile's state from HBM once:
//  * tiles are dealt to warps in fixed chunks of DENSE_CHUNK consecutive
//    tiles, round robin, with no work cursor; the padded state arrays hold
//    the specimens' tiles in tile order (a specimen's pad_off is its first
//    tile times TILE), so tile t's state starts at t * TILE whatever its
//    specimen, and the warp bulk-prefetches its next chunk's state into L2
//    (three copies of DENSE_CHUNK tiles) when it starts a chunk;
//  * a warp keeps its specimen's grid data, the division constants of its
//    grid dimensions and the coordinate origin and spacing in FP32 in shared
//    memory while the specimen does not change, and a tile's first grid point
//    comes from two multiply-high divisions instead of two integer divisions;
//  * a row tile's points take x from the tile's first column plus the lane's
//    offset and the row's y and z (point_coords4 is used only for tiles that
//    cross a row and for subset specimens);
//  * the model step skips the rate constants and the martensite equilibrium
//    of warps at rest (point_step4's IDLE form: the same values);
//  * the non-finite check sums the eight fractions (bounded by 1 when
//    finite) and tests the sum.
#ifndef MS_DENSE_CHUNK
#define MS_DENSE_CHUNK 4
#endif
constexpr int DENSE_CHUNK = MS_DENSE_CHUNK;
constexpr int DENSE_THREADS = 128;
// Minimum resident 128-thread blocks per SM: 5 (102 registers, 20 warps)
// measured fastest on the 512 x 512 x 64 and x 256 grids against 4, 6, 7, 8.
#ifndef MS_DENSE_MINB
#define MS_DENSE_MINB 5
#endif

// The state of tiles t0 .. t1 - 1 (consecutive, t0 < t1) into L2.
__device__ __forceinline__ void prefetch_dense(const TrackArgs<float, float>& a, int t0, int t1) {
  const int64_t g0 = int64_t(t0) * TILE;
  const unsigned bytes = unsigned(t1 - t0) * unsigned(TILE * sizeof(float));
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.xas + g0), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.xam + g0), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.aux + g0), "r"(bytes) : "memory");
}

// A warp's specimen in shared memory (written by lane 0 when the specimen
// changes), so that the grid data does not hold registers across the tile.
struct DenseSpec {
  int64_t n;
  const SrcLevelT<float>* lv;  // the specimen's two levels
  const SrcEntryT<float>* en;  // and their sources
  int32_t tile0, nx, ny, k_off, sub, small;
  float z_tol, ox, oy, oz, dx, dy, dz;
  UDiv dvx, dvy;
};

template <bool FAR, bool TWO = false>
__global__ void __launch_bounds__(DENSE_THREADS, MS_DENSE_MINB) k_track_dense(const TrackArgs<float, float> a) {
  __shared__ DenseSpec spw[DENSE_THREADS / 32];
  const int lane = threadIdx.x & 31;
  const int warp = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int n_warps = int(gridDim.x * (blockDim.x >> 5));
  DenseSpec& ds = spw[threadIdx.x >> 5];
  if constexpr (FAR) {
    float* sm = reinterpret_cast<float*>(ms_ff_smem);
    for (int i = threadIdx.x; i < FF_FLOATS; i += blockDim.x) sm[i] = a.ff[i];
    __syncthreads();
  }
  NoCount oc;
  unsigned long long n_src = 0, n_model = 0, ff_nodes = 0, ff_pairs = 0;
  unsigned done = 0;
  int s_cur = -1;  // the warp's specimen (warp-uniform)
  if (lane == 0 && warp * DENSE_CHUNK < a.n_tiles)
    prefetch_dense(a, warp * DENSE_CHUNK, min((warp + 1) * DENSE_CHUNK, a.n_tiles));
  for (int c = warp; c * DENSE_CHUNK < a.n_tiles; c += n_warps) {
    const int c1 = c + n_warps;
    if (lane == 0 && c1 * DENSE_CHUNK < a.n_tiles)
      prefetch_dense(a, c1 * DENSE_CHUNK, min((c1 + 1) * DENSE_CHUNK, a.n_tiles));
    const int t_end = min((c + 1) * DENSE_CHUNK, a.n_tiles);
    // the chunk's counts, in 32 bits (a chunk's are far below 2^32)
    unsigned src_c = 0, model_c = 0, fsrc_c = 0, fpair_c = 0;
    // the grid indices of the previous tile's first point, where the next
    // tile's follow by one carry (rows of at least TILE points)
    int32_t ci = 0, cj = 0, ck = 0;
    bool have_ijk = false;
    for (int tile = c * DENSE_CHUNK; tile < t_end; ++tile) {
      const int s = a.tile_spec[tile];
      if (s != s_cur) {
        s_cur = s;
        have_ijk = false;
        if (lane == 0) {
          const SpecDev& sp = a.specs[s];
          ds.n = sp.n;
          ds.lv = a.levels + int64_t(s) * 2;
          ds.en = a.entries + int64_t(s) * 2 * a.slots;
          ds.tile0 = int32_t(sp.tile0);
          ds.nx = sp.nx;
          ds.ny = sp.ny;
          ds.k_off = sp.k_off;
          ds.sub = sp.idx != nullptr;
          ds.small = sp.idx == nullptr && sp.n + 4 < (int64_t(1) << 31) &&
                     sp.nz + sp.k_off < (1 << 30);
          ds.z_tol = sp.z_tol;
          ds.ox = float(sp.ox); ds.oy = float(sp.oy); ds.oz = float(sp.oz);
          ds.dx = float(sp.dx); ds.dy = float(sp.dy); ds.dz = float(sp.dz);
          ds.dvx.init(uint32_t(sp.nx));
          ds.dvy.init(uint32_t(sp.ny));
        }
        __syncwarp();
      }
      const bool small = ds.small != 0;
      int64_t li_first;
      int rem;  // points of the tile, 1 .. 128
      if (small) {
        const int32_t l32 = (tile - ds.tile0) * TILE, left = int32_t(ds.n) - l32;
        li_first = l32;
        rem = left < TILE ? left : TILE;
      } else {
        li_first = int64_t(tile - ds.tile0) * TILE;
        const int64_t left = ds.n - li_first;
        rem = left < TILE ? int(left) : TILE;
      }
      const int64_t g0 = int64_t(tile) * TILE + lane * 4;
      bool valid[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) valid[q] = lane * 4 + q < rem;

      float xs[4], xm[4], ax[4];
      Vec4<float>::load(a.xas + g0, xs);
      Vec4<float>::load(a.xam + g0, xm);
      Vec4<float>::load(a.aux + g0, ax);

      // the tile's first grid point; a row tile keeps one (j, k)
      float px[4], py[4], pz[4];
      bool row = false;
      int32_t col0 = 0;
      if (small) {  // 32-bit indices (the conversions stay off the FP64 pipe)
        int32_t i0, j0, k0;
        if (have_ijk) {
          i0 = ci + TILE;
          j0 = cj;
          k0 = ck;
          if (i0 >= ds.nx) {
            i0 -= ds.nx;
            if (++j0 == ds.ny) {
              j0 = 0;
              ++k0;
            }
          }
        } else {
          const uint32_t l = uint32_t(li_first);
          const uint32_t r = ds.dvx.div(l);
          i0 = int32_t(l - r * uint32_t(ds.nx));
          k0 = int32_t(ds.dvy.div(r));
          j0 = int32_t(r) - k0 * ds.ny;
        }
        ci = i0;
        cj = j0;
        ck = k0;
        have_ijk = ds.nx >= TILE;
        col0 = i0;
        row = i0 + rem - 1 < ds.nx;
        if (row) {
          // the points past the specimen's end (a ragged last tile) take the
          // row's coordinates too; their results are never stored
          const float ox = ds.ox, dx = ds.dx;
          const float y0 = grid_coord<float>(ds.oy, float(j0), ds.dy);
          const float z0 = grid_coord<float>(ds.oz, float(k0 + ds.k_off), ds.dz);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            px[q] = grid_coord<float>(ox, float(i0 + lane * 4 + q), dx);
            py[q] = y0;
            pz[q] = z0;
          }
        }
      }
      if (!row) {
        int64_t col;
        point_coords4<float>(a.specs[s], li_first + lane * 4, valid, px, py, pz, col);
        const int64_t c0 = __shfl_sync(0xffffffffu, col, 0);
        if (!ds.sub) {
          row = c0 + rem - 1 < ds.nx;
          col0 = int32_t(c0);
        }
      }
      // a tile across two rows: the far field over both rows' ranges
      bool two = false;
      int m_two = 0;
      float x_first_b = 0.f, y_b = 0.f, z_b = 0.f;
      if constexpr (FAR && TWO) {
        two = !row && !ds.sub && col0 + rem - 1 < 2 * ds.nx;
        if (two) {
          m_two = ds.nx - col0;
          x_first_b = grid_coord<float>(ds.ox, float(-m_two), ds.dx);
          second_row_yz(py, pz, m_two, y_b, z_b);
        }
      }

      const SrcLevelT<float>* lv = ds.lv;
      const SrcEntryT<float>* en = ds.en;
      const SrcLevelT<float> L0 = lv[0], L1 = lv[1];
      float T[2][4];
      unsigned srcs = 0, fsrcs = 0, fsrcs2 = 0;
      const bool far0 = FAR && row && L0.axis == LEVEL_AXIS;
      const bool far1 = FAR && row && L1.axis == LEVEL_AXIS;
      if (row && L0.axis && L1.axis && !far0 && !far1 && L0.n == L1.n) {
        temps4_x2(L0, en, L1, en + a.slots, px, py[0], pz[0], T[0], T[1]);
        srcs = 2u * unsigned(L0.n);
      } else {
        float x_first = 0.f, x_span = 0.f, ff_dist = 0.f, py_row = 0.f, pz_row = 0.f;
        if constexpr (FAR) {
          x_first = grid_coord<float>(ds.ox, float(col0), ds.dx);
          x_span = __fmul_rn(float(TILE - 1), ds.dx);
          ff_dist = fmaxf(a.ff_dist, float(FF_RANGE_GUARD) * fabsf(x_span));
          py_row = __shfl_sync(0xffffffffu, py[0], 0);
          pz_row = __shfl_sync(0xffffffffu, pz[0], 0);
        }
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const SrcLevelT<float>& L = l == 0 ? L0 : L1;
          if ((l == 0 ? far0 : far1)) {
            int nn, nf;
            temps4_far(L, en + int64_t(l) * a.slots, px, py_row, pz_row, x_first, x_span,
                       ff_dist, lane, T[l], nn, nf, reinterpret_cast<const float*>(ms_ff_smem));
            srcs += nn;
            fsrcs += nf;
          } else if (FAR && TWO && two && L.axis == LEVEL_AXIS) {
            int nn, nf;
            temps4_far2(L, en + int64_t(l) * a.slots, px, py_row, pz_row, y_b, z_b, m_two,
                        x_first, x_first_b, x_span, ff_dist, lane, T[l], nn, nf,
                        reinterpret_cast<const float*>(ms_ff_smem));
            srcs += nn;
            fsrcs += nf;
            fsrcs2 += nf;
          } else {
            temps4<float>(L, en + int64_t(l) * a.slots, px, py, pz, row, T[l]);
            srcs += L.n;
          }
        }
      }
      const float zlim = L1.z_surf + ds.z_tol;
      bool run[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) run[q] = valid[q] && pz[q] <= zlim;
      float xeq[4];
      point_step4<NoCount, false, true>(a.m, T[0], T[1], a.dt, run, xs, xm, ax, oc, xeq, false);

      Vec4<float>::store(a.xas + g0, xs);
      Vec4<float>::store(a.xam + g0, xm);
      Vec4<float>::store(a.aux + g0, ax);
      const float sum = ((xs[0] + xs[1]) + (xs[2] + xs[3])) + ((xm[0] + xm[1]) + (xm[2] + xm[3]));
      if (!::isfinite(sum)) atomicOr(a.err, DEVERR_NONFINITE);
      src_c += srcs * unsigned(rem);
      model_c += unsigned(rem);
      if constexpr (FAR) {
        fsrc_c += fsrcs + fsrcs2;  // node sets: two for a tile across two rows
        fpair_c += fsrcs * unsigned(rem);
      }
      ++done;
    }
    n_src += src_c;
    n_model += model_c;
    ff_nodes += (unsigned long long)fsrc_c * FF_NODES;
    ff_pairs += fpair_c;
  }
  if (lane == 0 && done) {
    atomicAdd(&a.work->tile_steps_active, (unsigned long long)done);
    if (a.ops) {
      atomicAdd(&a.ops->source_evaluations, n_src);
      atomicAdd(&a.ops->model_point_steps, n_model);
      if (ff_nodes) {
        atomicAdd(&a.ops->farfield_node_evaluations, ff_nodes);
        atomicAdd(&a.ops->farfield_point_sources, ff_pairs);
      }
    }
  }
}

// ---------------------------------------------------- external T (ms_step)
template <typename AT, typename FT, bool IMPL>
__global__ void __launch_bounds__(256) k_step_ext(const StepArgs<AT, FT> a, int vec_T) {
  const int64_t i0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 4;
  if constexpr (kLockstep<AT, FT, IMPL>) {
    // every lane of the warp takes part in point_step4's votes; lanes past
    // the end advance no point
    float xs[4] = {0.0f, 0.0f, 0.0f, 0.0f}, xm[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float ax[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float T0[4] = {300.0f, 300.0f, 300.0f, 300.0f}, T1[4] = {300.0f, 300.0f, 300.0f, 300.0f};
    const int cnt = i0 < a.n ? (a.n - i0 < 4 ? int(a.n - i0) : 4) : 0;
    if (cnt > 0) {
      Vec4<float>::load(a.xas + i0, xs);  // state arrays are padded to whole tiles
      Vec4<float>::load(a.xam + i0, xm);
      Vec4<float>::load(a.aux + i0, ax);
      if (vec_T && cnt == 4) {
        const float4 t0 = __ldcs(reinterpret_cast<const float4*>(a.T0 + i0));
        const float4 t1 = __ldcs(reinterpret_cast<const float4*>(a.T1 + i0));
        T0[0] = t0.x; T0[1] = t0.y; T0[2] = t0.z; T0[3] = t0.w;
        T1[0] = t1.x; T1[1] = t1.y; T1[2] = t1.z; T1[3] = t1.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < cnt) {
            T0[q] = a.T0[i0 + q];
            T1[q] = a.T1[i0 + q];
          }
      }
    }
    bool run[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) run[q] = q < cnt;
    NoCount nc;
    float xeq[4];
    point_step4(a.m, T0, T1, a.dt, run, xs, xm, ax, nc, xeq, false);
    if (cnt > 0) {
      Vec4<float>::store(a.xas + i0, xs);
      Vec4<float>::store(a.xam + i0, xm);
      Vec4<float>::store(a.aux + i0, ax);
      bool ok = true;
#pragma unroll
      for (int q = 0; q < 4; ++q) ok = ok && finite_pair(xs[q], xm[q]);
      if (!ok) atomicOr(a.err, DEVERR_NONFINITE);
    }
    return;
  }
  unsigned fp_it = 0, fp_unconv = 0;
  if (i0 < a.n) {
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
    for (int q = 0; q < 4; ++q) {
      if (q >= cnt) continue;
      if constexpr (IMPL)
        point_step_implicit<AT, FT>(a.m, AT(T0[q]), AT(T1[q]), a.dt, a.n_sub, xs[q], xm[q], ax[q],
                                    fp_it, fp_unconv);
      else
        point_step<AT, FT>(a.m, AT(T0[q]), AT(T1[q]), a.dt, xs[q], xm[q], ax[q]);
    }
    Vec4<FT>::store(a.xas + i0, xs);
    Vec4<FT>::store(a.xam + i0, xm);
    Vec4<float>::store(a.aux + i0, ax);
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 4; ++q) ok = ok && finite_pair(xs[q], xm[q]);
    if (!ok) atomicOr(a.err, DEVERR_NONFINITE);
  }
  if constexpr (IMPL) {
    unsigned long long it = fp_it, un = fp_unconv;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      it += __shfl_xor_sync(0xffffffffu, it, o);
      un += __shfl_xor_sync(0xffffffffu, un, o);
    }
    if ((threadIdx.x & 31) == 0 && a.ops && it) {
      atomicAdd(&a.ops->fp_iterations, it);
      if (un) atomicAdd(&a.ops->fp_unconverged, un);
    }
  }
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

template <typename AT, typename FT>
__global__ void k_fractions(const ModelConstT<AT> m, const SpecDev* specs,
                            const int32_t* tile_spec, int64_t n_pad, const FT* dxas,
                            const FT* dxam, const float* T, const SrcLevelT<AT>* levels,
                            const SrcEntryT<AT>* entries, int32_t slots, double* xbeta,
                            double* xliq, double* T_out) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= n_pad) return;
  int s;
  int64_t nat;
  if (!padded_to_natural(specs, tile_spec, g, s, nat)) return;
  AT Tp;
  if (T) {
    Tp = AT(T[nat]);
  } else {
    const SpecDev& sp = specs[s];
    AT x, y, z;
    point_coords<AT>(sp, g - sp.pad_off, x, y, z);
    Tp = temp1<AT>(levels[s], entries + int64_t(s) * slots, x, y, z);
  }
  const double gl = double(liquid_fraction<AT>(m, Tp));
  if (xbeta) xbeta[nat] = (1.0 - gl) - double(dxas[g]) - double(dxam[g]);
  if (xliq) xliq[nat] = gl;
  if (T_out) T_out[nat] = double(Tp);
}

// The correction g of eq:explicit_correction on n independent points (FP64),
// at the temperatures T[i][0], ..., T[i][n_T - 1] in turn.
__global__ void k_correct(const ModelConstT<double> m, int64_t n, int n_T, const double* T,
                          double* xas, double* xam) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = xas[i], b = xam[i];
  for (int l = 0; l < n_T; ++l) correct<double, double>(m, T[i * n_T + l], a, b);
  xas[i] = a;
  xam[i] = b;
}

// Verification reductions over natural-order fraction arrays a (na points)
// and b (nb points), 4 arrays each (X_as, X_am, X_beta, X_liq):
// out[0] = max over i < n of max_k |a_k[j] - b_k[i]| (j = idx[i], or i),
// out[1] = max over a's points of |sum_k a_k - 1|, out[2] the same for b.
// Non-negative doubles order like their bit patterns, so the maxima are
// atomicMax on the bits; NaN is reported as +inf.
__device__ __forceinline__ double nan_to_inf(double v) { return v == v ? v : INFINITY; }

__global__ void k_verify(const double* a, int64_t na, const double* b, int64_t nb, int64_t n,
                         const int64_t* idx, unsigned long long* out) {
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  const int64_t top = max(max(na, nb), n);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < top;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (i < n) {
      const int64_t j = idx ? idx[i] : i;
      double d = 0.0;
      for (int k = 0; k < 4; ++k) d = fmax(d, nan_to_inf(fabs(a[k * na + j] - b[k * nb + i])));
      m0 = fmax(m0, d);
    }
    if (i < na) m1 = fmax(m1, nan_to_inf(fabs(a[i] + a[na + i] + a[2 * na + i] + a[3 * na + i] - 1.0)));
    if (i < nb) m2 = fmax(m2, nan_to_inf(fabs(b[i] + b[nb + i] + b[2 * nb + i] + b[3 * nb + i] - 1.0)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out + 0, (unsigned long long)__double_as_longlong(m0));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(m1));
    atomicMax(out + 2, (unsigned long long)__double_as_longlong(m2));
  }
}

inline unsigned blocks_for(int64_t n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

}  // namespace

// The Crank-Nicolson variants exist for (float, float) and (double, double).
template <typename AT, typename FT>
constexpr bool kHasImplicit =
    (std::is_same<AT, float>::value && std::is_same<FT, float>::value) ||
    (std::is_same<AT, double>::value && std::is_same<FT, double>::value);

namespace {

// The launches of the hot kernels, internal to this translation unit (the
// FMA-transcendental variant compiles the same file into other kernels).
template <typename AT, typename FT>
cudaError_t track_launch(const TrackArgs<AT, FT>& a, int block_threads, int grid_blocks,
                         cudaStream_t stream, bool implicit) {
  if (a.n_tiles <= 0 || grid_blocks <= 0) return cudaSuccess;
  const unsigned g = unsigned(grid_blocks);
  if constexpr (std::is_same<AT, float>::value) {
    if (a.ff) {  // far field: the weights in shared memory
      const size_t ffb = FF_FLOATS * sizeof(float);
      if (!implicit) {
        // tiles across two grid rows take the far field in their own
        // instantiation, so that layouts without them (rows of a multiple of
        // TILE points) run the compact one
        if (a.two_rows && std::is_same<FT, float>::value) {
          if (a.count_sfu)
            k_track<AT, FT, false, true, true, true><<<g, block_threads, ffb, stream>>>(a);
          else
            k_track<AT, FT, false, true, false, true><<<g, block_threads, ffb, stream>>>(a);
        } else if (a.count_sfu) {
          k_track<AT, FT, false, true, true><<<g, block_threads, ffb, stream>>>(a);
        } else {
          k_track<AT, FT, false, true><<<g, block_threads, ffb, stream>>>(a);
        }
      } else if constexpr (kHasImplicit<AT, FT>) {
        k_track<AT, FT, true, true><<<g, block_threads, ffb, stream>>>(a);
      } else {
        return cudaErrorNotSupported;
      }
      return cudaGetLastError();
    }
  }
  if (implicit) {
    if constexpr (kHasImplicit<AT, FT>)
      k_track<AT, FT, true><<<g, block_threads, 0, stream>>>(a);
    else
      return cudaErrorNotSupported;
  } else if (a.count_sfu) {
    k_track<AT, FT, false, false, true><<<g, block_threads, 0, stream>>>(a);
  } else {
    k_track<AT, FT, false><<<g, block_threads, 0, stream>>>(a);
  }
  return cudaGetLastError();
}

template <typename AT, typename FT>
cudaError_t step_launch(const StepArgs<AT, FT>& a, int block_threads, cudaStream_t stream,
                        bool implicit) {
  if (a.n <= 0) return cudaSuccess;
  const int vec = ((reinterpret_cast<uintptr_t>(a.T0) | reinterpret_cast<uintptr_t>(a.T1)) & 15) == 0;
  const unsigned blocks = blocks_for((a.n + 3) / 4, block_threads);
  if (implicit) {
    if constexpr (kHasImplicit<AT, FT>)
      k_step_ext<AT, FT, true><<<blocks, block_threads, 0, stream>>>(a, vec);
    else
      return cudaErrorNotSupported;
  } else {
    k_step_ext<AT, FT, false><<<blocks, block_threads, 0, stream>>>(a, vec);
  }
  return cudaGetLastError();
}

}  // namespace

#ifdef MS_FMA_TRANSCENDENTALS
// ----------------------------------- FMA-pipe exp2 / log2 (this file compiled again)
cudaError_t launch_track_fma(const TrackArgs<float, float>& a, int block_threads,
                             int grid_blocks, cudaStream_t stream, bool implicit) {
  return track_launch<float, float>(a, block_threads, grid_blocks, stream, implicit);
}
cudaError_t launch_step_ext_fma(const StepArgs<float, float>& a, int block_threads,
                                cudaStream_t stream, bool implicit) {
  return step_launch<float, float>(a, block_threads, stream, implicit);
}
#else
// ------------------------------------------------------------- launchers
template <typename AT>
cudaError_t launch_src_table(const TableArgs& a, WorkCounters* work, cudaStream_t stream) {
  const int64_t n = int64_t(a.n_specs) * a.n_levels * 32 + (a.win ? a.n_tracks : 0);
  if (n <= 0) return cudaSuccess;
  k_src_table<AT><<<blocks_for(n, 128), 128, 0, stream>>>(a, work);
  return cudaGetLastError();
}

cudaError_t launch_fill_f32(float* p, int64_t n, float v, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_fill_f32<<<blocks_for(n, 256), 256, 0, stream>>>(p, n, v);
  return cudaGetLastError();
}

cudaError_t launch_verify(const double* a, int64_t na, const double* b, int64_t nb, int64_t n,
                          const int64_t* idx, double* out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, 3 * sizeof(double), stream);
  if (e != cudaSuccess) return e;
  const int64_t top = std::max(std::max(na, nb), n);
  const unsigned blocks = unsigned(std::min<int64_t>((top + 255) / 256, 4096));
  k_verify<<<blocks > 0 ? blocks : 1, 256, 0, stream>>>(
      a, na, b, nb, n, idx, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}

cudaError_t launch_correct(const ModelConstT<double>& m, int64_t n, int n_T, const double* T,
                           double* xas, double* xam, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_correct<<<blocks_for(n, 256), 256, 0, stream>>>(m, n, n_T, T, xas, xam);
  return cudaGetLastError();
}

template <typename AT, typename FT>
int track_blocks_per_sm(int block_threads, bool implicit) {
  int nb = 0;
  cudaError_t e = cudaSuccess;
  if constexpr (kHasImplicit<AT, FT>) {
    if (implicit)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_track<AT, FT, true>, block_threads, 0);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_track<AT, FT, false>, block_threads, 0);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_track<AT, FT, false>, block_threads, 0);
  }
  if (e != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

template <typename AT, typename FT>
cudaError_t launch_track(const TrackArgs<AT, FT>& a, int block_threads, int grid_blocks,
                         cudaStream_t stream, bool implicit) {
  return track_launch<AT, FT>(a, block_threads, grid_blocks, stream, implicit);
}

int track_dense_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_track_dense<true>, DENSE_THREADS,
                                                    FF_FLOATS * sizeof(float)) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

int track_dense_grid(int64_t n_tiles, int blocks_per_sm, int sm_count) {
  const int64_t chunks = (n_tiles + DENSE_CHUNK - 1) / DENSE_CHUNK;
  const int64_t need = (chunks + DENSE_THREADS / 32 - 1) / (DENSE_THREADS / 32);
  return int(std::max<int64_t>(1, std::min<int64_t>(int64_t(blocks_per_sm) * sm_count, need)));
}

cudaError_t launch_track_dense(const TrackArgs<float, float>& a, int grid_blocks,
                               cudaStream_t stream) {
  if (a.n_tiles <= 0 || grid_blocks <= 0) return cudaSuccess;
  if (a.n_levels != 2 || a.tile_list) return cudaErrorInvalidValue;
  const unsigned g = unsigned(grid_blocks);
  if (a.ff) {
    if (a.two_rows)  // tiles across two grid rows: their own instantiation (as in k_track)
      k_track_dense<true, true><<<g, DENSE_THREADS, FF_FLOATS * sizeof(float), stream>>>(a);
    else
      k_track_dense<true><<<g, DENSE_THREADS, FF_FLOATS * sizeof(float), stream>>>(a);
  } else {
    k_track_dense<false><<<g, DENSE_THREADS, 0, stream>>>(a);
  }
  return cudaGetLastError();
}

template <typename AT, typename FT>
cudaError_t launch_step_ext(const StepArgs<AT, FT>& a, int block_threads, cudaStream_t stream,
                            bool implicit) {
  return step_launch<AT, FT>(a, block_threads, stream, implicit);
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

template <typename AT, typename FT>
cudaError_t launch_fractions(const ModelConstT<AT>& m, const SpecDev* specs,
                             const int32_t* tile_spec, int64_t n_tiles, const FT* dxas,
                             const FT* dxam, const float* T, const SrcLevelT<AT>* levels,
                             const SrcEntryT<AT>* entries, int32_t slots, double* xbeta,
                             double* xliq, double* T_out, cudaStream_t stream) {
  const int64_t n_pad = n_tiles * TILE;
  k_fractions<AT, FT><<<blocks_for(n_pad, 256), 256, 0, stream>>>(
      m, specs, tile_spec, n_pad, dxas, dxam, T, levels, entries, slots, xbeta, xliq, T_out);
  return cudaGetLastError();
}

#define MS_INSTANTIATE_FT(FT)                                                                     \
  template cudaError_t launch_set_state<FT>(const SpecDev*, const int32_t*, int64_t,             \
                                            const double*, const double*, const double*, FT*,    \
                                            FT*, float*, cudaStream_t, double, double);          \
  template cudaError_t launch_get_state<FT>(const SpecDev*, const int32_t*, int64_t, const FT*,  \
                                            const FT*, const float*, double*, double*, double*,  \
                                            cudaStream_t);

#define MS_INSTANTIATE(AT, FT)                                                                    \
  template int track_blocks_per_sm<AT, FT>(int, bool);                                           \
  template cudaError_t launch_track<AT, FT>(const TrackArgs<AT, FT>&, int, int, cudaStream_t,    \
                                            bool);                                               \
  template cudaError_t launch_step_ext<AT, FT>(const StepArgs<AT, FT>&, int, cudaStream_t, bool); \
  template cudaError_t launch_fractions<AT, FT>(                                                 \
      const ModelConstT<AT>&, const SpecDev*, const int32_t*, int64_t, const FT*, const FT*,     \
      const float*, const SrcLevelT<AT>*, const SrcEntryT<AT>*, int32_t, double*, double*,       \
      double*, cudaStream_t);

template cudaError_t launch_src_table<float>(const TableArgs&, WorkCounters*, cudaStream_t);
template cudaError_t launch_src_table<double>(const TableArgs&, WorkCounters*, cudaStream_t);
MS_INSTANTIATE_FT(float)
MS_INSTANTIATE_FT(double)
MS_INSTANTIATE_FT(KF)
MS_INSTANTIATE(float, float)
MS_INSTANTIATE(float, double)
MS_INSTANTIATE(float, KF)
MS_INSTANTIATE(double, double)
#endif  // MS_FMA_TRANSCENDENTALS

}  // namespace ms
