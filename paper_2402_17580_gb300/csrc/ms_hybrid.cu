// Hybrid hot kernel: ms_run_track with an attached surrogate.
//
// The same persistent tile loop as k_track (128-point tiles, 4 points per
// lane, temperatures from the source table), but the launch's steps are taken
// in windows of K = 8 r steps, r being the surrogate's temperature stride.
// Per window:
//   - the temperatures of the window's levels r, 2 r, ..., 8 r (its samples)
//     go to shared memory;
//   - band test per point on the window start and the samples: every sample
//     stays 40 K away from each temperature where the model switches branch
//     (T_am,start, T_as,end, T_as,start, T_as,start + T_reg) and below
//     T_s - 40 K, consecutive samples differ by at most 40 K, with r > 1 no
//     three consecutive samples point to a minimum below T_am,start or a
//     maximum above T_as,end near them (the path's extreme would lie between
//     samples, and the correction g depends on it there), no App. A
//     initiation is running, and the point is below the surface from the
//     window's first level on;
//   - passing points take X = g(T_8r, G(X_start) + y / 1e6) with
//     G = g(T_8r, .) o ... o g(T_r, .): the correction g of Sec. 2.2 at the
//     samples supplies the instantaneous part (clamping, the X_alpha <= 0.9
//     bound, the alpha_s cap, martensite dissolution and formation; G is
//     evaluated as g at one sample, which the band test makes equal) and the
//     MLP (12 -> 64 -> 64 -> 3, BF16 on the tensor cores, one m16n8k16 row
//     tile per 16 points, tiles with no MLP point skipped) the rest;
//   - a warp with a point that needs the explicit steps takes them for all
//     its non-idle points;
//   - the others take the K explicit steps of Sec. 3
//     (eq:explicit_integration + g) as k_track does: the four points of a
//     lane in lockstep, a warp vote skipping the levels where every running
//     point is cold and saturated (reading A9); levels between samples get
//     their temperatures only in warps that have such points;
//   - a fraction of the 128-point tiles' windows, chosen by a counter-based
//     hash of (tile, level), has its MLP points also run with the explicit
//     steps (the judge); the largest difference is kept in the counters, and
//     the MLP result stays unless the tile-window's largest difference passes
//     the judge's tolerance, which sends it back to the explicit steps'
//     result (ms_set_judge_tol).  Judging whole tiles keeps the explicit steps in
//     the few warps that judge (a per-point draw would put a judged point in
//     nearly every warp, and the warp would take the explicit steps for it).
// Points that are cold and saturated at the window start and every sample
// (the skip test of reading A9, at the samples) are left unchanged, and so
// are points on the alpha_s plateau's fixed point (X_as = 0.9, X_am = 0)
// whose samples stay below T_as,end, where the explicit steps are the
// identity.  With r > 1 both tests, like the band test, stand for the levels
// between samples; with r = 1 they are the per-level tests of k_track.  A
// launch's last window, when shorter than K, takes the explicit steps.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ms_internal.h"
#include "ms_mlp.cuh"
#include "ms_tile.cuh"

namespace ms {

namespace {

constexpr int HYB_WARPS = HYBRID_THREADS / 32;
constexpr float BAND_HALF_WIDTH = 40.0f;

// Point q of lane l is row l + 32 q of the warp's tile in all three arrays,
// so a warp's per-point accesses for one q are consecutive (no bank
// conflicts); the ODE path reads T the same way.
struct HybWarp {
  float T[MLP_WINDOW][TILE];                 // the window's new temperatures
  __nv_bfloat16 X[TILE][MLP_X_LD];           // MLP inputs (padded rows)
  float Y[MLP_Y_COLS][TILE];                 // MLP outputs, column-major
};
constexpr size_t MLP_SMEM = (sizeof(MlpDev) + 127) / 128 * 128;
constexpr size_t HYB_SMEM = MLP_SMEM + HYB_WARPS * sizeof(HybWarp);
static_assert(sizeof(MlpDev) % 16 == 0 && sizeof(HybWarp) % 128 == 0, "16-byte copies, aligned warp areas");
static_assert(2 * (HYB_SMEM + 1024) <= 228 * 1024, "two CTAs per SM");

__device__ __forceinline__ bool near(float T, float c) { return fabsf(T - c) < BAND_HALF_WIDTH; }

__device__ __forceinline__ bool in_band(const ModelConstT<float>& m, float T) {
  return !(T <= m.T_s - BAND_HALF_WIDTH) || near(T, m.T_am_start) || near(T, m.T_as_end) ||
         near(T, m.T_as_start) || near(T, m.T_cap0);
}

// Whether the parabola through three temperature samples a, b, c (equally
// spaced) has its vertex within two spacings of b, a minimum below T_am,start
// or a maximum above T_as,end: there the correction g depends on the path's
// extreme, which can lie between the samples (an abrupt turn puts it between
// them while the parabola's lies up to a spacing past them).
__device__ __forceinline__ bool extreme_between(const ModelConstT<float>& m, float a, float b,
                                                float c) {
  const float k = a - 2.0f * b + c;
  const float s = c - a;
  if (k == 0.0f || !(fabsf(s) <= 4.0f * fabsf(k))) return false;
  // vertex value v = b - s^2 / (8 k): v < T_am,start for k > 0 and
  // v > T_as,end for k < 0 both read 8 k (b - threshold) < s^2
  return 8.0f * k * (b - (k > 0.0f ? m.T_am_start : m.T_as_end)) < s * s;
}

// SplitMix64 output function (Steele, Lea, Flood 2014) of (tile, level).
__device__ __forceinline__ uint32_t judge_hash(uint64_t tile, uint64_t level) {
  uint64_t z = tile * 0x9E3779B97F4A7C15ull + level * 0xD1B54A32D192ED03ull + 0x2402175800ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return uint32_t((z ^ (z >> 31)) >> 32);
}

template <typename FT>
__device__ __forceinline__ float to_f(FT v) { return float(v); }
template <>
__device__ __forceinline__ float to_f<KF>(KF v) { return v.hi + v.lo; }

struct HybCount {
  unsigned long long surr = 0, ode = 0, judged = 0;
  unsigned long long rejected = 0;  // lane 0's count of the warp's sent-back tile-windows
  float err = 0.0f;
};

// One explicit step (T0 -> T1) of the lane's four points with run[q]: the
// FP32 state in lockstep (point_step4); the compensated state by the FP32
// step's increments (point_step4's INC mode), or point by point when a lane
// of the warp has an App. A initiation.  Every lane of the warp calls it.
// Returns X_alpha^eq's carry to the next level (point_step4's result).
template <typename FT>
__device__ __forceinline__ bool explicit_step4(const ModelConstT<float>& m, const float* T0,
                                               const float* T1, float dt, const bool* run,
                                               FT* xs, FT* xm, float* ax, float* xeq,
                                               bool have_xeq) {
  NoCount oc;
  if constexpr (std::is_same<FT, float>::value) {
    return point_step4(m, T0, T1, dt, run, xs, xm, ax, oc, xeq, have_xeq);
  } else {
    float fs[4], fm[4], du_s[4], du_m[4];
    unsigned mod = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      fs[q] = float(xs[q]);
      fm[q] = float(xm[q]);
    }
    const bool ok = point_step4<NoCount, true>(m, T0, T1, dt, run, fs, fm, ax, oc, xeq, have_xeq,
                                               du_s, du_m, &mod);
    if (ok) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (run[q]) {
          xs[q] = (mod >> (2 * q)) & 1u ? FT(fs[q]) : xs[q] + FT(du_s[q]);
          xm[q] = (mod >> (2 * q)) & 2u ? FT(fm[q]) : xm[q] + FT(du_m[q]);
        }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (run[q]) point_step<float, FT>(m, T0[q], T1[q], dt, xs[q], xm[q], ax[q]);
    }
    return ok;
  }
}

template <typename FT, int ACT, bool TWO>
__device__ __forceinline__ void hybrid_tile(const TrackArgs<float, FT>& a, const MlpDev& W,
                                            HybWarp& sm, int tile, int lane, float fdt,
                                            HybCount& cnt) {
  const unsigned full = 0xffffffffu;
  const int s = a.tile_spec[tile];
  const SpecDev& sp = a.specs[s];
  const int64_t local0 = int64_t(tile - sp.tile0) * TILE + lane * 4;
  const int64_t g0 = sp.pad_off + local0;

  float px[4], py[4], pz[4];
  bool valid[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) valid[q] = local0 + q < sp.n;
  int64_t col;
  point_coords4<float>(sp, local0, valid, px, py, pz, col);
  const bool row = tile_in_one_row(sp, tile);

  FT xs[4], xm[4];
  float ax[4];
  Vec4<FT>::load(a.xas + g0, xs);
  Vec4<FT>::load(a.xam + g0, xm);
  Vec4<float>::load(a.aux + g0, ax);

  const SrcLevelT<float>* lv = a.levels + int64_t(s) * a.n_levels;
  const SrcEntryT<float>* en = a.entries + int64_t(s) * a.n_levels * a.slots;
  const float z_tol = sp.z_tol;
  const bool skipping = a.m.T_thr > 0.0f;
  const int n_steps = a.n_levels - 1;
  const int r = a.mlp_stride;
  const int KW = MLP_WINDOW * r;
  // far field (as in k_track): the tile's x-range, first to 128th point
  const int64_t col0 = __shfl_sync(full, col, 0);
  const float x_first = grid_coord<float>(float(sp.ox), float(int32_t(col0)), float(sp.dx));
  const float x_span = __fmul_rn(float(TILE - 1), float(sp.dx));
  const float ff_dist = fmaxf(a.ff_dist, FF_RANGE_GUARD * fabsf(x_span));
  const bool far = a.ff != nullptr && row;
  const float py_row = __shfl_sync(full, py[0], 0);  // lane 0's first point is always valid
  const float pz_row = __shfl_sync(full, pz[0], 0);
  // a tile across two rows (as in k_track): the far field over both rows' ranges
  const int64_t span = min(sp.n - 1 - int64_t(tile - sp.tile0) * TILE, int64_t(TILE - 1));
  const bool far2 = TWO && a.ff != nullptr && !row && !sp.idx && col0 + span < 2 * int64_t(sp.nx);
  int m_two = 0;
  float x_first_b = 0.f, y_b = 0.f, z_b = 0.f;
  if (far2) {
    m_two = int(sp.nx - col0);
    x_first_b = grid_coord<float>(float(sp.ox), float(-m_two), float(sp.dx));
    second_row_yz(py, pz, m_two, y_b, z_b);
  }
  // the temperatures of 4 points at level lvl, far field where it applies
  auto temps = [&](int lvl, float* T) {
    const SrcLevelT<float> L = lv[lvl];
    if (far && L.axis == LEVEL_AXIS) {
      int nn, nf;
      temps4_far(L, en + int64_t(lvl) * a.slots, px, py_row, pz_row, x_first, x_span, ff_dist,
                 lane, T, nn, nf, a.ff);
    } else if (TWO && far2 && L.axis == LEVEL_AXIS) {
      int nn, nf;
      temps4_far2(L, en + int64_t(lvl) * a.slots, px, py_row, pz_row, y_b, z_b, m_two, x_first,
                  x_first_b, x_span, ff_dist, lane, T, nn, nf, a.ff);
    } else {
      temps4<float>(L, en + int64_t(lvl) * a.slots, px, py, pz, row, T);
    }
  };

  float T0[4];
  temps(0, T0);
  for (int w0 = 0; w0 < n_steps; w0 += KW) {
    const int K = min(KW, n_steps - w0);
    const bool whole = K == KW;
    bool use_mlp[4], use_ode[4], judged[4];
    bool lane_mlp = false, lane_exp = false;
    const float zl_first = lv[w0 + 1].z_surf + z_tol, zl_last = lv[w0 + K].z_surf + z_tol;
    if (whole) {
      // the samples, and the tests on them (the window start included)
      bool band[4], noop[4], cool[4];
      float Tp[4], Tpp[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        band[q] = in_band(a.m, T0[q]);
        noop[q] = skipping;
        cool[q] = T0[q] < a.m.T_as_end;
        Tp[q] = T0[q];
        Tpp[q] = T0[q];
      }
      for (int j = 0; j < MLP_WINDOW; ++j) {
        float T1[4];
        temps(w0 + r * (j + 1), T1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sm.T[j][lane + 32 * q] = T1[q];
          band[q] = band[q] || in_band(a.m, T1[q]) || !(fabsf(T1[q] - Tp[q]) <= BAND_HALF_WIDTH);
          if (r > 1 && j > 0) band[q] = band[q] || extreme_between(a.m, Tpp[q], Tp[q], T1[q]);
          Tpp[q] = Tp[q];
          cool[q] = cool[q] && T1[q] < a.m.T_as_end;
          noop[q] = noop[q] && step_is_noop<float, FT>(a.m, Tp[q], T1[q], xs[q], xm[q], ax[q]);
          Tp[q] = T1[q];
        }
      }
      const bool judge_tile =
          uint64_t(judge_hash(uint64_t(tile), uint64_t(a.level0 + w0))) < a.judge_thresh;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // below the surface from the window's first level on (surfaces only rise)
        const bool all_act = valid[q] && pz[q] <= zl_first;
        const bool any_act = valid[q] && pz[q] <= zl_last;
        // the alpha_s plateau's fixed point (X_as = 0.9, X_am = 0, no
        // initiation) below T_as,end: the explicit steps are the identity
        const bool fixed = xs[q] == FT(0.9) && xm[q] == FT(0) && ax[q] == 0.0f && cool[q];
        const bool idle = !any_act || noop[q] || fixed;
        use_mlp[q] = !idle && all_act && !band[q] && ax[q] == 0.0f;
        judged[q] = use_mlp[q] && judge_tile;
        use_ode[q] = !idle && !use_mlp[q];
      }
      // a warp that takes the explicit steps for some point takes them for
      // all its non-idle points: its pass costs the same, and the MLP and the
      // corrections are saved (the judge skips such windows)
      bool lane_ode = false;
#pragma unroll
      for (int q = 0; q < 4; ++q) lane_ode = lane_ode || use_ode[q];
      if (__any_sync(full, lane_ode)) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (use_mlp[q]) {
            use_mlp[q] = judged[q] = false;
            use_ode[q] = true;
          }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        use_mlp[q] = judged[q] = false;
        use_ode[q] = valid[q] && pz[q] <= zl_last;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      lane_mlp = lane_mlp || use_mlp[q];
      lane_exp = lane_exp || use_ode[q] || judged[q];
      cnt.surr += use_mlp[q];
      cnt.ode += use_ode[q];
      cnt.judged += judged[q];
    }

    FT rs[4], rm[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      rs[q] = xs[q];
      rm[q] = xm[q];
    }
    if (__ballot_sync(full, lane_mlp)) {
      // row tile mt holds rows 16 mt .. 16 mt + 15: point q = mt / 2 of lanes
      // 16 (mt % 2) .. 16 (mt % 2) + 15
      uint32_t mt_mask = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned bq = __ballot_sync(full, use_mlp[q]);
        if (bq & 0x0000ffffu) mt_mask |= 1u << (2 * q);
        if (bq & 0xffff0000u) mt_mask |= 2u << (2 * q);
      }
      // inputs: fractions at the window start, the 8 samples, log10(dt) + 5
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = lane + 32 * q;
        float f[MLP_IN_PAD];
#pragma unroll
        for (int k = 0; k < MLP_IN_PAD; ++k) f[k] = 0.0f;
        if (use_mlp[q]) {
          const float fs = to_f(xs[q]), fm = to_f(xm[q]);
          f[0] = fs;
          f[1] = fm;
          f[2] = 1.0f - fs - fm;
#pragma unroll
          for (int l = 0; l < MLP_WINDOW; ++l) f[3 + l] = (sm.T[l][row] - MLP_T_SHIFT) * MLP_T_SCALE;
          f[11] = fdt;
        }
        uint4 v0, v1;
        v0.x = pack_bf16(f[0], f[1]); v0.y = pack_bf16(f[2], f[3]);
        v0.z = pack_bf16(f[4], f[5]); v0.w = pack_bf16(f[6], f[7]);
        v1.x = pack_bf16(f[8], f[9]); v1.y = pack_bf16(f[10], f[11]);
        v1.z = 0u; v1.w = 0u;
        *reinterpret_cast<uint4*>(&sm.X[row][0]) = v0;
        *reinterpret_cast<uint4*>(&sm.X[row][8]) = v1;
      }
      __syncwarp();
      mlp_forward_warp<ACT>(W, &sm.X[0][0], &sm.Y[0][0], lane, mt_mask);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!use_mlp[q]) continue;
        const int row = lane + 32 * q;
        FT nas = xs[q], nam = xm[q];
        // the instantaneous part at the samples, G: the band test leaves
        // every sample of an MLP window in one of the ranges between the
        // switching temperatures, on one side of T_as,end, where g at the
        // samples in turn equals g at one of them: below T_as,end the
        // coldest (martensite formation keeps the largest target; the
        // literal reading A3 keeps the last), above it the hottest (the
        // lowest alpha equilibrium and alpha_s cap)
        float tmin = sm.T[0][row], tmax = tmin;
#pragma unroll
        for (int l = 1; l < MLP_WINDOW; ++l) {
          tmin = fminf(tmin, sm.T[l][row]);
          tmax = fmaxf(tmax, sm.T[l][row]);
        }
        const float tg = !(tmax < a.m.T_as_end)
                             ? tmax
                             : (a.m.martensite_literal ? sm.T[MLP_WINDOW - 1][row] : tmin);
        correct<float, FT>(a.m, tg, nas, nam);
        nas = nas + FT(sm.Y[0][row] * (1.0f / MLP_OUT_SCALE));
        nam = nam + FT(sm.Y[1][row] * (1.0f / MLP_OUT_SCALE));
        correct<float, FT>(a.m, sm.T[MLP_WINDOW - 1][row], nas, nam);
        rs[q] = nas;
        rm[q] = nam;
      }
    }

    // explicit steps: fallback points and judged MLP windows
    if (__any_sync(full, lane_exp)) {
      FT es[4], em[4];
      float ea[4], Tp[4], xeq[4];
      bool have_xeq = false;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        es[q] = xs[q];
        em[q] = xm[q];
        ea[q] = ax[q];
        Tp[q] = T0[q];
      }
      int j = 0, to_sample = r;   // the next sample and the levels to it
      for (int l = 1; l <= K; ++l) {
        float T1[4];
        if (whole && --to_sample == 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) T1[q] = sm.T[j][lane + 32 * q];
          ++j;
          to_sample = r;
        } else {
          temps(w0 + l, T1);
        }
        const float zlim = lv[w0 + l].z_surf + z_tol;
        bool run[4], nop = true;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          run[q] = (use_ode[q] || judged[q]) && valid[q] && pz[q] <= zlim;
          if (skipping)
            nop = nop && (!run[q] || step_is_noop<float, FT>(a.m, Tp[q], T1[q], es[q], em[q], ea[q]));
        }
        if (skipping && __all_sync(full, nop))
          have_xeq = false;
        else
          have_xeq = explicit_step4<FT>(a.m, Tp, T1, a.dt, run, es, em, ea, xeq, have_xeq);
#pragma unroll
        for (int q = 0; q < 4; ++q) Tp[q] = T1[q];
      }
      float werr = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (use_ode[q]) {
          xs[q] = es[q];
          xm[q] = em[q];
          ax[q] = ea[q];
        }
        if (judged[q]) {
          const float e = fmaxf(fabsf(to_f(es[q]) - to_f(rs[q])), fabsf(to_f(em[q]) - to_f(rm[q])));
          cnt.err = fmaxf(cnt.err, e);
          werr = fmaxf(werr, e);
        }
        T0[q] = Tp[q];
      }
      // the judge sends the tile-window back to the explicit steps when the
      // network's largest difference on it passes judge_tol (a NaN too)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float w2 = __shfl_xor_sync(full, werr, o);
        werr = (w2 > werr || w2 != w2) ? w2 : werr;
      }
      if (!(werr <= a.judge_tol)) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (judged[q]) {
            rs[q] = es[q];
            rm[q] = em[q];
            ax[q] = ea[q];
          }
        if (lane == 0) ++cnt.rejected;
      }
    } else if (whole) {
#pragma unroll
      for (int q = 0; q < 4; ++q) T0[q] = sm.T[MLP_WINDOW - 1][lane + 32 * q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (use_mlp[q]) {
        xs[q] = rs[q];
        xm[q] = rm[q];
      }
    }
    __syncwarp();  // the next window overwrites sm.T and sm.X
  }

  Vec4<FT>::store(a.xas + g0, xs);
  Vec4<FT>::store(a.xam + g0, xm);
  Vec4<float>::store(a.aux + g0, ax);
  bool ok = true;
  float ts = -INFINITY;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ok = ok && finite_pair(xs[q], xm[q]);
    if (valid[q]) ts = fmaxf(ts, point_tsat<float, FT>(a.m, xs[q], xm[q], ax[q]));
  }
  if (!ok) atomicOr(a.err, DEVERR_NONFINITE);
  if (a.tile_tsat) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ts = fmaxf(ts, __shfl_xor_sync(full, ts, o));
    if (lane == 0) a.tile_tsat[tile] = ts + 0.5f;
  }
}
template <typename FT, int ACT, bool TWO = false>
__global__ void __launch_bounds__(HYBRID_THREADS, 2) k_track_hybrid(const TrackArgs<float, FT> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  MlpDev& W = *reinterpret_cast<MlpDev*>(smem);
  {
    const uint4* src = static_cast<const uint4*>(a.mlp);
    uint4* dst = reinterpret_cast<uint4*>(smem);
    for (int i = threadIdx.x; i < int(sizeof(MlpDev) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  HybWarp& sm = reinterpret_cast<HybWarp*>(smem + MLP_SMEM)[warp];
  const float fdt = log10f(a.dt) + MLP_DT_SHIFT;
  const int n_work = a.tile_list ? a.work->n_active : a.n_tiles;
  unsigned long long done = 0;
  HybCount cnt;
  int nb[COST_BUCKETS];
#pragma unroll
  for (int b = 0; b < COST_BUCKETS; ++b) nb[b] = a.tile_list ? a.work->n_bucket[b] : 0;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(&a.work->next, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= n_work) break;
    hybrid_tile<FT, ACT, TWO>(a, W, sm, a.tile_list ? list_tile(a.tile_list, a.n_tiles, nb, w) : w, lane,
                    fdt, cnt);
    ++done;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cnt.surr += __shfl_xor_sync(0xffffffffu, cnt.surr, o);
    cnt.ode += __shfl_xor_sync(0xffffffffu, cnt.ode, o);
    cnt.judged += __shfl_xor_sync(0xffffffffu, cnt.judged, o);
    cnt.err = fmaxf(cnt.err, __shfl_xor_sync(0xffffffffu, cnt.err, o));
  }
  if (lane == 0) {
    if (done) atomicAdd(&a.work->tile_steps_active, done * (unsigned long long)(a.n_levels - 1));
    if (cnt.surr) atomicAdd(&a.hyb->surrogate_windows, cnt.surr);
    if (cnt.ode) atomicAdd(&a.hyb->ode_windows, cnt.ode);
    if (cnt.judged) atomicAdd(&a.hyb->judge_samples, cnt.judged);
    if (cnt.err > 0.0f) atomicMax(&a.hyb->judge_err_bits, __float_as_uint(cnt.err));
    if (cnt.rejected) atomicAdd(&a.hyb->judge_rejected, cnt.rejected);
  }
}

}  // namespace

template <typename FT>
int hybrid_blocks_per_sm(int activation) {
  auto k = activation == ACT_RELU ? k_track_hybrid<FT, ACT_RELU> : k_track_hybrid<FT, ACT_GELU>;
  auto k2 = activation == ACT_RELU ? k_track_hybrid<FT, ACT_RELU, true>
                                   : k_track_hybrid<FT, ACT_GELU, true>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(HYB_SMEM)) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(HYB_SMEM)) !=
          cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, HYBRID_THREADS, HYB_SMEM) != cudaSuccess)
    return 0;
  return nb;
}

template <typename FT>
cudaError_t launch_track_hybrid(const TrackArgs<float, FT>& a, int activation, int grid_blocks,
                                cudaStream_t stream) {
  if (a.n_tiles <= 0 || grid_blocks <= 0) return cudaSuccess;
  if (a.mlp_stride < 1 || a.mlp_stride > MLP_MAX_STRIDE) return cudaErrorInvalidValue;
  const unsigned g = unsigned(grid_blocks);
  // tiles across two grid rows take the far field in their own instantiation
  if (activation == ACT_RELU && a.two_rows)
    k_track_hybrid<FT, ACT_RELU, true><<<g, HYBRID_THREADS, HYB_SMEM, stream>>>(a);
  else if (activation == ACT_RELU)
    k_track_hybrid<FT, ACT_RELU><<<g, HYBRID_THREADS, HYB_SMEM, stream>>>(a);
  else if (a.two_rows)
    k_track_hybrid<FT, ACT_GELU, true><<<g, HYBRID_THREADS, HYB_SMEM, stream>>>(a);
  else
    k_track_hybrid<FT, ACT_GELU><<<g, HYBRID_THREADS, HYB_SMEM, stream>>>(a);
  return cudaGetLastError();
}

template int hybrid_blocks_per_sm<float>(int);
template int hybrid_blocks_per_sm<KF>(int);
template cudaError_t launch_track_hybrid<float>(const TrackArgs<float, float>&, int, int, cudaStream_t);
template cudaError_t launch_track_hybrid<KF>(const TrackArgs<float, KF>&, int, int, cudaStream_t);

}  // namespace ms
