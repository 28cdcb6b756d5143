// Active-set compaction (reading A9): per launch, the list of tiles that
// may get hot (a rigorous upper bound of their temperature over the launch's
// time window reaches T_thr) or whose martensite is not saturated.  A tile
// whose points all sit on the alpha_s plateau's fixed point (X_as = 0.9,
// X_am = 0: the room-temperature state no heat has touched) is hot only once
// the bound reaches T_as,end, below which its steps are the identity.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ms_internal.h"

namespace ms {

namespace {

constexpr double kE = 2.7182818284590452354;

inline unsigned blocks_for(int64_t n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

// ------------------------------------------------------------ active set
// Upper bound of the temperature of a tile over [t_a, t_b]: every started
// source of a layer current in the window contributes at most
// A P / (2 pi k) times the smaller of
//   exp(-v xi_min / alpha) / R_min   (R + xi >= 2 xi ahead of the path) and
//   max over R >= R_min of exp(-v rho_min^2 / (4 alpha R)) / R
//                                    (the wake: R + xi >= rho^2 / (2 R)),
// with R_min the distance between the tile's bounding box and the box of the
// source's path in the window, xi_min >= 0 the smallest along-track offset of
// a tile point ahead of the path and rho_min the distance between the tile's
// box and the source's line.  The interlayer scale is <= 1.  Subset
// specimens use the whole grid's box.  The path of every track in the window
// comes from the source-table launch (TrackWin, FP64).
__device__ bool tile_is_active(const ActiveArgs& a, int t) {
  const int s = a.tile_spec[t];
  const SpecDev& sp = a.specs[s];
  const float tsat = a.tile_tsat[t];
  if (!(tsat <= sp.T0)) return true;  // martensite not saturated at T0, or initiation running
  // every point on the alpha_s plateau's fixed point (tsat = -inf): the
  // steps are the identity while T < T_as,end, so only that bound matters
  const double T_hot = tsat == -INFINITY ? fmax(a.T_thr, a.T_as_end) : a.T_thr;
  int64_t ilo = 0, ihi = sp.nx - 1, jlo = 0, jhi = sp.ny - 1, k0 = 0, k1 = sp.nz - 1;
  if (!sp.idx) {
    const int64_t li0 = int64_t(t - sp.tile0) * TILE;
    const int64_t li1 = min(li0 + TILE - 1, sp.n - 1);
    const int64_t nxy = int64_t(sp.nx) * sp.ny;
    k0 = li0 / nxy;
    k1 = li1 / nxy;
    const int64_t j0 = (li0 - k0 * nxy) / sp.nx, j1 = (li1 - k1 * nxy) / sp.nx;
    const int64_t i0 = li0 - k0 * nxy - j0 * sp.nx, i1 = li1 - k1 * nxy - j1 * sp.nx;
    if (k0 == k1) {
      jlo = j0;
      jhi = j1;
      if (j0 == j1) {
        ilo = i0;
        ihi = i1;
      }
    }
  }
  const double xa = sp.ox + double(ilo) * sp.dx, xb = sp.ox + double(ihi) * sp.dx;
  const double ya = sp.oy + double(jlo) * sp.dy, yb = sp.oy + double(jhi) * sp.dy;
  const double za = sp.oz + double(k0 + sp.k_off) * sp.dz;
  const double zb = sp.oz + double(k1 + sp.k_off) * sp.dz;
  const double bx0 = fmin(xa, xb), bx1 = fmax(xa, xb), by0 = fmin(ya, yb), by1 = fmax(ya, yb);
  const float bz1 = float(fmax(za, zb));
  // Per source the geometry runs in FP32 on coordinates relative to the
  // tile's centre (|offsets| up to ~1 m, FP32 error < 1e-7 m); distances are
  // shrunk by kShrink and each term is inflated by 1 + 1e-4, which also
  // covers the FP32 rounding of the coefficient, the layer height and the
  // sum (n terms: n 2^-24 relative).
  constexpr float kShrink = 1e-7f;
  const double cxd = 0.5 * (bx0 + bx1), cyd = 0.5 * (by0 + by1);
  const float hx = float(0.5 * (bx1 - bx0)), hy = float(0.5 * (by1 - by0));
  const float inv_alpha = float(1.0 / sp.alpha);
  const float budget = float(T_hot - 1.0 - double(sp.T0));
  float sum = 0.0f;
  for (int j = 0; j < sp.n_tracks; ++j) {
    const TrackWin& tw = a.win[sp.track0 + j];
    if (!tw.on) continue;
    const float ux = tw.ux, uy = tw.uy, v = tw.v;
    // the source's path in the window, relative to the tile's centre
    const float ax = float(tw.ax - cxd), ay = float(tw.ay - cyd);
    const float bx = float(tw.bx - cxd), by = float(tw.by - cyd);
    const float dx = fmaxf(0.f, fmaxf(fminf(ax, bx) - hx, -hx - fmaxf(ax, bx)));
    const float dy = fmaxf(0.f, fmaxf(fminf(ay, by) - hy, -hy - fmaxf(ay, by)));
    const float dz = fmaxf(0.f, tw.z - bz1);
    const float R_min = sqrtf(dx * dx + dy * dy + dz * dz) - kShrink;
    if (!(R_min > 0.f)) return true;
    // smallest (x - x_s) . u over the box corners and the path's end points
    // (ahead of the path R + xi >= 2 xi), and the box corners' signed
    // distances from the source's line (which passes through a)
    float xi_min = INFINITY, s_lo = INFINITY, s_hi = -INFINITY;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float cx = (c & 1) ? hx : -hx, cy = (c & 2) ? hy : -hy;
      xi_min = fminf(xi_min, fminf((cx - ax) * ux + (cy - ay) * uy, (cx - bx) * ux + (cy - by) * uy));
      const float sd = (cx - ax) * uy - (cy - ay) * ux;
      s_lo = fminf(s_lo, sd);
      s_hi = fmaxf(s_hi, sd);
    }
    xi_min -= kShrink;
    const float ahead = xi_min > 0.f ? __expf(-v * xi_min * inv_alpha) : 1.f;
    // wake bound: R + xi = rho^2 / (R - xi) >= rho^2 / (2 R), rho being the
    // distance from the source's line, so a source contributes at most
    // C P exp(-a / R) / R with a = v rho_min^2 / (4 alpha); over R >= R_min
    // that is largest at R = max(R_min, a).
    const float lat =
        (s_lo <= 0.f && s_hi >= 0.f) ? 0.f : fmaxf(0.f, fminf(fabsf(s_lo), fabsf(s_hi)) - kShrink);
    const float aw = v * (lat * lat + dz * dz) * (0.25f * inv_alpha);
    const float wake = R_min >= aw ? __expf(-aw / R_min) / R_min : 1.f / (float(kE) * aw);
    sum += tw.cp * fminf(ahead / R_min, wake) * 1.0001f;
    if (sum >= budget) return true;  // already over: hot
  }
  return false;
}

// Cost class of an active tile: its cycles per level in the launch that last
// processed it against the previous launch's mean (0: >= 2x, 1: >= 1x, 2:
// >= 1/2 x, 3: below, or not measured).
__device__ __forceinline__ int cost_class(const ActiveArgs& a, int t, double mean) {
  if (!a.tile_cost || !(mean > 0.0)) return COST_BUCKETS - 1;
  const double c = double(a.tile_cost[t]);
  return c >= 2.0 * mean ? 0 : (c >= mean ? 1 : (c >= 0.5 * mean ? 2 : 3));
}

__global__ void k_active(const ActiveArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int prev = a.prev_slot & 1;
  const unsigned cnt = a.work->cost_cnt[prev];
  const double mean = cnt ? double(a.work->cost_sum[prev]) / double(cnt) : 0.0;
  if (t == 0) {  // this launch's slot, read by the next launch's active set
    a.work->cost_cnt[prev ^ 1] = 0;
    a.work->cost_sum[prev ^ 1] = 0;
  }
  const bool act = t < a.n_tiles && tile_is_active(a, t);
  const int cls = act ? cost_class(a, t, mean) : -1;
  const unsigned any = __ballot_sync(0xffffffffu, act);
  if (!any) return;
  if (lane == 0) atomicAdd(&a.work->n_active, __popc(any));
#pragma unroll
  for (int b = 0; b < COST_BUCKETS; ++b) {
    const unsigned mask = __ballot_sync(0xffffffffu, cls == b);
    if (!mask) continue;
    int base = 0;
    if (lane == 0) base = atomicAdd(&a.work->n_bucket[b], __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (cls == b)
      a.tile_list[int64_t(b) * a.n_tiles + base + __popc(mask & ((1u << lane) - 1u))] = t;
  }
}

}  // namespace

cudaError_t launch_active(const ActiveArgs& a, cudaStream_t stream) {
  if (a.n_tiles <= 0) return cudaSuccess;
  k_active<<<blocks_for(a.n_tiles, 128), 128, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace ms
