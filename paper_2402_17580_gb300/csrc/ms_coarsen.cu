// Phase-aware coarsening criterion (Sec. 3, the adaptive-mesh passage): an
// octant of eight sibling cells of one refinement level may be coarsened
// only where, for every phase (beta, alpha_s, alpha_m), its values lie close
// to each other.
//
// On the point grid: octant i of level l >= 1 spans the points i 2^l ..
// (i + 1) 2^l along an axis with n > 1 points (floor((n - 1) / 2^l)
// octants), and the whole axis if n == 1.  It may be coarsened when each
// phase's max - min over its points is <= tol.  Level 1 reduces the 3 x 3 x 3
// points of each octant; level l > 1 reduces the 2 x 2 x 2 children of level
// l - 1 (their spans tile the parent's, shared faces included), so every
// point is read once from memory per level-1 octant that holds it and the
// upper levels touch only the per-octant minima and maxima.  Levels 1 and 2
// run in one kernel (a thread reduces the level-1 octants of one level-2
// slot), so the level-1 ranges never go to memory.  The decisions
// are exact: minima and maxima are exact, the range is one FP64 subtraction.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ms_internal.h"

namespace ms {

namespace {

struct Range3 {
  double lo[3], hi[3];
};

__device__ __forceinline__ void span(int i, int n, int w, int& a, int& b) {
  if (n == 1) {
    a = 0;
    b = 0;
  } else {
    a = i * w;
    b = a + w;
  }
}

__device__ __forceinline__ bool decide(const Range3& r, double tol) {
  bool ok = true;
#pragma unroll
  for (int p = 0; p < 3; ++p) ok = ok && !(r.hi[p] - r.lo[p] > tol);
  return ok;
}

__device__ __forceinline__ void emit(const Range3& r, int64_t o, int64_t n_oct, double tol,
                                     Range3* mm, uint8_t* mask, unsigned long long* n_ok) {
  const bool ok = o < n_oct && decide(r, tol);
  if (o < n_oct) {
    if (mm) mm[o] = r;
    mask[o] = ok ? 1 : 0;
  }
  const unsigned b = __ballot_sync(0xffffffffu, ok);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_ok, (unsigned long long)__popc(b));
}

inline __host__ __device__ int axis_count(int n, int level) {
  return n == 1 ? 1 : (n - 1) >> level;
}

__device__ __forceinline__ void merge(Range3& r, const Range3& s) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    r.lo[p] = fmin(r.lo[p], s.lo[p]);
    r.hi[p] = fmax(r.hi[p], s.hi[p]);
  }
}

__device__ __forceinline__ Range3 empty_range() {
  Range3 r;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    r.lo[p] = INFINITY;
    r.hi[p] = -INFINITY;
  }
  return r;
}

// Levels 1 and 2 together: one thread per level-2 slot (the 2 x 2 x 2 level-1
// octants that would make a level-2 octant; at a ragged end of an axis a slot
// holds the one level-1 octant without a sibling, and no level-2 octant).
// Each level-1 octant reduces its 3 x 3 x 3 points (fewer on flat axes) and
// writes its mask; the slot's level-2 octant, where it exists, merges them
// and writes its mask and ranges.
__global__ void k_coarsen_l12(const double* __restrict__ xa, const double* __restrict__ xm,
                              const double* __restrict__ xb, int nx, int ny, int nz, double tol,
                              int want2, Range3* mm2, uint8_t* mask1, uint8_t* mask2,
                              unsigned long long* n_ok) {
  const int l1x = axis_count(nx, 1), l1y = axis_count(ny, 1), l1z = axis_count(nz, 1);
  const int l2x = axis_count(nx, 2), l2y = axis_count(ny, 2), l2z = axis_count(nz, 2);
  const int sx = nx == 1 ? 1 : (l1x + 1) / 2, sy = ny == 1 ? 1 : (l1y + 1) / 2;
  const int sz = nz == 1 ? 1 : (l1z + 1) / 2;
  const int64_t n_slot = int64_t(sx) * sy * sz;
  const int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  unsigned ok1 = 0, ok2 = 0;
  if (o < n_slot) {
    const int si = int(o % sx), sj = int((o / sx) % sy), sk = int(o / (int64_t(sx) * sy));
    const int ni = nx == 1 ? 1 : 2, nj = ny == 1 ? 1 : 2, nk = nz == 1 ? 1 : 2;
    Range3 par = empty_range();
    bool full = true;
    for (int ck = 0; ck < nk; ++ck) {
      const int qk = sk * nk + ck;
      if (qk >= l1z) { full = false; continue; }
      for (int cj = 0; cj < nj; ++cj) {
        const int qj = sj * nj + cj;
        if (qj >= l1y) { full = false; continue; }
        for (int ci = 0; ci < ni; ++ci) {
          const int qi = si * ni + ci;
          if (qi >= l1x) { full = false; continue; }
          int i0, i1, j0, j1, k0, k1;
          span(qi, nx, 2, i0, i1);
          span(qj, ny, 2, j0, j1);
          span(qk, nz, 2, k0, k1);
          Range3 r = empty_range();
          for (int kk = k0; kk <= k1; ++kk)
            for (int jj = j0; jj <= j1; ++jj) {
              const int64_t row = (int64_t(kk) * ny + jj) * nx;
              for (int ii = i0; ii <= i1; ++ii) {
                const double v[3] = {__ldg(xa + row + ii), __ldg(xm + row + ii),
                                     __ldg(xb + row + ii)};
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                  r.lo[p] = fmin(r.lo[p], v[p]);
                  r.hi[p] = fmax(r.hi[p], v[p]);
                }
              }
            }
          const bool d = decide(r, tol);
          mask1[(int64_t(qk) * l1y + qj) * l1x + qi] = d ? 1 : 0;
          ok1 += d ? 1u : 0u;
          merge(par, r);
        }
      }
    }
    // the level-2 octant exists exactly where the slot holds all its children
    if (want2 && full && si < l2x && sj < l2y && sk < l2z) {
      const int64_t o2 = (int64_t(sk) * l2y + sj) * l2x + si;
      const bool d = decide(par, tol);
      mask2[o2] = d ? 1 : 0;
      if (mm2) mm2[o2] = par;
      ok2 = d ? 1u : 0u;
    }
  }
  ok1 = __reduce_add_sync(0xffffffffu, ok1);
  ok2 = __reduce_add_sync(0xffffffffu, ok2);
  if ((threadIdx.x & 31) == 0) {
    if (ok1) atomicAdd(&n_ok[0], (unsigned long long)ok1);
    if (ok2 && want2) atomicAdd(&n_ok[1], (unsigned long long)ok2);
  }
}

// Level l > 1 from the children's ranges (level l - 1, ccx x ccy x ccz).
__global__ void k_coarsen_up(const Range3* __restrict__ child, int ccx, int ccy, int flat_x,
                             int flat_y, int flat_z, int cx, int cy, int cz, double tol,
                             Range3* mm, uint8_t* mask, unsigned long long* n_ok) {
  const int64_t n_oct = int64_t(cx) * cy * cz;
  const int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  Range3 r;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    r.lo[p] = INFINITY;
    r.hi[p] = -INFINITY;
  }
  if (o < n_oct) {
    const int i = int(o % cx);
    const int j = int((o / cx) % cy);
    const int k = int(o / (int64_t(cx) * cy));
    const int ni = flat_x ? 1 : 2, nj = flat_y ? 1 : 2, nk = flat_z ? 1 : 2;
    for (int c = 0; c < nk; ++c)
      for (int b = 0; b < nj; ++b)
        for (int a = 0; a < ni; ++a) {
          const int64_t q = (int64_t(k * nk + c) * ccy + (j * nj + b)) * ccx + (i * ni + a);
          const Range3 s = child[q];
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            r.lo[p] = fmin(r.lo[p], s.lo[p]);
            r.hi[p] = fmax(r.hi[p], s.hi[p]);
          }
        }
  }
  emit(r, o, n_oct, tol, mm, mask, n_ok);
}

}  // namespace

int64_t coarsen_counts(const int32_t dims[3], int n_levels, int64_t* per_level) {
  int64_t total = 0;
  for (int l = 1; l <= n_levels; ++l) {
    const int64_t c = int64_t(axis_count(dims[0], l)) * axis_count(dims[1], l) *
                      axis_count(dims[2], l);
    if (per_level) per_level[l - 1] = c;
    total += c;
  }
  return total;
}

size_t coarsen_scratch_bytes(const int32_t dims[3]) {
  // the level-2 ranges and the level-3 ranges (levels above alternate
  // between the two buffers), then the per-level counters
  const int64_t l2 = int64_t(axis_count(dims[0], 2)) * axis_count(dims[1], 2) *
                     axis_count(dims[2], 2);
  const int64_t l3 = int64_t(axis_count(dims[0], 3)) * axis_count(dims[1], 3) *
                     axis_count(dims[2], 3);
  return size_t(l2 + l3) * sizeof(Range3) + 64 * sizeof(unsigned long long);
}

cudaError_t launch_coarsen(const double* xa, const double* xm, const double* xb,
                           const int32_t dims[3], double tol, int n_levels, uint8_t* mask,
                           void* scratch, unsigned long long* n_ok, cudaStream_t stream) {
  const int nx = dims[0], ny = dims[1], nz = dims[2];
  int64_t per[64];
  coarsen_counts(dims, n_levels, per);
  Range3* A = static_cast<Range3*>(scratch);  // level 2 and the even levels above
  Range3* B = A + (n_levels >= 2 ? per[1] : 0);  // level 3 and the odd levels above
  cudaError_t e = cudaMemsetAsync(n_ok, 0, sizeof(unsigned long long) * size_t(n_levels), stream);
  if (e != cudaSuccess) return e;
  const int T = 256;
  if (per[0] > 0) {
    const int64_t slots = int64_t(nx == 1 ? 1 : (axis_count(nx, 1) + 1) / 2) *
                          (ny == 1 ? 1 : (axis_count(ny, 1) + 1) / 2) *
                          (nz == 1 ? 1 : (axis_count(nz, 1) + 1) / 2);
    k_coarsen_l12<<<unsigned((slots + T - 1) / T), T, 0, stream>>>(
        xa, xm, xb, nx, ny, nz, tol, n_levels >= 2, n_levels >= 3 ? A : nullptr, mask,
        mask + per[0], n_ok);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  int64_t off = per[0] + (n_levels >= 2 ? per[1] : 0);
  for (int l = 3; l <= n_levels; ++l) {
    const int cx = axis_count(nx, l), cy = axis_count(ny, l), cz = axis_count(nz, l);
    const int64_t n = per[l - 1];
    if (n > 0) {
      const Range3* in = (l & 1) ? A : B;
      Range3* out = (l == n_levels) ? nullptr : ((l & 1) ? B : A);
      k_coarsen_up<<<unsigned((n + T - 1) / T), T, 0, stream>>>(
          in, axis_count(nx, l - 1), axis_count(ny, l - 1), nx == 1, ny == 1, nz == 1, cx, cy,
          cz, tol, out, mask + off, n_ok + (l - 1));
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    off += n;
  }
  return cudaSuccess;
}

}  // namespace ms

// =============================================================== C ABI
namespace {

int check_coarsen_args(const int32_t* dims, int32_t n_levels, double tol) {
  if (!dims || dims[0] < 1 || dims[1] < 1 || dims[2] < 1)
    return ms::record_error(MS_ERR_INVALID_ARG, "grid dims must be >= 1");
  if (n_levels < 1 || n_levels > MS_COARSEN_MAX_LEVELS)
    return ms::record_error(MS_ERR_INVALID_ARG, "n_levels must be in [1, MS_COARSEN_MAX_LEVELS]");
  if (!(tol >= 0.0 && tol <= 1e300))
    return ms::record_error(MS_ERR_INVALID_ARG, "tol must be finite and >= 0");
  return MS_OK;
}

}  // namespace

extern "C" int ms_coarsen_sizes(const int32_t* dims, int32_t n_levels, int64_t* counts,
                                size_t* scratch_bytes) {
  int rc = check_coarsen_args(dims, n_levels, 0.0);
  if (rc != MS_OK) return rc;
  if (!counts) return ms::record_error(MS_ERR_INVALID_ARG, "counts is NULL");
  ms::coarsen_counts(dims, n_levels, counts);
  if (scratch_bytes) *scratch_bytes = ms::coarsen_scratch_bytes(dims) + 64 * sizeof(unsigned long long);
  return MS_OK;
}

extern "C" int ms_coarsen_mask(const double* x_as, const double* x_am, const double* x_beta,
                               const int32_t* dims, double tol, int32_t n_levels, uint8_t* mask,
                               int64_t* n_coarse, void* scratch, size_t scratch_bytes,
                               int32_t flags, void* stream) {
  int rc = check_coarsen_args(dims, n_levels, tol);
  if (rc != MS_OK) return rc;
  if (!x_as || !x_am || !x_beta || !mask)
    return ms::record_error(MS_ERR_INVALID_ARG, "NULL argument");
  const bool dev = (flags & MS_PTR_DEVICE) != 0;
  const int64_t n = int64_t(dims[0]) * dims[1] * dims[2];
  const int64_t total = ms::coarsen_counts(dims, n_levels, nullptr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sb = ms::coarsen_scratch_bytes(dims);
  const size_t need = sb + 64 * sizeof(unsigned long long);
  if (scratch && (!dev || scratch_bytes < need || (reinterpret_cast<uintptr_t>(scratch) & 15)))
    return ms::record_error(MS_ERR_INVALID_ARG,
                            "scratch needs MS_PTR_DEVICE, 16-byte alignment and the size "
                            "ms_coarsen_sizes gives");
  const size_t in_b = dev ? 0 : size_t(n) * 3 * sizeof(double);
  const size_t mask_b = dev ? 0 : size_t(total);
  char* own = nullptr;
  char* buf = static_cast<char*>(scratch);
  if (!buf) {
    if (cudaMalloc(&own, need + in_b + mask_b) != cudaSuccess)
      return ms::record_error(MS_ERR_OOM, "device allocation for the coarsening criterion failed");
    buf = own;
  }
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(buf + sb);
  double* din = reinterpret_cast<double*>(buf + need);
  uint8_t* dmask = dev ? mask : reinterpret_cast<uint8_t*>(din) + in_b;
  const double *a = x_as, *m = x_am, *b = x_beta;
  cudaError_t e = cudaSuccess;
  if (!dev) {
    const size_t nb = size_t(n) * sizeof(double);
    e = cudaMemcpyAsync(din, x_as, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(din + n, x_am, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(din + 2 * n, x_beta, nb, cudaMemcpyHostToDevice, st);
    a = din;
    m = din + n;
    b = din + 2 * n;
  }
  if (e == cudaSuccess)
    e = ms::launch_coarsen(a, m, b, dims, tol, n_levels, dmask, buf, cnt, st);
  unsigned long long hc[64] = {};
  if (e == cudaSuccess && !dev && total > 0)
    e = cudaMemcpyAsync(mask, dmask, size_t(total), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hc, cnt, sizeof(unsigned long long) * size_t(n_levels),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (own) cudaFree(own);
  if (e != cudaSuccess) return ms::record_error(MS_ERR_CUDA, cudaGetErrorString(e));
  if (n_coarse)
    for (int l = 0; l < n_levels; ++l) n_coarse[l] = int64_t(hc[l]);
  return MS_OK;
}
