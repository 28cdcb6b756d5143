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
// l - 1 (their spans tile the parent's, shared faces included), so the
// upper levels touch only the per-octant minima and maxima.  Levels 1 and 2
// run in one kernel (a block stages its brick of points in shared memory and
// reduces its level-1 octants and the level-2 octants they make), so the
// level-1 ranges never go to memory.  The decisions are exact: minima and
// maxima are exact, the range is one FP64 subtraction, and the test is
// range <= tol (false for a NaN, which reaches the range).
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ms_internal.h"

namespace ms {

namespace {

struct Range3 {
  double lo[3], hi[3];
};

// Order-preserving 64-bit integer keys of doubles: with the sign bit set the
// other 63 bits are flipped, so the signed integer order is the order of the
// doubles (-0 just below +0, NaNs beyond the infinities), and a key gives
// back its double exactly.
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dval(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

__device__ __forceinline__ bool decide(const Range3& r, double tol) {
  bool ok = true;
#pragma unroll
  for (int p = 0; p < 3; ++p) ok = ok && (r.hi[p] - r.lo[p] <= tol);
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

// Levels 1 and 2 together.  A block of CB_X x CB_Y x CB_Z threads takes as
// many level-1 octants (one per thread) and stages their points in shared
// memory: every warp copies whole rows of the block's point brick of all
// three fields at once with asynchronous copies (coalesced; one copy group
// per field, so the reduction of one field overlaps the copies of the next;
// the brick's faces are shared with the neighbouring blocks and read by
// both), so every point comes from memory once per block that holds it.
// Each field's values are turned into their integer keys in place, a thread
// reduces its octant's 3 x 3 x 3 points (fewer on a flat axis) and writes the
// level-1 mask; the level-2 octants, made of 2 x 2 x 2 level-1 octants of the
// same block (the block's extents are even), are then reduced from the
// threads' ranges in shared memory, one (octant, field, bound) per thread.
//
// Minima and maxima are taken on the doubles' integer keys (dkey), on the
// ALU pipe rather than the FP64 pipe; the keys give back the doubles
// exactly, so the ranges and the decisions are those of the doubles.
constexpr int CB_X = 16, CB_Y = 4, CB_Z = 4;
constexpr int CB_T = CB_X * CB_Y * CB_Z;
constexpr int CP_X = 2 * CB_X + 1, CP_Y = 2 * CB_Y + 1, CP_Z = 2 * CB_Z + 1;
constexpr int CP_N = CP_X * CP_Y * CP_Z;
constexpr size_t COARSEN_SMEM = 3 * size_t(CP_N) * sizeof(long long);
static_assert(6 * CB_T * sizeof(long long) + CB_T * sizeof(int) <= CP_N * sizeof(long long),
              "the level-2 ranges reuse the first field's brick");

struct KeyRange3 {
  long long lo[3], hi[3];
};

__device__ __forceinline__ bool decide_keys(const long long* lo, const long long* hi, int stride,
                                            double tol) {
  bool ok = true;
#pragma unroll
  for (int p = 0; p < 3; ++p) ok = ok && (dval(hi[p * stride]) - dval(lo[p * stride]) <= tol);
  return ok;
}

template <bool SOLID>
__global__ void __launch_bounds__(CB_T) k_coarsen_l12(
    const double* __restrict__ xa, const double* __restrict__ xm, const double* __restrict__ xb,
    int nx, int ny, int nz, double tol, int want2, Range3* mm2, uint8_t* mask1, uint8_t* mask2,
    unsigned long long* n_ok) {
  // SOLID: no flat axis, so every octant spans 3 x 3 x 3 points (unrolled).
  // Dynamic shared memory: the three fields' bricks; once the first field is
  // reduced (every thread has passed the second field's barrier) its brick
  // holds the threads' ranges (rr[6][CB_T]: lo of the fields, then hi) and
  // their flags.
  extern __shared__ long long csm[];
  long long* pts = csm;
  long long* rr = csm;
  int* have_s = reinterpret_cast<int*>(rr + 6 * CB_T);
  const int l1x = axis_count(nx, 1), l1y = axis_count(ny, 1), l1z = axis_count(nz, 1);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tx = tid % CB_X, ty = (tid / CB_X) % CB_Y, tz = tid / (CB_X * CB_Y);
  const int qi = blockIdx.x * CB_X + tx, qj = blockIdx.y * CB_Y + ty, qk = blockIdx.z * CB_Z + tz;
  const bool have = qi < l1x && qj < l1y && qk < l1z;
  // the block's point brick: along a flat axis the single point
  const int x0 = nx == 1 ? 0 : 2 * blockIdx.x * CB_X, y0 = ny == 1 ? 0 : 2 * blockIdx.y * CB_Y;
  const int z0 = nz == 1 ? 0 : 2 * blockIdx.z * CB_Z;
  const int wx = min(CP_X, nx - x0), wy = min(CP_Y, ny - y0), wz = min(CP_Z, nz - z0);
  // the thread's octant inside the brick
  const int i0 = nx == 1 ? 0 : 2 * tx, j0 = ny == 1 ? 0 : 2 * ty, k0 = nz == 1 ? 0 : 2 * tz;
  const int ei = nx == 1 ? 0 : 2, ej = ny == 1 ? 0 : 2, ek = nz == 1 ? 0 : 2;

  // asynchronous copies of the three bricks; warp wid takes rows wid, wid + 8, ...
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const double* f = p == 0 ? xa : (p == 1 ? xm : xb);
    int jj = wid, kk = 0;
    while (jj >= wy) {
      jj -= wy;
      ++kk;
    }
    while (kk < wz) {
      const double* src = f + (int64_t(z0 + kk) * ny + (y0 + jj)) * nx + x0;
      const unsigned dst = unsigned(__cvta_generic_to_shared(pts + p * CP_N + (kk * CP_Y + jj) * CP_X));
      for (int ii = lane; ii < wx; ii += 32)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst + 8u * unsigned(ii)),
                     "l"(src + ii)
                     : "memory");
      jj += CB_T / 32;
      while (jj >= wy) {
        jj -= wy;
        ++kk;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }

  long long lo[3], hi[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    if (p == 0) asm volatile("cp.async.wait_group 2;" ::: "memory");
    if (p == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    if (p == 2) asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();  // every thread's copies of this field have landed
    long long* b = pts + p * CP_N;
    for (int e = tid; e < CP_N; e += CB_T) b[e] = dkey(__longlong_as_double(b[e]));
    __syncthreads();
    const long long* mine = b + (k0 * CP_Y + j0) * CP_X + i0;
    long long l = 0x7fffffffffffffffLL, h = -0x7fffffffffffffffLL - 1;
    if (have) {
      if constexpr (SOLID) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int bb = 0; bb < 3; ++bb)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const long long v = mine[(c * CP_Y + bb) * CP_X + a];
              l = llmin(l, v);
              h = llmax(h, v);
            }
      } else {
        for (int c = 0; c <= ek; ++c)
          for (int bb = 0; bb <= ej; ++bb)
            for (int a = 0; a <= ei; ++a) {
              const long long v = mine[(c * CP_Y + bb) * CP_X + a];
              l = llmin(l, v);
              h = llmax(h, v);
            }
      }
    }
    lo[p] = l;
    hi[p] = h;
  }
  unsigned ok1 = 0;
  if (have) {
    const bool d = decide_keys(lo, hi, 1, tol);
    mask1[(int64_t(qk) * l1y + qj) * l1x + qi] = d ? 1 : 0;
    ok1 = d ? 1u : 0u;
  }
  ok1 = __reduce_add_sync(0xffffffffu, ok1);
  if (lane == 0 && ok1) atomicAdd(&n_ok[0], (unsigned long long)ok1);
  if (!want2) return;  // uniform over the block

  // level 2: slots of ni x nj x nk level-1 octants inside the block
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    rr[p * CB_T + tid] = lo[p];
    rr[(3 + p) * CB_T + tid] = hi[p];
  }
  have_s[tid] = have ? 1 : 0;
  __syncthreads();
  const int ni = nx == 1 ? 1 : 2, nj = ny == 1 ? 1 : 2, nk = nz == 1 ? 1 : 2;
  const int sxn = CB_X / ni, syn = CB_Y / nj, szn = CB_Z / nk;
  const int n_slot = sxn * syn * szn;  // <= CB_T
  const int l2x = axis_count(nx, 2), l2y = axis_count(ny, 2), l2z = axis_count(nz, 2);
  // (slot, bound) per thread: the bound's key over the slot's children,
  // written over the first child's entry once every thread has read
  long long red[6];
  int first[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) {  // 6 n_slot <= 6 CB_T tasks
    const int t = tid + r * CB_T;
    first[r] = -1;
    if (t < 6 * n_slot) {
      const int slot = t % n_slot, w = t / n_slot;  // w: 0..2 lo of field w, 3..5 hi
      const int a = slot % sxn, b = (slot / sxn) % syn, c = slot / (sxn * syn);
      long long v = w < 3 ? 0x7fffffffffffffffLL : -0x7fffffffffffffffLL - 1;
      for (int cc = 0; cc < nk; ++cc)
        for (int bb = 0; bb < nj; ++bb)
          for (int aa = 0; aa < ni; ++aa) {
            const int u = ((c * nk + cc) * CB_Y + (b * nj + bb)) * CB_X + (a * ni + aa);
            const long long x = rr[w * CB_T + u];
            v = w < 3 ? llmin(v, x) : llmax(v, x);
          }
      red[r] = v;
      first[r] = w * CB_T + ((c * nk) * CB_Y + b * nj) * CB_X + a * ni;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 6; ++r)
    if (first[r] >= 0) rr[first[r]] = red[r];
  __syncthreads();
  unsigned ok2 = 0;
  for (int slot = tid; slot < n_slot; slot += CB_T) {
    const int a = slot % sxn, b = (slot / sxn) % syn, c = slot / (sxn * syn);
    const int si = (nx == 1 ? 0 : blockIdx.x * sxn) + a, sj = (ny == 1 ? 0 : blockIdx.y * syn) + b;
    const int sk = (nz == 1 ? 0 : blockIdx.z * szn) + c;
    if (si >= l2x || sj >= l2y || sk >= l2z) continue;
    bool full = true;
    for (int cc = 0; cc < nk; ++cc)
      for (int bb = 0; bb < nj; ++bb)
        for (int aa = 0; aa < ni; ++aa)
          full = full && have_s[((c * nk + cc) * CB_Y + (b * nj + bb)) * CB_X + (a * ni + aa)];
    if (!full) continue;
    const int u0 = ((c * nk) * CB_Y + b * nj) * CB_X + a * ni;
    const int64_t o2 = (int64_t(sk) * l2y + sj) * l2x + si;
    const bool d = decide_keys(rr + u0, rr + 3 * CB_T + u0, CB_T, tol);
    mask2[o2] = d ? 1 : 0;
    ok2 += d ? 1u : 0u;
    if (mm2) {
      Range3 out;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        out.lo[p] = dval(rr[p * CB_T + u0]);
        out.hi[p] = dval(rr[(3 + p) * CB_T + u0]);
      }
      mm2[o2] = out;
    }
  }
  ok2 = __reduce_add_sync(0xffffffffu, ok2);
  if (lane == 0 && ok2) atomicAdd(&n_ok[1], (unsigned long long)ok2);
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
            r.lo[p] = dkey(s.lo[p]) < dkey(r.lo[p]) ? s.lo[p] : r.lo[p];
            r.hi[p] = dkey(s.hi[p]) > dkey(r.hi[p]) ? s.hi[p] : r.hi[p];
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
    const dim3 grid(unsigned((axis_count(nx, 1) + CB_X - 1) / CB_X),
                    unsigned((axis_count(ny, 1) + CB_Y - 1) / CB_Y),
                    unsigned((axis_count(nz, 1) + CB_Z - 1) / CB_Z));
    if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
    static bool attr = false;  // opt in to the dynamic shared memory once per process
    if (!attr) {
      e = cudaFuncSetAttribute(k_coarsen_l12<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(COARSEN_SMEM));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_coarsen_l12<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(COARSEN_SMEM));
      if (e != cudaSuccess) return e;
      attr = true;
    }
    if (nx > 1 && ny > 1 && nz > 1)
      k_coarsen_l12<true><<<grid, CB_T, COARSEN_SMEM, stream>>>(
          xa, xm, xb, nx, ny, nz, tol, n_levels >= 2, n_levels >= 3 ? A : nullptr, mask,
          mask + per[0], n_ok);
    else
      k_coarsen_l12<false><<<grid, CB_T, COARSEN_SMEM, stream>>>(
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
