// The learned surrogate's object, training kernels and batched inference.
//
//  k_mlp_pack     FP32 master parameters -> the padded BF16 layout (MlpDev)
//                 that inference and training read.
//  k_mlp_fwd_bwd_tc  forward, MSE loss and backward on the tensor cores
//                 (mma.sync m16n8k16, BF16 operands, FP32 accumulation), 16
//                 samples per warp tile; writes each tile's weight-gradient
//                 operands (transposed, BF16) to the scratch.
//  k_mlp_wgrad_tc the weight gradients as tensor-core contractions over the
//                 samples, split over blocks; k_mlp_reduce_partials adds the
//                 blocks' partials in a fixed order.
//  k_adam         Adam on the FP32 master copy, then repack.
//  k_mlp_infer    batched inference on the tensor cores (mma.sync bf16,
//                 FP32 accumulation), 128 samples per warp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "ms_internal.h"
#include "ms_mlp.cuh"

using ms::MlpDev;

struct ms_surrogate {
  float* params = nullptr;   // FP32 master copy
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  MlpDev* mlp = nullptr;     // inference layout
  double* loss = nullptr;
  void* scratch = nullptr;   // per-tile operands of the weight gradient, block partials
  size_t scratch_cap = 0;    // bytes
  int64_t step = 0;
  int32_t act = MS_ACT_GELU;  // hidden activation
  int32_t stride = 1;         // levels between the window's temperature samples
  cudaStream_t own = nullptr, stream = nullptr;
};

namespace {


#define SG_CUDA(...)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                  \
    if (e_ != cudaSuccess) return ms::record_error(e_ == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

__global__ void k_mlp_pack(const float* p, MlpDev* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ms::MLP_H * ms::MLP_W1_LD) {
    const int j = i / ms::MLP_W1_LD, k = i % ms::MLP_W1_LD;
    d->w1[i] = __float2bfloat16_rn(k < ms::MLP_IN ? p[ms::MLP_OFF_W1 + j * ms::MLP_IN + k] : 0.0f);
  }
  if (i < ms::MLP_H * ms::MLP_W2_LD) {
    const int j = i / ms::MLP_W2_LD, k = i % ms::MLP_W2_LD;
    d->w2[i] = __float2bfloat16_rn(k < ms::MLP_H ? p[ms::MLP_OFF_W2 + j * ms::MLP_H + k] : 0.0f);
  }
  if (i < ms::MLP_OUT_PAD * ms::MLP_W3_LD) {
    const int o = i / ms::MLP_W3_LD, k = i % ms::MLP_W3_LD;
    d->w3[i] = __float2bfloat16_rn(o < ms::MLP_OUT && k < ms::MLP_H
                                       ? p[ms::MLP_OFF_W3 + o * ms::MLP_H + k] : 0.0f);
  }
  if (i < ms::MLP_H) {
    d->b1[i] = p[ms::MLP_OFF_B1 + i];
    d->b2[i] = p[ms::MLP_OFF_B2 + i];
  }
  if (i < ms::MLP_OUT_PAD) d->b3[i] = i < ms::MLP_OUT ? p[ms::MLP_OFF_B3 + i] : 0.0f;
}

// ------------------------------------------------------------ training
// Forward and backward on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation): every warp takes 16-sample tiles.  The activations are
// rounded to BF16 between layers as in the inference pass; the backward pass
// feeds its upstream gradients to the tensor cores in BF16 as well.  Per
// tile the kernel writes the operands of the weight-gradient contraction,
// transposed (feature-major, 16 samples per row) and in BF16, to the
// scratch: the inputs (with a column of ones for the first bias), both
// hidden activations, both hidden pre-activation gradients and the output
// gradient.  k_mlp_wgrad_tc then contracts them over the samples.
constexpr int kT = 16;                                    // samples per tile
constexpr int kRowX = 0, kRowA1 = 16, kRowA2 = 80, kRowD1 = 144, kRowD2 = 208, kRowDy = 272;
constexpr int kTileRows = 288;                            // feature rows per tile
constexpr int kTileElems = kTileRows * kT;                // BF16 per tile
constexpr int kW2T_LD = ms::MLP_W2_LD, kW3T_LD = ms::MLP_W1_LD;
constexpr int kFwdWarps = 4;

struct TrainSmem {
  MlpDev W;                                               // forward operands
  __nv_bfloat16 w2t[ms::MLP_H * kW2T_LD];                 // W2 transposed [in][out]
  __nv_bfloat16 w3t[ms::MLP_H * kW3T_LD];                 // W3 transposed [in][out (16)]
  __nv_bfloat16 stage[kFwdWarps][kTileElems];             // per warp: one tile's operands
};

__device__ __forceinline__ void put(__nv_bfloat16* st, int row, int col, float v) {
  st[row * kT + col] = __float2bfloat16_rn(v);
}

template <int ACT>
__global__ void __launch_bounds__(kFwdWarps * 32) k_mlp_fwd_bwd_tc(
    const MlpDev* __restrict__ wd, const float* __restrict__ x, const float* __restrict__ t,
    int64_t n, __nv_bfloat16* __restrict__ sc, double* loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(wd);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&S.W);
    for (int i = threadIdx.x; i < int(sizeof(MlpDev) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ms::MLP_H * kW2T_LD; i += blockDim.x) {
    const int r = i / kW2T_LD, c = i % kW2T_LD;   // w2t[r = in][c = out] = W2[out][in]
    S.w2t[i] = c < ms::MLP_H ? S.W.w2[c * ms::MLP_W2_LD + r] : __float2bfloat16_rn(0.0f);
  }
  for (int i = threadIdx.x; i < ms::MLP_H * kW3T_LD; i += blockDim.x) {
    const int r = i / kW3T_LD, c = i % kW3T_LD;   // w3t[r = in][c = out] = W3[out][in]
    S.w3t[i] = c < ms::MLP_OUT_PAD ? S.W.w3[c * ms::MLP_W3_LD + r] : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  __nv_bfloat16* st = S.stage[warp];
  const int64_t n_tiles = (n + kT - 1) / kT;
  const float inv = 1.0f / float(3 * n);
  double lsum = 0.0;
  for (int64_t tile = int64_t(blockIdx.x) * kFwdWarps + warp; tile < n_tiles;
       tile += int64_t(gridDim.x) * kFwdWarps) {
    const int64_t s0 = tile * kT;
    const int64_t sa = s0 + g, sb = s0 + g + 8;           // this lane's two sample rows
    const bool va = sa < n, vb = sb < n;
    // inputs: features 0..11, a column of ones at 12 (the first bias's gradient)
    float xa[16], xb[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      xa[k] = k < ms::MLP_IN ? (va ? ms::bf16r(x[sa * ms::MLP_IN + k]) : 0.0f) : (k == 12 && va ? 1.0f : 0.0f);
      xb[k] = k < ms::MLP_IN ? (vb ? ms::bf16r(x[sb * ms::MLP_IN + k]) : 0.0f) : (k == 12 && vb ? 1.0f : 0.0f);
    }
    uint32_t a[4];
    a[0] = ms::pack_bf16(xa[2 * q], xa[2 * q + 1]);
    a[1] = ms::pack_bf16(xb[2 * q], xb[2 * q + 1]);
    a[2] = ms::pack_bf16(xa[8 + 2 * q], xa[8 + 2 * q + 1]);
    a[3] = ms::pack_bf16(xb[8 + 2 * q], xb[8 + 2 * q + 1]);
    // the inputs' ones column must not reach the forward pass: W1's padding
    // columns (12..15) are zero
    float h1[8][4], h2[8][4];
#pragma unroll
    for (int tt = 0; tt < 8; ++tt) {
      const float c[4] = {S.W.b1[8 * tt + 2 * q], S.W.b1[8 * tt + 2 * q + 1], S.W.b1[8 * tt + 2 * q],
                          S.W.b1[8 * tt + 2 * q + 1]};
      const __nv_bfloat16* wr = S.W.w1 + (8 * tt + g) * ms::MLP_W1_LD;
      ms::mma_bf16_16816(h1[tt], a, ms::ld32(wr + 2 * q), ms::ld32(wr + 8 + 2 * q), c);
    }
    uint32_t f1[4][4], f2[4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      f1[kc][0] = ms::pack_act<ACT>(h1[2 * kc][0], h1[2 * kc][1]);
      f1[kc][1] = ms::pack_act<ACT>(h1[2 * kc][2], h1[2 * kc][3]);
      f1[kc][2] = ms::pack_act<ACT>(h1[2 * kc + 1][0], h1[2 * kc + 1][1]);
      f1[kc][3] = ms::pack_act<ACT>(h1[2 * kc + 1][2], h1[2 * kc + 1][3]);
    }
#pragma unroll
    for (int tt = 0; tt < 8; ++tt) {
      h2[tt][0] = h2[tt][2] = S.W.b2[8 * tt + 2 * q];
      h2[tt][1] = h2[tt][3] = S.W.b2[8 * tt + 2 * q + 1];
      const __nv_bfloat16* wr = S.W.w2 + (8 * tt + g) * ms::MLP_W2_LD;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        ms::mma_bf16_16816(h2[tt], f1[kc], ms::ld32(wr + 16 * kc + 2 * q),
                           ms::ld32(wr + 16 * kc + 8 + 2 * q), h2[tt]);
    }
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      f2[kc][0] = ms::pack_act<ACT>(h2[2 * kc][0], h2[2 * kc][1]);
      f2[kc][1] = ms::pack_act<ACT>(h2[2 * kc][2], h2[2 * kc][3]);
      f2[kc][2] = ms::pack_act<ACT>(h2[2 * kc + 1][0], h2[2 * kc + 1][1]);
      f2[kc][3] = ms::pack_act<ACT>(h2[2 * kc + 1][2], h2[2 * kc + 1][3]);
    }
    float y[4] = {S.W.b3[2 * q], S.W.b3[2 * q + 1], S.W.b3[2 * q], S.W.b3[2 * q + 1]};
    {
      const __nv_bfloat16* wr = S.W.w3 + g * ms::MLP_W3_LD;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        ms::mma_bf16_16816(y, f2[kc], ms::ld32(wr + 16 * kc + 2 * q),
                           ms::ld32(wr + 16 * kc + 8 + 2 * q), y);
    }
    // output gradient dL/dy = 2 (y - t) / (3 n) on the 3 outputs of valid rows
    float dy[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = 2 * q + (e & 1);
      const bool v = (e < 2 ? va : vb) && c < ms::MLP_OUT;
      const int64_t sr = e < 2 ? sa : sb;
      const float r = v ? y[e] - t[sr * ms::MLP_OUT + c] : 0.0f;
      lsum += double(r) * double(r) * double(inv);
      dy[e] = 2.0f * r * inv;
    }
    // dL/dh2 = (dy W3) * act'(h2): dy as the A operand (K = outputs, 8 of 16)
    uint32_t fd[4] = {ms::pack_bf16(dy[0], dy[1]), ms::pack_bf16(dy[2], dy[3]), 0u, 0u};
    float d2[8][4];
#pragma unroll
    for (int tt = 0; tt < 8; ++tt) {
      const float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const __nv_bfloat16* wr = S.w3t + (8 * tt + g) * kW3T_LD;
      ms::mma_bf16_16816(d2[tt], fd, ms::ld32(wr + 2 * q), ms::ld32(wr + 8 + 2 * q), z);
#pragma unroll
      for (int e = 0; e < 4; ++e) d2[tt][e] *= ms::act_grad<ACT>(h2[tt][e]);
    }
    // dL/dh1 = (dh2 W2) * act'(h1)
    uint32_t fg[4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      fg[kc][0] = ms::pack_bf16(d2[2 * kc][0], d2[2 * kc][1]);
      fg[kc][1] = ms::pack_bf16(d2[2 * kc][2], d2[2 * kc][3]);
      fg[kc][2] = ms::pack_bf16(d2[2 * kc + 1][0], d2[2 * kc + 1][1]);
      fg[kc][3] = ms::pack_bf16(d2[2 * kc + 1][2], d2[2 * kc + 1][3]);
    }
    // stage the tile's operands, transposed: row = feature, column = sample
#pragma unroll
    for (int k = 0; k < 2; ++k) {   // inputs: this lane's features 2q, 2q + 1, 8 + 2q, 9 + 2q
      put(st, kRowX + 8 * k + 2 * q, g, xa[8 * k + 2 * q]);
      put(st, kRowX + 8 * k + 2 * q + 1, g, xa[8 * k + 2 * q + 1]);
      put(st, kRowX + 8 * k + 2 * q, g + 8, xb[8 * k + 2 * q]);
      put(st, kRowX + 8 * k + 2 * q + 1, g + 8, xb[8 * k + 2 * q + 1]);
    }
#pragma unroll
    for (int tt = 0; tt < 8; ++tt) {
      const int f0 = 8 * tt + 2 * q;
      put(st, kRowA1 + f0, g, ms::act<ACT>(h1[tt][0]));
      put(st, kRowA1 + f0 + 1, g, ms::act<ACT>(h1[tt][1]));
      put(st, kRowA1 + f0, g + 8, ms::act<ACT>(h1[tt][2]));
      put(st, kRowA1 + f0 + 1, g + 8, ms::act<ACT>(h1[tt][3]));
      put(st, kRowA2 + f0, g, ms::act<ACT>(h2[tt][0]));
      put(st, kRowA2 + f0 + 1, g, ms::act<ACT>(h2[tt][1]));
      put(st, kRowA2 + f0, g + 8, ms::act<ACT>(h2[tt][2]));
      put(st, kRowA2 + f0 + 1, g + 8, ms::act<ACT>(h2[tt][3]));
      put(st, kRowD2 + f0, g, d2[tt][0]);
      put(st, kRowD2 + f0 + 1, g, d2[tt][1]);
      put(st, kRowD2 + f0, g + 8, d2[tt][2]);
      put(st, kRowD2 + f0 + 1, g + 8, d2[tt][3]);
    }
#pragma unroll
    for (int tt = 0; tt < 8; ++tt) {
      float d1[4];
      const float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const __nv_bfloat16* wr = S.w2t + (8 * tt + g) * kW2T_LD;
      ms::mma_bf16_16816(d1, fg[0], ms::ld32(wr + 2 * q), ms::ld32(wr + 8 + 2 * q), z);
#pragma unroll
      for (int kc = 1; kc < 4; ++kc)
        ms::mma_bf16_16816(d1, fg[kc], ms::ld32(wr + 16 * kc + 2 * q),
                           ms::ld32(wr + 16 * kc + 8 + 2 * q), d1);
      const int f0 = 8 * tt + 2 * q;
      put(st, kRowD1 + f0, g, d1[0] * ms::act_grad<ACT>(h1[tt][0]));
      put(st, kRowD1 + f0 + 1, g, d1[1] * ms::act_grad<ACT>(h1[tt][1]));
      put(st, kRowD1 + f0, g + 8, d1[2] * ms::act_grad<ACT>(h1[tt][2]));
      put(st, kRowD1 + f0 + 1, g + 8, d1[3] * ms::act_grad<ACT>(h1[tt][3]));
    }
    // output gradient rows 0..7 (this lane's outputs 2q, 2q + 1), rows 8..15 zero
    put(st, kRowDy + 2 * q, g, dy[0]);
    put(st, kRowDy + 2 * q + 1, g, dy[1]);
    put(st, kRowDy + 2 * q, g + 8, dy[2]);
    put(st, kRowDy + 2 * q + 1, g + 8, dy[3]);
    put(st, kRowDy + 8 + 2 * q, g, 0.0f);
    put(st, kRowDy + 9 + 2 * q, g, 0.0f);
    put(st, kRowDy + 8 + 2 * q, g + 8, 0.0f);
    put(st, kRowDy + 9 + 2 * q, g + 8, 0.0f);
    __syncwarp();
    const uint4* src = reinterpret_cast<const uint4*>(st);
    uint4* dst = reinterpret_cast<uint4*>(sc + tile * kTileElems);
    for (int i = lane; i < kTileElems / 8; i += 32) dst[i] = src[i];
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0 && lsum != 0.0) atomicAdd(loss, lsum);
}

// Weight gradients on the tensor cores: dW = (upstream gradient)^T x
// (activation), contracted over the samples of the tiles k_mlp_fwd_bwd_tc
// wrote.  Each block takes a contiguous range of tiles (split over the
// samples) and writes its partial gradient of every parameter; warp w owns
// rows 16w .. 16w + 15 of dW2, dW1 (whose input column 12 is the ones
// column, i.e. the first bias) and db2 (against a column of ones), columns
// 16w .. 16w + 15 of dW3, and warp 0 db3.  k_mlp_reduce_partials adds the
// blocks' partials in block order.
constexpr int kGradBlocks = 128;

__global__ void __launch_bounds__(128) k_mlp_wgrad_tc(const __nv_bfloat16* __restrict__ sc,
                                                      int64_t n_tiles, float* __restrict__ partial) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int64_t t0 = n_tiles * blockIdx.x / gridDim.x, t1 = n_tiles * (blockIdx.x + 1) / gridDim.x;
  float a2c[8][4] = {}, a1c[2][4] = {}, b2c[4] = {}, a3c[2][4] = {}, b3c[4] = {};
  const uint32_t one = g == 0 ? ms::pack_bf16(1.0f, 1.0f) : 0u;  // B = ones in column 0
  auto frag_a = [&](const __nv_bfloat16* base, int row, uint32_t* a) {
    a[0] = ms::ld32(base + (row + g) * kT + 2 * q);
    a[1] = ms::ld32(base + (row + g + 8) * kT + 2 * q);
    a[2] = ms::ld32(base + (row + g) * kT + 8 + 2 * q);
    a[3] = ms::ld32(base + (row + g + 8) * kT + 8 + 2 * q);
  };
  for (int64_t tile = t0; tile < t1; ++tile) {
    const __nv_bfloat16* base = sc + tile * kTileElems;
    uint32_t ad2[4], ad1[4], ady[4];
    frag_a(base, kRowD2 + 16 * warp, ad2);
    frag_a(base, kRowD1 + 16 * warp, ad1);
    frag_a(base, kRowDy, ady);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const __nv_bfloat16* r = base + (kRowA1 + 8 * nt + g) * kT;
      ms::mma_bf16_16816(a2c[nt], ad2, ms::ld32(r + 2 * q), ms::ld32(r + 8 + 2 * q), a2c[nt]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const __nv_bfloat16* r = base + (kRowX + 8 * nt + g) * kT;
      ms::mma_bf16_16816(a1c[nt], ad1, ms::ld32(r + 2 * q), ms::ld32(r + 8 + 2 * q), a1c[nt]);
      const __nv_bfloat16* r3 = base + (kRowA2 + 16 * warp + 8 * nt + g) * kT;
      ms::mma_bf16_16816(a3c[nt], ady, ms::ld32(r3 + 2 * q), ms::ld32(r3 + 8 + 2 * q), a3c[nt]);
    }
    ms::mma_bf16_16816(b2c, ad2, one, one, b2c);
    if (warp == 0) ms::mma_bf16_16816(b3c, ady, one, one, b3c);
  }
  float* out = partial + int64_t(blockIdx.x) * ms::MLP_PARAMS;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int row = 16 * warp + g + (e >= 2 ? 8 : 0);   // j2 or j1
    const int col = 2 * q + (e & 1);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) out[ms::MLP_OFF_W2 + row * ms::MLP_H + 8 * nt + col] = a2c[nt][e];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int i = 8 * nt + col;
      if (i < ms::MLP_IN) out[ms::MLP_OFF_W1 + row * ms::MLP_IN + i] = a1c[nt][e];
      else if (i == 12) out[ms::MLP_OFF_B1 + row] = a1c[nt][e];
      const int o = g + (e >= 2 ? 8 : 0);
      if (o < ms::MLP_OUT) out[ms::MLP_OFF_W3 + o * ms::MLP_H + 16 * warp + 8 * nt + col] = a3c[nt][e];
    }
    if (col == 0) {
      out[ms::MLP_OFF_B2 + row] = b2c[e];
      const int o = g + (e >= 2 ? 8 : 0);
      if (warp == 0 && o < ms::MLP_OUT) out[ms::MLP_OFF_B3 + o] = b3c[e];
    }
  }
}

__global__ void k_mlp_reduce_partials(const float* __restrict__ partial, int blocks, float* grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ms::MLP_PARAMS) return;
  float acc = 0.0f;
  for (int b = 0; b < blocks; ++b) acc += partial[int64_t(b) * ms::MLP_PARAMS + i];
  grad[i] = acc;
}

__global__ void k_adam(float* p, float* m, float* v, const float* g, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ms::MLP_PARAMS) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Batched inference: each warp takes 128 samples (x: [n][12], y: [n][3]).
template <int ACT>
__global__ void __launch_bounds__(128) k_mlp_infer(const MlpDev* __restrict__ wd,
                                                   const float* __restrict__ x, float* __restrict__ y,
                                                   int64_t n) {
  extern __shared__ __align__(16) unsigned char smem[];
  MlpDev& W = *reinterpret_cast<MlpDev*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(smem + sizeof(MlpDev)) + warp * 128 * ms::MLP_X_LD;
  float* Y = reinterpret_cast<float*>(smem + sizeof(MlpDev) + 4 * 128 * ms::MLP_X_LD * 2) +
             warp * 128 * ms::MLP_Y_COLS;
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(wd);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&W);
    for (int i = threadIdx.x; i < int(sizeof(MlpDev) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int64_t base = (int64_t(blockIdx.x) * 4 + warp) * 128;
  for (int r = lane; r < 128; r += 32) {
    const int64_t s = base + r;
    for (int k = 0; k < ms::MLP_IN_PAD; ++k)
      X[r * ms::MLP_X_LD + k] = __float2bfloat16_rn(s < n && k < ms::MLP_IN ? x[s * ms::MLP_IN + k] : 0.0f);
  }
  __syncwarp();
  ms::mlp_forward_warp<ACT>(W, X, Y, lane);
  __syncwarp();
  for (int r = lane; r < 128; r += 32) {
    const int64_t s = base + r;
    if (s < n)
      for (int i = 0; i < ms::MLP_OUT; ++i) y[s * ms::MLP_OUT + i] = Y[i * 128 + r];
  }
}

constexpr size_t kInferSmem = sizeof(MlpDev) + 4 * 128 * ms::MLP_X_LD * 2 + 4 * 128 * ms::MLP_Y_COLS * 4;
static_assert(kInferSmem <= 48 * 1024, "k_mlp_infer stays within the default dynamic shared memory");
static_assert(sizeof(MlpDev) % 16 == 0, "MlpDev is copied in 16-byte words");

int pack(ms_surrogate* s) {
  // one thread per parameter; the largest packed block (padded W2) is smaller
  static_assert(ms::MLP_PARAMS >= ms::MLP_H * ms::MLP_W2_LD, "pack grid");
  k_mlp_pack<<<(ms::MLP_PARAMS + 255) / 256, 256, 0, s->stream>>>(s->params, s->mlp);
  SG_CUDA(cudaGetLastError());
  return MS_OK;
}

int gradient(ms_surrogate* s, const float* x, const float* t, int64_t n) {
  const int64_t n_tiles = (n + kT - 1) / kT;
  const size_t need = size_t(n_tiles) * kTileElems * sizeof(__nv_bfloat16) +
                      size_t(kGradBlocks) * ms::MLP_PARAMS * sizeof(float);
  if (need > s->scratch_cap) {
    SG_CUDA(cudaStreamSynchronize(s->stream));
    cudaFree(s->scratch);
    s->scratch = nullptr;
    s->scratch_cap = 0;
    SG_CUDA(cudaMalloc(&s->scratch, need));
    s->scratch_cap = need;
  }
  __nv_bfloat16* tiles = reinterpret_cast<__nv_bfloat16*>(s->scratch);
  float* partial = reinterpret_cast<float*>(reinterpret_cast<char*>(s->scratch) +
                                            size_t(n_tiles) * kTileElems * sizeof(__nv_bfloat16));
  SG_CUDA(cudaMemsetAsync(s->loss, 0, sizeof(double), s->stream));
  auto fwd_bwd = s->act == MS_ACT_RELU ? k_mlp_fwd_bwd_tc<ms::ACT_RELU> : k_mlp_fwd_bwd_tc<ms::ACT_GELU>;
  SG_CUDA(cudaFuncSetAttribute(fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(sizeof(TrainSmem))));
  const int fwd_blocks = int(std::min<int64_t>((n_tiles + kFwdWarps - 1) / kFwdWarps, 2048));
  fwd_bwd<<<fwd_blocks, kFwdWarps * 32, sizeof(TrainSmem), s->stream>>>(s->mlp, x, t, n, tiles,
                                                                       s->loss);
  SG_CUDA(cudaGetLastError());
  const int gb = int(std::min<int64_t>(n_tiles, kGradBlocks));
  k_mlp_wgrad_tc<<<gb, 128, 0, s->stream>>>(tiles, n_tiles, partial);
  SG_CUDA(cudaGetLastError());
  k_mlp_reduce_partials<<<(ms::MLP_PARAMS + 255) / 256, 256, 0, s->stream>>>(partial, gb, s->grad);
  SG_CUDA(cudaGetLastError());
  return MS_OK;
}

}  // namespace

namespace ms {
const MlpDev* surrogate_weights(const ms_surrogate* s) { return s ? s->mlp : nullptr; }
int surrogate_activation(const ms_surrogate* s) { return s ? s->act : MS_ACT_GELU; }
int surrogate_stride(const ms_surrogate* s) { return s ? s->stride : 1; }
}  // namespace ms

extern "C" {

int ms_surrogate_create(const float* params, ms_surrogate** out) {
  return ms_surrogate_create_ex(params, MS_ACT_GELU, 1, out);
}

int ms_surrogate_create_ex(const float* params, int32_t activation, int32_t stride,
                           ms_surrogate** out) {
  if (!params || !out) return ms::record_error(MS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (activation != MS_ACT_GELU && activation != MS_ACT_RELU)
    return ms::record_error(MS_ERR_INVALID_ARG, "activation must be MS_ACT_GELU or MS_ACT_RELU");
  if (stride < 1 || stride > ms::MLP_MAX_STRIDE || (stride & (stride - 1)) != 0)
    return ms::record_error(MS_ERR_INVALID_ARG, "stride must be 1, 2, 4, 8 or 16");
  for (int i = 0; i < ms::MLP_PARAMS; ++i)
    if (!std::isfinite(params[i])) return ms::record_error(MS_ERR_INVALID_ARG, "non-finite parameter");
  ms_surrogate* s = new (std::nothrow) ms_surrogate();
  if (!s) return ms::record_error(MS_ERR_OOM, "host allocation failed");
  s->act = activation;
  s->stride = stride;
  auto bail = [&](int rc) { ms_surrogate_destroy(s); return rc; };
  const size_t pb = ms::MLP_PARAMS * sizeof(float);
  if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess)
    return bail(ms::record_error(MS_ERR_CUDA, "stream creation failed"));
  s->stream = s->own;
  if (cudaMalloc(&s->params, pb) != cudaSuccess ||
      cudaMalloc(&s->m, pb) != cudaSuccess || cudaMalloc(&s->v, pb) != cudaSuccess ||
      cudaMalloc(&s->grad, pb) != cudaSuccess || cudaMalloc(&s->mlp, sizeof(MlpDev)) != cudaSuccess ||
      cudaMalloc(&s->loss, sizeof(double)) != cudaSuccess)
    return bail(ms::record_error(MS_ERR_OOM, "device allocation failed"));
  if (cudaMemcpy(s->params, params, pb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->m, 0, pb) != cudaSuccess || cudaMemset(s->v, 0, pb) != cudaSuccess)
    return bail(ms::record_error(MS_ERR_CUDA, "upload failed"));
  int rc = pack(s);
  if (rc != MS_OK) return bail(rc);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess)
    return bail(ms::record_error(MS_ERR_CUDA, "pack failed"));
  *out = s;
  return MS_OK;
}

void ms_surrogate_destroy(ms_surrogate* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  cudaFree(s->params);
  cudaFree(s->m);
  cudaFree(s->v);
  cudaFree(s->grad);
  cudaFree(s->mlp);
  cudaFree(s->loss);
  cudaFree(s->scratch);
  if (s->own) cudaStreamDestroy(s->own);
  delete s;
}

int ms_surrogate_set_stream(ms_surrogate* s, void* stream) {
  if (!s) return ms::record_error(MS_ERR_INVALID_ARG, "NULL surrogate");
  SG_CUDA(cudaStreamSynchronize(s->stream));
  s->stream = stream ? static_cast<cudaStream_t>(stream) : s->own;
  return MS_OK;
}

int ms_surrogate_get_config(const ms_surrogate* s, int32_t* activation, int32_t* stride) {
  if (!s || !activation || !stride) return ms::record_error(MS_ERR_INVALID_ARG, "NULL argument");
  *activation = s->act;
  *stride = s->stride;
  return MS_OK;
}

int ms_surrogate_get_params(ms_surrogate* s, float* params) {
  if (!s || !params) return ms::record_error(MS_ERR_INVALID_ARG, "NULL argument");
  SG_CUDA(cudaMemcpyAsync(params, s->params, ms::MLP_PARAMS * sizeof(float), cudaMemcpyDeviceToHost,
                          s->stream));
  SG_CUDA(cudaStreamSynchronize(s->stream));
  return MS_OK;
}

int ms_surrogate_forward(ms_surrogate* s, const float* x, float* y, int64_t n) {
  if (!s || !x || !y || n < 0) return ms::record_error(MS_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return MS_OK;
  const int64_t warps = (n + 127) / 128;
  if (s->act == MS_ACT_RELU)
    k_mlp_infer<ms::ACT_RELU><<<unsigned((warps + 3) / 4), 128, kInferSmem, s->stream>>>(s->mlp, x, y, n);
  else
    k_mlp_infer<ms::ACT_GELU><<<unsigned((warps + 3) / 4), 128, kInferSmem, s->stream>>>(s->mlp, x, y, n);
  SG_CUDA(cudaGetLastError());
  return MS_OK;
}

int ms_surrogate_gradient(ms_surrogate* s, const float* x, const float* t, int64_t n, float* grad,
                          double* loss) {
  if (!s || !x || !t || n <= 0) return ms::record_error(MS_ERR_INVALID_ARG, "bad argument");
  int rc = gradient(s, x, t, n);
  if (rc != MS_OK) return rc;
  if (grad)
    SG_CUDA(cudaMemcpyAsync(grad, s->grad, ms::MLP_PARAMS * sizeof(float), cudaMemcpyDeviceToDevice,
                            s->stream));
  if (loss) {
    SG_CUDA(cudaMemcpyAsync(loss, s->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SG_CUDA(cudaStreamSynchronize(s->stream));
  }
  return MS_OK;
}

int ms_surrogate_train_step(ms_surrogate* s, const float* x, const float* t, int64_t n, double lr,
                            double* loss) {
  if (!s || !x || !t || n <= 0 || !(lr > 0)) return ms::record_error(MS_ERR_INVALID_ARG, "bad argument");
  int rc = gradient(s, x, t, n);
  if (rc != MS_OK) return rc;
  s->step++;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = float(1.0 / (1.0 - std::pow(b1, double(s->step))));
  const float c2 = float(1.0 / (1.0 - std::pow(b2, double(s->step))));
  k_adam<<<(ms::MLP_PARAMS + 255) / 256, 256, 0, s->stream>>>(s->params, s->m, s->v, s->grad,
                                                                float(lr), float(b1), float(b2),
                                                                1e-8f, c1, c2);
  SG_CUDA(cudaGetLastError());
  if ((rc = pack(s)) != MS_OK) return rc;
  if (loss) {
    SG_CUDA(cudaMemcpyAsync(loss, s->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    SG_CUDA(cudaStreamSynchronize(s->stream));
  }
  return MS_OK;
}

}  // extern "C"
