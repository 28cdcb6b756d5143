// The learned surrogate: a 12 -> 64 -> 64 -> 3 MLP with BF16 weights and FP32
// accumulation, advancing a point's fractions over a window of 8 r explicit
// steps (r = 1, 2, 4, 8 or 16, the surrogate's temperature stride).
//
// Inputs (12): X_as, X_am, X_beta at the window start, the temperatures of the
// window's levels r, 2 r, ..., 8 r as (T - 1000 K) / 1000 K, log10(dt) + 5.
// Outputs (3): 1e6 x the window's diffusive residual of X_as, X_am, X_beta:
// the fractions at the window end minus g(T_8r, G(start fractions)), G being
// the correction of Sec. 2.2 applied at the 8 sampled temperatures in turn.
//
// Parameter vector (FP32 master copy, 5187 values): W1[64][12], b1[64],
// W2[64][64], b2[64], W3[3][64], b3[3] (weights row-major, out x in).
// Inference layout (MlpDev): BF16 W1 [64][12] stored with a row stride of 24,
// W2 [64][64] with a stride of 72, W3 [3][64] as 8 rows of stride 72 (zero
// padding); FP32 biases.  The padded strides put the 8 rows a warp reads for
// one B fragment of mma.m16n8k16 in 8 different groups of 4 banks, so the
// fragment loads from shared memory are free of bank conflicts (a stride of
// 64 BF16 = 128 bytes would put all 8 rows in the same bank).
//
// Hidden activation: GELU in the tanh form
// 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) or ReLU max(x, 0), chosen
// when the surrogate is created.  Activations are rounded to BF16 between
// layers in both the training and the inference forward pass, so the two
// agree up to FP32 summation order.  ReLU and the BF16 rounding commute
// (rounding keeps the sign and maps 0 to 0), so the inference pass applies
// ReLU inside the conversion that packs two activations into a BF16 pair.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace ms {

constexpr int MLP_IN = 12, MLP_H = 64, MLP_OUT = 3;
constexpr int MLP_IN_PAD = 16, MLP_OUT_PAD = 8;
constexpr int MLP_W1_LD = 24, MLP_W2_LD = 72, MLP_W3_LD = 72;  // BF16 row strides
constexpr int MLP_X_LD = 24;   // row stride of the BF16 input tile [128][MLP_X_LD]
constexpr int MLP_Y_COLS = 4;  // FP32 output tile, column-major [MLP_Y_COLS][128]
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_IN;   // 768
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;            // 832
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;    // 4928
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;            // 4992
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_OUT * MLP_H;  // 5184
constexpr int MLP_PARAMS = MLP_OFF_B3 + MLP_OUT;          // 5187
constexpr int MLP_WINDOW = 8;                             // temperature samples per window
constexpr int MLP_MAX_STRIDE = 16;                        // levels between samples: 1, 2, 4, 8, 16
constexpr int ACT_GELU = 0, ACT_RELU = 1;                 // hidden activations

constexpr float MLP_T_SHIFT = 1000.0f, MLP_T_SCALE = 1.0e-3f;
constexpr float MLP_DT_SHIFT = 5.0f, MLP_OUT_SCALE = 1.0e6f;

struct MlpDev {
  __nv_bfloat16 w1[MLP_H * MLP_W1_LD];
  __nv_bfloat16 w2[MLP_H * MLP_W2_LD];
  __nv_bfloat16 w3[MLP_OUT_PAD * MLP_W3_LD];
  float b1[MLP_H];
  float b2[MLP_H];
  float b3[MLP_OUT_PAD];
};

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float GELU_C = 0.7978845608028654f;  // sqrt(2 / pi)
constexpr float GELU_A = 0.044715f;

__device__ __forceinline__ float gelu(float x) {
  const float u = GELU_C * fmaf(GELU_A * x, x * x, x);
  return 0.5f * x * (1.0f + tanh_approx(u));
}

__device__ __forceinline__ float gelu_grad(float x) {
  const float u = GELU_C * fmaf(GELU_A * x, x * x, x);
  const float th = tanh_approx(u);
  return 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * GELU_C * fmaf(3.0f * GELU_A, x * x, 1.0f);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <int ACT>
__device__ __forceinline__ float act(float x) {
  if constexpr (ACT == ACT_RELU) return fmaxf(x, 0.0f);
  else return gelu(x);
}

// derivative of the activation at the pre-activation x (ReLU: 0 at x = 0)
template <int ACT>
__device__ __forceinline__ float act_grad(float x) {
  if constexpr (ACT == ACT_RELU) return x > 0.0f ? 1.0f : 0.0f;
  else return gelu_grad(x);
}

// The activations of two pre-activations packed as a BF16 pair (lo in the
// low half).  ReLU: one round-to-nearest conversion with the .relu clamp.
template <int ACT>
__device__ __forceinline__ uint32_t pack_act(float lo, float hi) {
  if constexpr (ACT == ACT_RELU) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
  } else {
    return pack_bf16(gelu(lo), gelu(hi));
  }
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + C, FP32 accumulate.
__device__ __forceinline__ void mma_bf16_16816(float* d, const uint32_t* a, uint32_t b0,
                                               uint32_t b1, const float* c) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%11,%12,%13};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]),
        "f"(c[2]), "f"(c[3]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// Four 8x8 BF16 matrices from shared memory (ldmatrix): lane i gives the
// address of row i % 8 of matrix i / 8 (16 contiguous bytes, 16-byte
// aligned); r[j] of lane l holds row l / 4, columns 2 (l % 4) and
// 2 (l % 4) + 1 of matrix j, i.e. one mma.m16n8k16 A or B fragment register.
__device__ __forceinline__ void ldsm_x4(const void* row_addr, uint32_t* r) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(row_addr));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a)
               : "memory");
}

__device__ __forceinline__ float2 ld_f2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// Forward pass of one warp over 128 samples with tensor cores.  X: the
// warp's [128][MLP_X_LD] BF16 inputs (features 12..15 zero) and Y: its FP32
// outputs, column-major [MLP_Y_COLS][128] (output c of row r at Y[c * 128 + r],
// columns 0..2 meaningful), both in shared memory; W: the weights (shared
// memory).  Rows are processed in 8 tiles of 16; each layer's accumulator
// fragments are repacked in registers as the next layer's A fragments, and
// the input and weight fragments come four at a time with ldmatrix.  Row
// tile mt is computed only if bit mt of mt_mask (warp-uniform) is set.
template <int ACT>
__device__ __forceinline__ void mlp_forward_warp(const MlpDev& W, const __nv_bfloat16* X, float* Y,
                                                 int lane, uint32_t mt_mask = 0xffu) {
  const int g = lane >> 2, q = lane & 3;
  const int r8 = lane & 7, m4 = lane >> 3;   // ldmatrix: row of the matrix, matrix
#pragma unroll 1
  for (int mt = 0; mt < 8; ++mt) {
    if (!((mt_mask >> mt) & 1u)) continue;
    const int ra = mt * 16 + g, rb = ra + 8;
    // A: rows 0-7 / 8-15 of the tile, features 0-7 / 8-15
    uint32_t a[4];
    ldsm_x4(X + (mt * 16 + r8 + 8 * (m4 & 1)) * MLP_X_LD + 8 * (m4 >> 1), a);
    float h[8][4];
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      // B of n-tiles t and t + 1: W1 rows 8 t .. 8 t + 15, features 0-7 / 8-15
      uint32_t b[4];
      ldsm_x4(W.w1 + (8 * t + r8 + 8 * (m4 >> 1)) * MLP_W1_LD + 8 * (m4 & 1), b);
      const float2 c0 = ld_f2(W.b1 + 8 * t + 2 * q), c1 = ld_f2(W.b1 + 8 * t + 8 + 2 * q);
      const float cc0[4] = {c0.x, c0.y, c0.x, c0.y}, cc1[4] = {c1.x, c1.y, c1.x, c1.y};
      mma_bf16_16816(h[t], a, b[0], b[1], cc0);
      mma_bf16_16816(h[t + 1], a, b[2], b[3], cc1);
    }
    uint32_t a2[4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      a2[kc][0] = pack_act<ACT>(h[2 * kc][0], h[2 * kc][1]);
      a2[kc][1] = pack_act<ACT>(h[2 * kc][2], h[2 * kc][3]);
      a2[kc][2] = pack_act<ACT>(h[2 * kc + 1][0], h[2 * kc + 1][1]);
      a2[kc][3] = pack_act<ACT>(h[2 * kc + 1][2], h[2 * kc + 1][3]);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const float2 c = ld_f2(W.b2 + 8 * t + 2 * q);
      h[t][0] = h[t][2] = c.x;
      h[t][1] = h[t][3] = c.y;
      const __nv_bfloat16* wr = W.w2 + (8 * t + r8) * MLP_W2_LD + 8 * m4;
#pragma unroll
      for (int kc = 0; kc < 4; kc += 2) {
        // B of k-chunks kc and kc + 1: W2 rows 8 t .. 8 t + 7, 32 inputs
        uint32_t b[4];
        ldsm_x4(wr + 16 * kc, b);
        mma_bf16_16816(h[t], a2[kc], b[0], b[1], h[t]);
        mma_bf16_16816(h[t], a2[kc + 1], b[2], b[3], h[t]);
      }
    }
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      a2[kc][0] = pack_act<ACT>(h[2 * kc][0], h[2 * kc][1]);
      a2[kc][1] = pack_act<ACT>(h[2 * kc][2], h[2 * kc][3]);
      a2[kc][2] = pack_act<ACT>(h[2 * kc + 1][0], h[2 * kc + 1][1]);
      a2[kc][3] = pack_act<ACT>(h[2 * kc + 1][2], h[2 * kc + 1][3]);
    }
    const float2 c3 = ld_f2(W.b3 + 2 * q);
    float y[4] = {c3.x, c3.y, c3.x, c3.y};
    const __nv_bfloat16* wr = W.w3 + r8 * MLP_W3_LD + 8 * m4;
#pragma unroll
    for (int kc = 0; kc < 4; kc += 2) {
      uint32_t b[4];
      ldsm_x4(wr + 16 * kc, b);
      mma_bf16_16816(y, a2[kc], b[0], b[1], y);
      mma_bf16_16816(y, a2[kc + 1], b[2], b[3], y);
    }
    if (q < 2) {  // output columns 0..3 (3 is padding)
      Y[(2 * q) * 128 + ra] = y[0];
      Y[(2 * q + 1) * 128 + ra] = y[1];
      Y[(2 * q) * 128 + rb] = y[2];
      Y[(2 * q + 1) * 128 + rb] = y[3];
    }
  }
}

}  // namespace ms
