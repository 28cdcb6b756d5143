// The learned surrogate's object, training kernels and batched inference.
//
//  k_mlp_pack     FP32 master parameters -> BF16-rounded FP32 copy (training
//                 forward) and the padded BF16 inference layout (MlpDev).
//  k_mlp_fwd_bwd  one thread per sample: forward with the BF16-rounded
//                 weights and activations, FP32 accumulation, MSE loss, and
//                 the backward pass to the pre-activation gradients, stored
//                 feature-major for the weight-gradient reduction.
//  k_mlp_wgrad    one warp per parameter: dW = sum over the batch of
//                 (upstream gradient x activation).
//  k_adam         Adam on the FP32 master copy, then repack.
//  k_mlp_infer    batched inference on the tensor cores (mma.sync bf16,
//                 FP32 accumulation), 128 samples per warp.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "ms_internal.h"
#include "ms_mlp.cuh"

using ms::MlpDev;

struct ms_surrogate {
  float* params = nullptr;   // FP32 master copy
  float* wr = nullptr;       // BF16-rounded FP32 copy used by the training forward
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  MlpDev* mlp = nullptr;     // inference layout
  double* loss = nullptr;
  float* scratch = nullptr;  // per-sample activations and gradients
  size_t scratch_cap = 0;    // samples
  int64_t step = 0;
  cudaStream_t own = nullptr, stream = nullptr;
};

namespace {

constexpr int kScratchPerSample = ms::MLP_IN + 4 * ms::MLP_H + ms::MLP_OUT;  // xs, a1, a2, dh1, dh2, dy

#define SG_CUDA(...)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                  \
    if (e_ != cudaSuccess) return ms::record_error(e_ == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

__global__ void k_mlp_pack(const float* p, float* wr, MlpDev* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ms::MLP_PARAMS) wr[i] = ms::bf16r(p[i]);
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

// Per-sample forward and backward.  Scratch layout (feature-major, n
// samples): xs[12][n], a1[64][n], a2[64][n], dh1[64][n], dh2[64][n], dy[3][n].
__global__ void __launch_bounds__(128) k_mlp_fwd_bwd(const float* __restrict__ wr,
                                                     const float* __restrict__ x,
                                                     const float* __restrict__ t, int64_t n,
                                                     float* __restrict__ sc, double* loss) {
  extern __shared__ float W[];  // MLP_PARAMS
  for (int i = threadIdx.x; i < ms::MLP_PARAMS; i += blockDim.x) W[i] = wr[i];
  __syncthreads();
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double lsum = 0.0;
  if (s < n) {
    const float* W1 = W + ms::MLP_OFF_W1; const float* B1 = W + ms::MLP_OFF_B1;
    const float* W2 = W + ms::MLP_OFF_W2; const float* B2 = W + ms::MLP_OFF_B2;
    const float* W3 = W + ms::MLP_OFF_W3; const float* B3 = W + ms::MLP_OFF_B3;
    float* xs = sc;
    float* a1s = xs + int64_t(ms::MLP_IN) * n;
    float* a2s = a1s + int64_t(ms::MLP_H) * n;
    float* dh1s = a2s + int64_t(ms::MLP_H) * n;
    float* dh2s = dh1s + int64_t(ms::MLP_H) * n;
    float* dys = dh2s + int64_t(ms::MLP_H) * n;
    float xv[ms::MLP_IN], h1[ms::MLP_H], a1[ms::MLP_H], h2[ms::MLP_H], a2[ms::MLP_H];
    for (int k = 0; k < ms::MLP_IN; ++k) {
      xv[k] = ms::bf16r(x[s * ms::MLP_IN + k]);
      xs[k * n + s] = xv[k];
    }
    for (int j = 0; j < ms::MLP_H; ++j) {
      float acc = B1[j];
      for (int k = 0; k < ms::MLP_IN; ++k) acc = fmaf(W1[j * ms::MLP_IN + k], xv[k], acc);
      h1[j] = acc;
      a1[j] = ms::bf16r(ms::gelu(acc));
      a1s[j * n + s] = a1[j];
    }
    for (int j = 0; j < ms::MLP_H; ++j) {
      float acc = B2[j];
      for (int k = 0; k < ms::MLP_H; ++k) acc = fmaf(W2[j * ms::MLP_H + k], a1[k], acc);
      h2[j] = acc;
      a2[j] = ms::bf16r(ms::gelu(acc));
      a2s[j * n + s] = a2[j];
    }
    float dy[ms::MLP_OUT];
    const float inv = 1.0f / float(3 * n);
    for (int i = 0; i < ms::MLP_OUT; ++i) {
      float acc = B3[i];
      for (int k = 0; k < ms::MLP_H; ++k) acc = fmaf(W3[i * ms::MLP_H + k], a2[k], acc);
      const float r = acc - t[s * ms::MLP_OUT + i];
      lsum += double(r) * double(r) * double(inv);
      dy[i] = 2.0f * r * inv;
      dys[i * n + s] = dy[i];
    }
    // h2 now holds dL/dh2
    for (int k = 0; k < ms::MLP_H; ++k) {
      float da = 0.0f;
      for (int i = 0; i < ms::MLP_OUT; ++i) da = fmaf(dy[i], W3[i * ms::MLP_H + k], da);
      h2[k] = da * ms::gelu_grad(h2[k]);
      dh2s[k * n + s] = h2[k];
    }
    for (int k = 0; k < ms::MLP_H; ++k) {
      float da = 0.0f;
      for (int j = 0; j < ms::MLP_H; ++j) da = fmaf(h2[j], W2[j * ms::MLP_H + k], da);
      dh1s[k * n + s] = da * ms::gelu_grad(h1[k]);
    }
  }
  // block reduction of the loss
  __shared__ double red[128];
  red[threadIdx.x] = lsum;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (int(threadIdx.x) < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// grad[p] for every parameter: one warp per parameter, lanes stride the batch.
__global__ void k_mlp_wgrad(const float* __restrict__ sc, int64_t n, float* __restrict__ grad) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= ms::MLP_PARAMS) return;
  const float* xs = sc;
  const float* a1s = xs + int64_t(ms::MLP_IN) * n;
  const float* a2s = a1s + int64_t(ms::MLP_H) * n;
  const float* dh1s = a2s + int64_t(ms::MLP_H) * n;
  const float* dh2s = dh1s + int64_t(ms::MLP_H) * n;
  const float* dys = dh2s + int64_t(ms::MLP_H) * n;
  const float* up;
  const float* act = nullptr;
  if (p < ms::MLP_OFF_B1) {
    up = dh1s + (p / ms::MLP_IN) * n;
    act = xs + (p % ms::MLP_IN) * n;
  } else if (p < ms::MLP_OFF_W2) {
    up = dh1s + (p - ms::MLP_OFF_B1) * n;
  } else if (p < ms::MLP_OFF_B2) {
    const int q = p - ms::MLP_OFF_W2;
    up = dh2s + (q / ms::MLP_H) * n;
    act = a1s + (q % ms::MLP_H) * n;
  } else if (p < ms::MLP_OFF_W3) {
    up = dh2s + (p - ms::MLP_OFF_B2) * n;
  } else if (p < ms::MLP_OFF_B3) {
    const int q = p - ms::MLP_OFF_W3;
    up = dys + (q / ms::MLP_H) * n;
    act = a2s + (q % ms::MLP_H) * n;
  } else {
    up = dys + (p - ms::MLP_OFF_B3) * n;
  }
  float acc = 0.0f;
  for (int64_t s = lane; s < n; s += 32) acc = fmaf(up[s], act ? act[s] : 1.0f, acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) grad[p] = acc;
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
  ms::mlp_forward_warp(W, X, Y, lane);
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
  k_mlp_pack<<<(ms::MLP_PARAMS + 255) / 256, 256, 0, s->stream>>>(s->params, s->wr, s->mlp);
  SG_CUDA(cudaGetLastError());
  return MS_OK;
}

int gradient(ms_surrogate* s, const float* x, const float* t, int64_t n) {
  if (size_t(n) > s->scratch_cap) {
    SG_CUDA(cudaStreamSynchronize(s->stream));
    cudaFree(s->scratch);
    s->scratch = nullptr;
    s->scratch_cap = 0;
    SG_CUDA(cudaMalloc(&s->scratch, size_t(n) * kScratchPerSample * sizeof(float)));
    s->scratch_cap = size_t(n);
  }
  SG_CUDA(cudaMemsetAsync(s->loss, 0, sizeof(double), s->stream));
  const size_t sm = ms::MLP_PARAMS * sizeof(float);
  k_mlp_fwd_bwd<<<unsigned((n + 127) / 128), 128, sm, s->stream>>>(s->wr, x, t, n, s->scratch, s->loss);
  SG_CUDA(cudaGetLastError());
  k_mlp_wgrad<<<(ms::MLP_PARAMS * 32 + 255) / 256, 256, 0, s->stream>>>(s->scratch, n, s->grad);
  SG_CUDA(cudaGetLastError());
  return MS_OK;
}

}  // namespace

namespace ms {
const MlpDev* surrogate_weights(const ms_surrogate* s) { return s ? s->mlp : nullptr; }
}  // namespace ms

extern "C" {

int ms_surrogate_create(const float* params, ms_surrogate** out) {
  if (!params || !out) return ms::record_error(MS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  for (int i = 0; i < ms::MLP_PARAMS; ++i)
    if (!std::isfinite(params[i])) return ms::record_error(MS_ERR_INVALID_ARG, "non-finite parameter");
  ms_surrogate* s = new (std::nothrow) ms_surrogate();
  if (!s) return ms::record_error(MS_ERR_OOM, "host allocation failed");
  auto bail = [&](int rc) { ms_surrogate_destroy(s); return rc; };
  const size_t pb = ms::MLP_PARAMS * sizeof(float);
  if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess)
    return bail(ms::record_error(MS_ERR_CUDA, "stream creation failed"));
  s->stream = s->own;
  if (cudaMalloc(&s->params, pb) != cudaSuccess || cudaMalloc(&s->wr, pb) != cudaSuccess ||
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
  cudaFree(s->wr);
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
  k_mlp_infer<<<unsigned((warps + 3) / 4), 128, kInferSmem, s->stream>>>(s->mlp, x, y, n);
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
