// Throughput probes of the SM pipes the hot kernel leans on (the SFU for
// ex2 / lg2 / rsqrt / rcp, and FFMA for reference).  Each thread runs 8
// independent chains so the pipe, not the latency, limits the rate.  Inputs
// stay bounded without extra instructions (negation / absolute-value operand
// modifiers), so every issued instruction in the loop body is the probed one.
#include <cuda_runtime.h>

#include <cstdint>

#include "ms_internal.h"

namespace ms {
namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float op_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  return y;
}
__device__ __forceinline__ float op_lg2(float x) {
  float y;
  asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(fabsf(x)));
  return y;
}
__device__ __forceinline__ float op_rsqrt(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(fabsf(x)));
  return y;
}
// rcp alternates with rsqrt (a chain of reciprocals alone returns to its
// start every second step); the rcp rate follows from the mixed rate and the
// rsqrt probe.
__device__ __forceinline__ float op_rcp(float x) {
  float y, z;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(z) : "f"(fabsf(y)));
  return z;
}
__device__ __forceinline__ float op_ffma(float x) {
  float y;
  asm volatile("fma.rn.f32 %0, %1, 0f3F000000, 0f3E800000;" : "=f"(y) : "f"(x));
  return y;
}

template <int OP>
__global__ void k_probe(int iters, float seed, float* sink, unsigned long long* cyc,
                        unsigned long long* ns) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed + 0.01f * c + 1e-6f * threadIdx.x;
  unsigned long long c0 = 0, t0 = 0;
  if (threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if (OP == 0) v[c] = op_ex2(v[c]);
        if (OP == 1) v[c] = op_lg2(v[c]);
        if (OP == 2) v[c] = op_rsqrt(v[c]);
        if (OP == 3) v[c] = op_rcp(v[c]);
        if (OP == 4) v[c] = op_ffma(v[c]);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == 12345.678f) sink[threadIdx.x] = s;  // keep the chains alive
  if (threadIdx.x == 0) {
    unsigned long long c1 = clock64(), t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    atomicAdd(cyc, c1 - c0);
    atomicAdd(ns, t1 - t0);
  }
}

template <int OP>
cudaError_t run_probe(int blocks, int threads, int iters, float* sink, unsigned long long* acc,
                      cudaStream_t s) {
  k_probe<OP><<<blocks, threads, 0, s>>>(iters, 0.5f, sink, acc, acc + 1);
  return cudaGetLastError();
}

}  // namespace
}  // namespace ms

extern "C" int ms_probe_sfu(int op, double* ops_per_s, double* sm_mhz) {
  if (op < 0 || op > 4 || !ops_per_s) return MS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MS_ERR_CUDA;
  const int threads = 256, blocks = sms * 8, iters = 2048;
  float* sink = nullptr;
  unsigned long long* acc = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MS_OK;
  if (cudaMalloc(&sink, threads * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&acc, 2 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MS_ERR_CUDA;
  }
  float best = 1e30f;
  unsigned long long host[2] = {0, 0};
  for (int rep = 0; rc == MS_OK && rep < 4; ++rep) {
    cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), s);
    cudaEventRecord(e0, s);
    cudaError_t e;
    switch (op) {
      case 0: e = ms::run_probe<0>(blocks, threads, iters, sink, acc, s); break;
      case 1: e = ms::run_probe<1>(blocks, threads, iters, sink, acc, s); break;
      case 2: e = ms::run_probe<2>(blocks, threads, iters, sink, acc, s); break;
      case 3: e = ms::run_probe<3>(blocks, threads, iters, sink, acc, s); break;
      default: e = ms::run_probe<4>(blocks, threads, iters, sink, acc, s); break;
    }
    cudaEventRecord(e1, s);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = MS_ERR_CUDA;
      break;
    }
    float ms_ = 0.f;
    cudaEventElapsedTime(&ms_, e0, e1);
    if (rep > 0 && ms_ < best) {
      best = ms_;
      cudaMemcpy(host, acc, sizeof(host), cudaMemcpyDeviceToHost);
    }
  }
  if (rc == MS_OK) {
    const double ops = double(blocks) * threads * iters * 8.0 * ms::kChains * (op == 3 ? 2.0 : 1.0);
    *ops_per_s = ops / (best * 1e-3);
    if (sm_mhz) *sm_mhz = host[1] ? double(host[0]) / double(host[1]) * 1e3 : 0.0;
  }
  cudaFree(sink);
  cudaFree(acc);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return rc;
}

// ------------------------------------------------ transcendentals, evaluated
namespace ms {
namespace {

__global__ void k_eval_transcendental(int which, const float* x, float* y, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = x[i];
  y[i] = which == 0 ? fma_ex2(v) : which == 1 ? fma_lg2(v) : which == 2 ? sfu_ex2(v) : sfu_lg2(v);
}

}  // namespace
}  // namespace ms

extern "C" int ms_eval_transcendental(int which, const float* x, float* y, int64_t n) {
  if (which < 0 || which > 3 || !x || !y || n < 0)
    return ms::record_error(MS_ERR_INVALID_ARG, "which must be 0..3, x and y non-NULL, n >= 0");
  if (n == 0) return MS_OK;
  float* d = nullptr;
  if (cudaMalloc(&d, size_t(n) * 2 * sizeof(float)) != cudaSuccess)
    return ms::record_error(MS_ERR_OOM, "device allocation failed");
  cudaError_t e = cudaMemcpy(d, x, size_t(n) * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    ms::k_eval_transcendental<<<unsigned((n + 255) / 256), 256>>>(which, d, d + n, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(y, d + n, size_t(n) * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return ms::record_error(MS_ERR_CUDA, cudaGetErrorString(e));
  return MS_OK;
}
