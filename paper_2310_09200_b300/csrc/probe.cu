// probe.cu — measured rates for the rooflines: bipp_ss_measure_sincos_rate,
// the SFU rate that bounds the on-the-fly phase generation of the synthesis
// (Algorithm 2 "GEMMEXP" evaluates exp(j theta) for every pixel-station pair;
// Sec. 2.9 counts that work as N_pix N_st per step), and
// bipp_ss_measure_fma_rates, the FP32 and FP64 FMA rates that bound the
// eigensolve (Sec. 2.3) on the CUDA cores.
//
// Every thread runs kChains independent chains of __sincosf (the fast
// intrinsic the synthesis kernels use), each result feeding the next argument
// through one FMA, so the special-function unit is the only pipe near its
// limit: one sine and one cosine result per pair, an FMA and an FMUL beside
// them on the FP32 pipe (128 lanes per SM per clock against the SFU's 16).
#include <stdio.h>

#include "bipp_internal.cuh"
#include "bipp_ss.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__global__ void __launch_bounds__(kThreads) k_sincos_rate(float* out, float seed) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = seed * (float)(threadIdx.x + 1) + 0.1f * (float)k;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float s, c;
      __sincosf(x[k], &s, &c);
      x[k] = fmaf(c, 0.75f, s);  // stays in [-1.25, 1.25]: a well-scaled argument every time
    }
  }
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps every chain live
}

// Independent FMA chains in FP32 or FP64 (the CUDA-core pipes that bound the
// eigensolver's FP32 stage, its double-float products and the FP64 Jacobi).
template <typename R, int ITERS>
__global__ void __launch_bounds__(kThreads) k_fma_rate(R* out, R seed) {
  R x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = seed * (R)(threadIdx.x + 1) + (R)0.01 * (R)k;
  const R a = (R)0.999, c = (R)0.001;
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, c);  // converges to 1: stays finite
  }
  R acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// Best-of-`repeats` time of `launch` (after one warm-up launch) on a fresh stream; < 0 on failure.
template <typename F>
float best_ms(int repeats, F&& launch) {
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = -1.f;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess) {
    launch(s);
    for (int r = 0; r < repeats; ++r) {
      float ms = 0.f;
      cudaEventRecord(e0, s);
      launch(s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        best = -1.f;
        break;
      }
      if (best < 0.f || ms < best) best = ms;
    }
    if (cudaGetLastError() != cudaSuccess) best = -1.f;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return best;
}

}  // namespace

extern "C" int bipp_ss_measure_fma_rates(int32_t device, int32_t repeats, double* fp32_flops, double* fp64_flops) {
  if (!fp32_flops || !fp64_flops || repeats < 1 || repeats > 100)
    return bipp::set_global_error(BIPP_ERR_INVALID_ARG, "need fp32_flops, fp64_flops and 1 <= repeats <= 100");
  *fp32_flops = *fp64_flops = 0.0;
  int dev = device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess)
    return bipp::set_global_error(BIPP_ERR_CUDA, "cudaGetDevice failed");
  int n_sm = 0;
  if (cudaSetDevice(dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1)
    return bipp::set_global_error(BIPP_ERR_CUDA, "cannot select the device or read its SM count");
  const int blocks = n_sm * kBlocksPerSm;
  constexpr int kIt32 = 8192, kIt64 = 256;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * kThreads) != cudaSuccess) {
    (void)cudaGetLastError();
    return bipp::set_global_error(BIPP_ERR_OUT_OF_MEMORY, "probe output buffer");
  }
  const float ms32 = best_ms(repeats, [&](cudaStream_t s) {
    k_fma_rate<float, kIt32><<<blocks, kThreads, 0, s>>>(reinterpret_cast<float*>(out), 1e-3f);
  });
  const float ms64 = best_ms(repeats, [&](cudaStream_t s) {
    k_fma_rate<double, kIt64><<<blocks, kThreads, 0, s>>>(out, 1e-3);
  });
  cudaFree(out);
  if (ms32 <= 0.f || ms64 <= 0.f) return bipp::set_global_error(BIPP_ERR_CUDA, "probe launch failed");
  const double lanes = (double)blocks * kThreads * kChains;
  *fp32_flops = 2.0 * lanes * kIt32 / (ms32 * 1e-3);
  *fp64_flops = 2.0 * lanes * kIt64 / (ms64 * 1e-3);
  return BIPP_OK;
}

extern "C" int bipp_ss_measure_sincos_rate(int32_t device, int32_t repeats, double* pairs_per_s) {
  if (!pairs_per_s || repeats < 1 || repeats > 100)
    return bipp::set_global_error(BIPP_ERR_INVALID_ARG, "need pairs_per_s and 1 <= repeats <= 100");
  *pairs_per_s = 0.0;
  int dev = device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess)
    return bipp::set_global_error(BIPP_ERR_CUDA, "cudaGetDevice failed");
  int n_sm = 0;
  if (cudaSetDevice(dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1)
    return bipp::set_global_error(BIPP_ERR_CUDA, "cannot select the device or read its SM count");
  const int blocks = n_sm * kBlocksPerSm;
  float* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BIPP_OK;
  if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess) {
    (void)cudaGetLastError();
    return bipp::set_global_error(BIPP_ERR_OUT_OF_MEMORY, "probe output buffer");
  }
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = bipp::set_global_error(BIPP_ERR_CUDA, "stream/event creation failed");
  } else {
    k_sincos_rate<<<blocks, kThreads, 0, s>>>(out, 1e-3f);  // warm-up (clocks, instruction cache)
    float best_ms = 0.f;
    for (int r = 0; r < repeats && rc == BIPP_OK; ++r) {
      float ms = 0.f;
      cudaEventRecord(e0, s);
      k_sincos_rate<<<blocks, kThreads, 0, s>>>(out, 1e-3f * (float)(r + 2));
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = bipp::set_global_error(BIPP_ERR_CUDA, "probe launch failed");
        break;
      }
      if (r == 0 || ms < best_ms) best_ms = ms;
    }
    if (rc == BIPP_OK && cudaGetLastError() != cudaSuccess) rc = bipp::set_global_error(BIPP_ERR_CUDA, "probe");
    if (rc == BIPP_OK) {
      const double pairs = (double)blocks * kThreads * kIters * kChains;
      *pairs_per_s = pairs / (best_ms * 1e-3);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  return rc;
}
