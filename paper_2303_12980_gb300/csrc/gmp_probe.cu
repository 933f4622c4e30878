// Throughput probes (diagnostics): FP32 FMA (scalar and packed pairs) and
// SFU ex2 rates of the current device at its present clocks, so that the
// kernels can be reported against a measured ceiling next to the nominal
// one (SMs x 128 FP32 lanes x 2 FLOP x clock).
#include "gmp.h"
#include "gmp_internal.cuh"

#include <cstdio>

namespace {

constexpr int kChains = 8;

// kChains independent FMA chains per thread; the result is stored only under
// a condition that never holds, which keeps the chains live.
__global__ void k_probe_fma(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
  const float b = 0.9999f, c = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) out[threadIdx.x] = s;
}

// The same with packed FP32 pairs (two FMAs per instruction).
__global__ void k_probe_fma2(float* out, int iters) {
  float2 a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = make_float2(1.0f + 1e-3f * (float)(threadIdx.x + k), 1.0f);
  const float2 b = make_float2(0.9999f, 0.9998f), c = make_float2(1e-4f, 2e-4f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = gmp_fma2(a[k], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  if (s == -1.0f) out[threadIdx.x] = s;
}

// kChains independent ex2 chains per thread (x <- 2^x - 1.5 stays in
// (-1.5, 0.5)); one FP32 add per ex2 runs on the FMA pipe.
__global__ void k_probe_ex2(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = -0.5f - 1e-3f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __fadd_rn(gmp_ex2(a[k]), -1.5f);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 1e30f) out[threadIdx.x] = s;
}

}  // namespace

extern "C" gmp_status gmp_probe_peaks(int device, double* fma_tflops, double* fma2_tflops, double* ex2_tops) {
  if (!fma_tflops || !fma2_tflops || !ex2_tops) return GMP_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GMP_ERR_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return GMP_ERR_CUDA;
  }
  const int threads = 256;
  const int blocks = prop.multiProcessorCount * (prop.maxThreadsPerMultiProcessor / threads);
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gmp_status st = GMP_OK;
  if (cudaMalloc(&out, sizeof(float) * threads) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    st = GMP_ERR_CUDA;
  }
  // FLOP (or ex2) per launch and the measured rate
  auto run = [&](void (*fn)(float*, int), int iters, double ops_per_iter, double* rate) {
    if (st != GMP_OK) return;
    fn<<<blocks, threads>>>(out, iters / 8);  // warm-up and clock ramp
    cudaEventRecord(e0);
    fn<<<blocks, threads>>>(out, iters);
    cudaEventRecord(e1);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f) {
      cudaGetLastError();
      st = GMP_ERR_CUDA;
      return;
    }
    *rate = (double)blocks * threads * iters * ops_per_iter / (ms * 1e-3) / 1e12;
  };
  run(k_probe_fma, 1 << 14, 2.0 * kChains, fma_tflops);
  run(k_probe_fma2, 1 << 14, 4.0 * kChains, fma2_tflops);
  run(k_probe_ex2, 1 << 12, 1.0 * kChains, ex2_tops);
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}
