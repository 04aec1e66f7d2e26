// opf_fma_rate: the device's sustained FP64 or FP32 fused multiply-add rate,
// the denominator of the rooflines of the ALU-bound kernels (the radial
// solves and the FP64 transforms are bound by the FP64 rate, the mixed-
// precision transforms by the FP32 rate).  Every thread runs kChains
// independent FMA recurrences a <- a * b + c (|b| < 1, so the values stay
// bounded and normal), enough in flight per warp to hide the FMA latency;
// the grid covers every SM many times over.
#include <cuda_runtime.h>

#include <string>

#include "opf_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(int iters, T b, T c, T* out) {
  T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[blockIdx.x * kThreads + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
int run(int iters, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return OPF_ECUDA;
  const int blocks = sms * 16;
  T* out = nullptr;
  if (cudaMalloc((void**)&out, (size_t)blocks * kThreads * sizeof(T)) != cudaSuccess) return OPF_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T b = (T)0.999, c = (T)1e-4;
  k_fma_rate<T><<<blocks, kThreads>>>(iters / 8, b, c, out);  // warm-up
  cudaEventRecord(e0);
  k_fma_rate<T><<<blocks, kThreads>>>(iters, b, c, out);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || !(ms > 0.f)) return OPF_ECUDA;
  const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return OPF_OK;
}

}  // namespace

extern "C" int opf_fma_rate(int precision, double* tflops) {
  if (!tflops || (precision != 0 && precision != 1)) {
    opf::set_last_error("opf_fma_rate: precision 0 (FP64) or 1 (FP32) and a non-NULL output");
    return OPF_EINVAL;
  }
  const int rc = precision == 0 ? run<double>(4096, tflops) : run<float>(1 << 17, tflops);
  if (rc != OPF_OK) opf::set_last_error("opf_fma_rate: CUDA failure (" + std::to_string(rc) + ")");
  return rc;
}
