// Device probes of the benchmark (uh_debug.h): the FP64 fused multiply-add rate.
#include <cuda_runtime.h>

#include "uh.h"
#include "uh_debug.h"
#include "uh_internal.h"

namespace {

// 8 independent chains per thread so that the FMA pipe, not the dependency latency, bounds the
// rate; the result is stored so the chains are not removed.
__global__ void dfma_kernel(int iters, double* sink) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  const double m = 0.999999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.6789) sink[blockIdx.x] = s;  // practically never: keeps the chains alive
}

}  // namespace

extern "C" int uh_debug_dfma_rate(int32_t iters, double* tflops, void* stream) {
  if (iters < 1000 || !tflops) return uh::set_error(UH_EINVAL, "uh_debug_dfma_rate: iters %d, tflops %p", iters,
                                                    static_cast<void*>(tflops));
  int dev = 0, sms = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = 4 * sms, block = 256;
  if (e == cudaSuccess) e = cudaMalloc(&sink, static_cast<size_t>(grid) * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  if (e == cudaSuccess) {
    dfma_kernel<<<grid, block, 0, st>>>(iters / 10, sink);  // warm-up
    cudaEventRecord(e0, st);
    dfma_kernel<<<grid, block, 0, st>>>(iters, sink);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return uh::set_error(UH_ECUDA, "uh_debug_dfma_rate: %s", cudaGetErrorString(e));
  const double fmas = static_cast<double>(grid) * block * 8.0 * iters;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return UH_OK;
}
