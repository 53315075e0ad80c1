// Device capability probe: the FP64 FMA rate of the current GPU, the ceiling of
// the FP64 evaluation mode (its kernels are bound by DFMA issue on GB300).
#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace {

__global__ void __launch_bounds__(256) k_dfma_loop(double* out, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = threadIdx.x + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" hmat_status hmat_measure_fp64_peak(double* gflops) {
  if (!gflops) return HMAT_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HMAT_ECUDA;
  const int blocks = sms * 4, threads = 256, iters = 1 << 13;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hmat_status st = HMAT_ECUDA;
  float ms = 0.0f;
  if (cudaMalloc((void**)&out, sizeof(double) * blocks * threads) != cudaSuccess) return HMAT_ENOMEM;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    k_dfma_loop<<<blocks, threads>>>(out, 64, 1.0000001, 1e-9);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0);
      k_dfma_loop<<<blocks, threads>>>(out, iters, 1.0000001, 1e-9);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) break;
      best = ms < best ? ms : best;
      if (r == 2) st = HMAT_OK;
    }
    ms = best;
  }
  if (cudaGetLastError() != cudaSuccess) st = HMAT_ECUDA;
  if (st == HMAT_OK) *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e6);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}
