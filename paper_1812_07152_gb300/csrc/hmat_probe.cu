// Device probes: the FP64 FMA rate of the current GPU, the ceiling of the FP64
// evaluation mode (its kernels are bound by DFMA issue on GB300), and a bitwise check
// of the integer-unit FP32 <-> FP64 conversions of the mixed mode against the
// hardware's.
#include <cuda_runtime.h>

#include "hmat_fp.cuh"
#include "hmat_internal.h"

using namespace hmat;

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Sample i: the first ones special values (signed zeros, infinities, NaN, the ends of
// the normal and subnormal ranges), then random bit patterns (every exponent class),
// every fourth double with its 29 low bits at the rounding tie of the narrowing.
__constant__ uint64_t kSpecial64[] = {0x0ull, 0x8000000000000000ull, 0x7FF0000000000000ull, 0xFFF0000000000000ull,
                                      0x7FF8000000000000ull, 0x3810000000000000ull, 0x380FFFFFFFFFFFFFull,
                                      0x47EFFFFFE0000000ull, 0x47EFFFFFF0000000ull, 0x0000000000000001ull,
                                      0x3FF0000010000000ull, 0x3FF0000030000000ull};
__constant__ uint32_t kSpecial32[] = {0x0u, 0x80000000u, 0x7F800000u, 0xFF800000u, 0x7FC00000u, 0x00800000u,
                                      0x007FFFFFu, 0x7F7FFFFFu, 0x00000001u, 0x3F800000u, 0x80800000u, 0x807FFFFFu};
constexpr int kSpecials = 12;

__global__ void __launch_bounds__(256) k_conv_check(int64_t n, uint64_t seed, unsigned long long* bad) {
  unsigned long long b_w = 0, b_n = 0, b_s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r1 = splitmix64(seed ^ (2 * (uint64_t)i)), r2 = splitmix64(seed ^ (2 * (uint64_t)i + 1));
    if (i < kSpecials * kSpecials) {
      r1 = kSpecial64[i / kSpecials];
      r2 = (r2 & 0xFFFFFFFF00000000ull) | kSpecial32[i % kSpecials];
    }
    const uint64_t bits = (i & 3) == 0 && i >= kSpecials * kSpecials ? ((r1 & ~0x1FFFFFFFull) | 0x10000000ull) : r1;
    const double d = __longlong_as_double((long long)bits);
    const float f = __uint_as_float((uint32_t)r2);
    const int e = (int)((r2 >> 32) % 601) - 300;
    const double sc = ldexp(1.0, e);
    const double w1 = (double)f;
    const float n1 = __double2float_rn(d);
    const double s1 = d * sc;
    const double w0 = widen_f32<false>(f), w0o = widen_f32<true>(f);
    const float n0 = narrow_f64<false>(d), n0o = narrow_f64<true>(d);
    const double s0 = scale_pow2<false>(d, e, sc), s0o = scale_pow2<true>(d, e, sc);
    auto same_d = [](double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b); };
    auto same_f = [](float a, float b) { return __float_as_uint(a) == __float_as_uint(b) || (a != a && b != b); };
    b_w += !same_d(w0, w1) + !same_d(w0o, w1);
    b_n += !same_f(n0, n1) + !same_f(n0o, n1);
    b_s += !same_d(s0, s1) + !same_d(s0o, s1);
  }
  if (b_w) atomicAdd(bad, b_w);
  if (b_n) atomicAdd(bad + 1, b_n);
  if (b_s) atomicAdd(bad + 2, b_s);
}

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

extern "C" hmat_status hmat_selftest_conversions(int64_t n, uint64_t seed, int64_t* mismatches) {
  if (!mismatches || n < 0) return HMAT_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HMAT_ECUDA;
  unsigned long long* bad = nullptr;
  if (cudaMalloc((void**)&bad, 3 * sizeof(unsigned long long)) != cudaSuccess) return HMAT_ENOMEM;
  unsigned long long host[3] = {0, 0, 0};
  cudaError_t e = cudaMemset(bad, 0, 3 * sizeof(unsigned long long));
  if (e == cudaSuccess && n > 0) {
    k_conv_check<<<sms * 8, 256>>>(n, seed, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(host, bad, sizeof(host), cudaMemcpyDeviceToHost);
  cudaFree(bad);
  if (e != cudaSuccess) return cuda_status(e);
  for (int i = 0; i < 3; ++i) mismatches[i] = (int64_t)host[i];
  return HMAT_OK;
}
