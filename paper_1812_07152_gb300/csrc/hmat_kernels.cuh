// One entry K(x, y) of a kernel matrix in FP64, the kernel functions of Section 1
// (Gaussian, inverse multiquadric) and Section 4.1 (1/r, 0 for coincident points).
// Shared by the load-time block evaluator and the near field that evaluates its blocks
// on the fly, so that both produce the same value bit for bit. Few FP64 operations per
// entry (this GPU issues about 2 per clock per SM): the squared distance by fused
// multiply-adds in dimension order, the Gaussian's exponent by a multiply with the
// precomputed -1 / (2 h^2), the inverse square roots by rsqrt.
#pragma once

#include <cstdint>

#include "hmat_internal.h"

namespace hmat {

struct KernelSpec {
  int32_t kernel;         // HMAT_KERNEL_*
  double neg_inv_two_h2;  // Gaussian: -1 / (2 h^2)
  double c2;              // inverse multiquadric: c^2
};

__host__ __device__ inline KernelSpec kernel_spec(int kernel, double param) {
  return KernelSpec{kernel, -1.0 / (2.0 * param * param), param * param};
}

__device__ __forceinline__ double kernel_entry(const KernelSpec& ks, const double* __restrict__ x,
                                               const double* __restrict__ y, int dim) {
  double r2 = 0.0;
  for (int k = 0; k < dim; ++k) {
    const double diff = __dsub_rn(x[k], y[k]);
    r2 = __fma_rn(diff, diff, r2);
  }
  if (ks.kernel == HMAT_KERNEL_GAUSSIAN) return exp(__dmul_rn(r2, ks.neg_inv_two_h2));
  if (ks.kernel == HMAT_KERNEL_IMQ) return rsqrt(__dadd_rn(r2, ks.c2));
  return r2 > 0.0 ? rsqrt(r2) : 0.0;
}

}  // namespace hmat
