// Far field of the mixed-precision mode: the upward pass, the coupling reduction and
// the downward pass as FP32 grouped GEMMs (products and sums in FP32) on an FP32
// copy of the bases and coupling blocks. The upward leaf step reads W (FP64) and the
// downward leaf step adds into Y (FP64).
#include "hmat_gemm.cuh"

namespace hmat {

cudaError_t launch_f32_phase(const Handle& h, const Phase& ph, const void* X, bool x_is_f64, const int64_t* x_map,
                             void* Y, bool y_is_f64, const int64_t* y_map, int64_t q, cudaStream_t stream) {
  const float* a = h.arena32;
  const int64_t sh = h.arena32_shift;
  if (x_is_f64 && !y_is_f64)
    return gemm::launch_phase<float, double, float, float>(h, ph, a, sh, (const double*)X, x_map, (float*)Y, y_map,
                                                           q, stream);
  if (!x_is_f64 && y_is_f64)
    return gemm::launch_phase<float, float, double, float>(h, ph, a, sh, (const float*)X, x_map, (double*)Y, y_map,
                                                           q, stream);
  if (!x_is_f64 && !y_is_f64)
    return gemm::launch_phase<float, float, float, float>(h, ph, a, sh, (const float*)X, x_map, (float*)Y, y_map, q,
                                                          stream);
  return cudaErrorInvalidValue;
}

}  // namespace hmat
