// Upward and downward passes of the mixed-precision mode as FP32 grouped GEMMs
// (products and sums in FP32, operands copied into shared memory with cp.async) on
// FP32 copies of the bases laid out for 16-byte copies. The upward leaf step reads the FP32 tree-order copy of W
// that the split step writes; the downward leaf step adds into Y (FP64). The coupling
// reduction between them runs here too when the ranks are small, else on the tensor
// cores (hmat_mixed.cu).
#include "hmat_gemm_f32.cuh"

namespace hmat {

cudaError_t launch_f32_phase(const Handle& h, const Phase& ph, const float* X, const int64_t* x_map, void* Y,
                             bool y_is_f64, const int64_t* y_map, int64_t q, cudaStream_t stream) {
  // the FP32 arena holds the operands of the FP32 phases only (the coupling blocks
  // only when the coupling runs in FP32)
  if (ph.kind == PH_NEAR || (ph.kind == PH_COUPLING && h.tc_coupling)) return cudaErrorInvalidValue;
  if (y_is_f64)
    return gemm::launch_phase_f32<double>(h, ph, h.arena32, X, x_map, (double*)Y, y_map, q, stream);
  return gemm::launch_phase_f32<float>(h, ph, h.arena32, X, x_map, (float*)Y, y_map, q, stream);
}

}  // namespace hmat
