// Far field of the mixed-precision mode: the upward pass, the coupling reduction and
// the downward pass as FP32 grouped GEMMs (products and sums in FP32, operands
// copied into shared memory with cp.async) on an FP32 copy of the bases and coupling
// blocks. The upward leaf step reads the FP32 tree-order copy of W that the split
// step writes; the downward leaf step adds into Y (FP64).
#include "hmat_gemm.cuh"

namespace hmat {

cudaError_t launch_f32_phase(const Handle& h, const Phase& ph, const float* X, const int64_t* x_map, void* Y,
                             bool y_is_f64, const int64_t* y_map, int64_t q, cudaStream_t stream) {
  // the FP32 arena starts at the bases: near blocks have no FP32 copy
  if (ph.kind == PH_NEAR) return cudaErrorInvalidValue;
  if (y_is_f64)
    return gemm::launch_phase_f32<double>(h, ph, h.arena32, h.arena32_shift, X, x_map, (double*)Y, y_map, q, stream);
  return gemm::launch_phase_f32<float>(h, ph, h.arena32, h.arena32_shift, X, x_map, (float*)Y, y_map, q, stream);
}

}  // namespace hmat
