// FP64 near field with its blocks evaluated on the fly (HMAT_BUILD_NEAR_OTF): the grouped
// GEMM of hmat_gemm.cuh whose A operand is K(x_i, x_j) computed from the tree-ordered
// points, in a translation unit of its own so that it compiles beside hmat_fp64.cu.
#include "hmat_gemm.cuh"

namespace hmat {

cudaError_t launch_fp64_near_otf(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map, double* Y,
                                 const int64_t* y_map, int64_t q, int shape, int64_t n_tiles, cudaStream_t stream) {
  if (!h.near_otf || ph.kind != PH_NEAR) return cudaErrorInvalidValue;
  return gemm::launch_phase<double, double, double, double, true>(h, ph, shape, n_tiles, h.arena, 0, X, x_map, Y,
                                                                  y_map, q, stream);
}

}  // namespace hmat
