// FP64 evaluation (HMAT_MODE_FP64): every phase is the grouped GEMM of
// hmat_gemm.cuh in double precision.
//
// On GB300 the FP64 pipe retires about 2 DFMA per clock per SM, 1/58 of FP32,
// so these launches are bound by DFMA issue and not by memory: register tiles of
// up to 4x4 outputs per thread, double-buffered shared-memory operand tiles, row
// tiles matched to each task's height and column tiles (1 to 64 wide) matched to q
// so that few DFMAs are spent on padding.
#include "hmat_gemm.cuh"

namespace hmat {

cudaError_t launch_fp64_phase(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map,
                              double* Y, const int64_t* y_map, int64_t q, int shape, int64_t n_tiles,
                              cudaStream_t stream) {
  if (h.near_otf && ph.kind == PH_NEAR)  // hmat_fp64_otf.cu
    return launch_fp64_near_otf(h, ph, X, x_map, Y, y_map, q, shape, n_tiles, stream);
  return gemm::launch_phase<double, double, double, double>(h, ph, shape, n_tiles, h.arena, 0, X, x_map, Y, y_map,
                                                            q, stream);
}

int fp64_default_shape(int64_t q) { return gemm::default_col_shape(q); }

int fp64_shape_columns(int shape) { return shape >= 0 && shape < gemm::kColShapes ? gemm::kColBN[shape] : 0; }

}  // namespace hmat
