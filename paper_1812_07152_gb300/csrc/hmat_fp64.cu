// FP64 evaluation (HMAT_MODE_FP64): every phase is the grouped GEMM of
// hmat_gemm.cuh in double precision.
//
// On GB300 the FP64 pipe retires about 2 DFMA per clock per SM, 1/58 of FP32,
// so these launches are bound by DFMA issue and not by memory: register tiles of
// 4x4 outputs per thread, double-buffered shared-memory operand tiles, row tiles
// matched to each task's height and column tiles matched to q so that no DFMA is
// spent on padding.
#include "hmat_gemm.cuh"

namespace hmat {

cudaError_t launch_fp64_phase(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map,
                              double* Y, const int64_t* y_map, int64_t q, cudaStream_t stream) {
  return gemm::launch_phase<double, double, double, double>(h, ph, h.arena, 0, X, x_map, Y, y_map, q, stream);
}

}  // namespace hmat
