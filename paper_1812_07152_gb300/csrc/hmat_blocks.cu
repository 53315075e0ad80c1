// Device evaluation of dense kernel blocks K(I, J) straight into the packed arena:
// the near blocks D_ij = K(I_i, I_j) and the coupling blocks B_ab = K(S_a, S_b)
// of the inspector's compression (Section 3.1). One CTA per block, coalesced
// row-major writes; the kernel functions are those of Section 1 (1/r: Section 4.1).
#include <cuda_runtime.h>

#include "hmat_internal.h"
#include "hmat_kernels.cuh"

namespace hmat {
namespace {

constexpr int kMaxDim = 64;

__global__ void __launch_bounds__(256)
k_eval_blocks(const BlockJob* __restrict__ jobs, const double* __restrict__ pts, int dim,
              const int64_t* __restrict__ skel, int kernel, double param, double* __restrict__ arena) {
  const BlockJob job = jobs[blockIdx.x];
  double* out = arena + job.a_off;
  const int64_t total = (int64_t)job.rows * job.cols;
  const KernelSpec ks = kernel_spec(kernel, param);
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int r = (int)(e / job.cols), c = (int)(e % job.cols);
    const int64_t pr = job.row_skel ? skel[job.row_off + r] : job.row_off + r;
    const int64_t pc = job.col_skel ? skel[job.col_off + c] : job.col_off + c;
    out[r * job.ld + c] = kernel_entry(ks, pts + pr * dim, pts + pc * dim, dim);
  }
}

}  // namespace

cudaError_t launch_eval_blocks(const BlockJob* jobs, int64_t n_jobs, const double* pts, int dim,
                               const int64_t* skel_pts, int kernel, double param, double* arena,
                               cudaStream_t stream) {
  if (dim <= 0 || dim > kMaxDim) return cudaErrorInvalidValue;
  const int64_t max_grid = 2147483647;
  for (int64_t s = 0; s < n_jobs; s += max_grid) {
    const int64_t cnt = n_jobs - s < max_grid ? n_jobs - s : max_grid;
    k_eval_blocks<<<(unsigned)cnt, 256, 0, stream>>>(jobs + s, pts, dim, skel_pts, kernel, param, arena);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hmat
