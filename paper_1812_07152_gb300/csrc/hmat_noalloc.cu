// hmat_eval_noalloc: the FP64 evaluation with its skeleton workspaces in a static
// device array instead of handle-owned cudaMalloc memory, for callers that must not
// allocate device memory during an evaluation (see include/hmat.h).
#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace {

constexpr int64_t kScratchValues = HMAT_NOALLOC_SCRATCH_VALUES;

// The workspace of every no-alloc evaluation in this process on this device:
// the first half holds the upward weights w, the second the downward potentials u.
static __device__ __align__(256) double g_noalloc_scratch[kScratchValues];

}  // namespace

namespace hmat {

// Device address of the array on the current device. Called by hmat_load and
// hmat_build (which allocate anyway) with the handle's device current: under lazy
// module loading the lookup is what loads this file's module and allocates the
// array, so it must not happen inside hmat_eval_noalloc.
cudaError_t noalloc_scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  *out = e == cudaSuccess ? static_cast<double*>(p) : nullptr;
  return e;
}

}  // namespace hmat

using namespace hmat;

extern "C" hmat_status hmat_eval_noalloc(hmat_t h, const double* W, double* Y, int64_t q, void* stream) {
  if (!h || q < 0) return HMAT_EINVAL;
  if (!h->has_fp64) return HMAT_EUNSUPPORTED;
  if (q == 0 || h->n_points == 0) return HMAT_OK;
  if (!W || !Y || W == Y) return HMAT_EINVAL;
  const char* w0 = (const char*)W;
  const char* y0 = (const char*)Y;
  const int64_t bytes = h->n_points * q * (int64_t)sizeof(double);
  if (w0 < y0 + bytes && y0 < w0 + bytes) return HMAT_EINVAL;  // W and Y overlap
  const int64_t half = kScratchValues / 2;
  if (h->sum_rank > 0 && q > half / h->sum_rank) return HMAT_EINVAL;  // workspaces exceed the array
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (dev != h->device) return HMAT_EINVAL;
  double* base = h->noalloc_scratch;  // resolved when the handle was loaded
  if (!base) return HMAT_ECUDA;
  double* ws = base;
  double* us = base + half;
  cudaStream_t s = (cudaStream_t)stream;
  const TuneEntry* tuned = find_tuned(*h, q, HMAT_MODE_FP64);
  for (size_t i = 0; i < h->phases.size(); ++i) {
    const Phase& ph = h->phases[i];
    const double* X = ph.x == MAT_USER ? W : (ph.x == MAT_SKEL_W ? ws : us);
    double* Yd = ph.y == MAT_USER ? Y : (ph.y == MAT_SKEL_W ? ws : us);
    const int64_t* xm = phase_x_map(*h, ph);
    const int64_t* ym = ph.y == MAT_USER ? h->perm : nullptr;
    const int shape = tuned && i < tuned->shape.size() ? tuned->shape[i] : -1;
    const cudaError_t e = launch_fp64_phase(*h, ph, X, xm, Yd, ym, q, shape, -1, s);
    if (e != cudaSuccess) return HMAT_ECUDA;
  }
  return HMAT_OK;
}
