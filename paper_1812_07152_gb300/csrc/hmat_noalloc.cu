// hmat_eval_noalloc: the FP64 evaluation with its skeleton workspaces in a static
// device array instead of handle-owned cudaMalloc memory, for callers that must not
// allocate device memory during an evaluation (see include/hmat.h).
#include <cuda_runtime.h>

#include <mutex>

#include "hmat_internal.h"

namespace {

constexpr int64_t kScratchValues = HMAT_NOALLOC_SCRATCH_VALUES;
constexpr int kMaxDevices = 64;

// The workspace of every no-alloc evaluation in this process on this device:
// the first half holds the upward weights w, the second the downward potentials u.
static __device__ __align__(256) double g_noalloc_scratch[kScratchValues];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on device `dev` (looked up once per device, with it current).
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<double*>(g_scratch_addr[dev]);
  return cudaSuccess;
}

}  // namespace

using namespace hmat;

extern "C" hmat_status hmat_eval_noalloc(hmat_t h, const double* W, double* Y, int64_t q, void* stream) {
  if (!h || q < 0) return HMAT_EINVAL;
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
  if (dev < 0 || dev >= kMaxDevices) return HMAT_EUNSUPPORTED;
  double* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return HMAT_ECUDA;
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
