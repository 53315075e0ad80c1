// Batched evaluation: many HMatrices of uneven size, rank and q evaluated together
// as the parallel branches of one CUDA graph (one launch per batch once captured).
#include <cstring>
#include <new>
#include <vector>

#include "hmat_internal.h"

using namespace hmat;

struct hmat_batch {
  int device = -1;
  int mode = HMAT_MODE_FP64;
  std::vector<hmat_t> handles;
  std::vector<EvalContext*> ctx;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> join;
  cudaStream_t capture = nullptr;   // the graph is captured on this stream (never the legacy default stream)
  cudaEvent_t fork = nullptr;
  // the captured graph and the arguments it was captured for
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key_w;
  std::vector<void*> key_y;
  std::vector<int64_t> key_q;
  int key_dtype = HMAT_DTYPE_F64;
};

namespace {

void batch_release(hmat_batch* b) {
  if (b->capture) cudaStreamSynchronize(b->capture);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  for (EvalContext* c : b->ctx) ctx_destroy(c);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

}  // namespace

extern "C" hmat_status hmat_batch_create(const hmat_t* handles, int count, int mode, hmat_batch_t* out) {
  if (!out) return HMAT_EINVAL;
  *out = nullptr;
  if (!handles || count <= 0) return HMAT_EINVAL;
  if (mode != HMAT_MODE_FP64 && mode != HMAT_MODE_MIXED) return HMAT_EUNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || handles[i]->device != dev) return HMAT_EINVAL;
    if (mode == HMAT_MODE_MIXED && !handles[i]->has_mixed) return HMAT_EUNSUPPORTED;
    if (mode == HMAT_MODE_FP64 && !handles[i]->has_fp64) return HMAT_EUNSUPPORTED;
  }
  hmat_batch* b = new (std::nothrow) hmat_batch();
  if (!b) return HMAT_ENOMEM;
  b->device = dev;
  b->mode = mode;
  b->handles.assign(handles, handles + count);
  cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    EvalContext* c = nullptr;
    hmat_status st = ctx_create(*handles[i], &c);
    if (st != HMAT_OK) {
      batch_release(b);
      return st;
    }
    b->ctx.push_back(c);
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branch.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->join.push_back(ev);
  }
  if (e != cudaSuccess) {
    batch_release(b);
    return cuda_status(e);
  }
  *out = b;
  return HMAT_OK;
}

extern "C" hmat_status hmat_batch_eval_typed(hmat_batch_t b, const void* const* W, void* const* Y, const int64_t* q,
                                             int dtype, void* stream) {
  if (!b || !W || !Y || !q) return HMAT_EINVAL;
  if (dtype != HMAT_DTYPE_F64 && dtype != HMAT_DTYPE_F32) return HMAT_EINVAL;
  const int n = (int)b->handles.size();
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (dev != b->device) return HMAT_EINVAL;
  for (int i = 0; i < n; ++i) {
    const hmat_t h = b->handles[i];
    if (q[i] < 0) return HMAT_EINVAL;
    if (q[i] > 0 && h->n_points > 0) {
      if (!W[i] || !Y[i] || W[i] == Y[i]) return HMAT_EINVAL;
      if (b->mode == HMAT_MODE_MIXED && (q[i] + 127) / 128 > 65535) return HMAT_EUNSUPPORTED;
    }
  }
  const bool same = b->exec && dtype == b->key_dtype && std::equal(W, W + n, b->key_w.begin()) &&
                    std::equal(Y, Y + n, b->key_y.begin()) && std::equal(q, q + n, b->key_q.begin());
  cudaStream_t s = (cudaStream_t)stream;
  if (!same) {
    // workspaces first: allocation cannot happen inside a capture
    for (int i = 0; i < n; ++i) {
      if (q[i] == 0 || b->handles[i]->n_points == 0) continue;
      hmat_status st = ctx_reserve(*b->handles[i], b->ctx[i], q[i], b->mode, dtype);
      if (st != HMAT_OK) return st;
    }
    if (b->exec) {
      cudaStreamSynchronize(b->capture);
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    // capture every member's evaluation as a branch forked from the capture stream
    std::vector<int> profiling(n);
    for (int i = 0; i < n; ++i) {
      profiling[i] = b->handles[i]->profiling;
      b->handles[i]->profiling = 0;
    }
    hmat_status st = HMAT_OK;
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->capture);
    for (int i = 0; i < n && e == cudaSuccess && st == HMAT_OK; ++i) {
      if (q[i] == 0 || b->handles[i]->n_points == 0) continue;
      e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
      if (e != cudaSuccess) break;
      st = eval_impl(b->handles[i], b->ctx[i], W[i], Y[i], q[i], b->mode, dtype, b->branch[i]);
      if (st != HMAT_OK) break;
      e = cudaEventRecord(b->join[i], b->branch[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->capture, b->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->capture, &graph);
    for (int i = 0; i < n; ++i) b->handles[i]->profiling = profiling[i];
    if (e == cudaSuccess) e = ee;
    if (st == HMAT_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != HMAT_OK) return st;
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return cuda_status(e);
    }
    b->key_w.assign(W, W + n);
    b->key_y.assign(Y, Y + n);
    b->key_q.assign(q, q + n);
    b->key_dtype = dtype;
  }
  return cuda_status(cudaGraphLaunch(b->exec, s));
}

extern "C" hmat_status hmat_batch_eval(hmat_batch_t b, const double* const* W, double* const* Y, const int64_t* q,
                                       void* stream) {
  return hmat_batch_eval_typed(b, reinterpret_cast<const void* const*>(W), reinterpret_cast<void* const*>(Y), q,
                               HMAT_DTYPE_F64, stream);
}

extern "C" hmat_status hmat_batch_free(hmat_batch_t b) {
  if (!b) return HMAT_OK;
  batch_release(b);
  return HMAT_OK;
}
