// Serving: a request loop over resident HMatrices with memory-bounded admission
// and continuous batching (requests on one matrix that wait together run as one
// evaluation with their W columns side by side).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hmat_internal.h"

using namespace hmat;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  int matrix = 0;
  int dtype = HMAT_DTYPE_F64;
  const void* W = nullptr;
  void* Y = nullptr;
  int64_t ldw = 0, ldy = 0;
  int64_t q = 0;
  Clock::time_point submitted;
  bool done = false;
  hmat_status status = HMAT_OK;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  EvalContext* ctx[64] = {};  // one context per matrix (created on first use)
  std::vector<int64_t> members;  // request ids of the evaluation in flight
  int64_t bytes = 0;             // device bytes of that evaluation
  bool busy = false;
};

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct hmat_server {
  int device = -1;
  hmat_server_params params{};
  std::vector<hmat_t> handles;
  std::vector<Slot> slots;
  cudaMemPool_t pool = nullptr;

  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<int64_t> pending;
  std::unordered_map<int64_t, Request> requests;
  int64_t next_id = 1;
  bool stop = false;
  std::thread dispatcher;

  int64_t in_flight_bytes = 0, peak_bytes = 0;
  int64_t evaluations = 0, batched_requests = 0, rejected = 0;
  std::vector<double> latencies_ms;
  std::vector<std::vector<double>> matrix_latencies_ms;  // per matrix

  // bytes of one evaluation of `matrix` with q columns: workspaces + device W and Y
  int64_t need(int matrix, int64_t q, int dtype) const {
    const Handle& h = *handles[matrix];
    return align256(ctx_bytes(h, q, params.mode, dtype)) + 2 * align256(h.n_points * q * dtype_bytes(dtype));
  }

  void run();
  void record(const Request& r, Clock::time_point now);
  hmat_status launch(Slot& sl, int matrix, int dtype, const std::vector<int64_t>& ids, int64_t q_total);
  void retire(Slot& sl, hmat_status st);
};

void hmat_server::record(const Request& r, Clock::time_point now) {
  const double ms = std::chrono::duration<double, std::milli>(now - r.submitted).count();
  latencies_ms.push_back(ms);
  matrix_latencies_ms[r.matrix].push_back(ms);
}

hmat_status hmat_server::launch(Slot& sl, int matrix, int dtype, const std::vector<int64_t>& ids, int64_t q_total) {
  Handle* h = handles[matrix];
  const int64_t n = h->n_points;
  const int64_t es = dtype_bytes(dtype);
  const int64_t bytes = need(matrix, q_total, dtype);
  cudaStream_t s = sl.stream;
  if (!sl.ctx[matrix]) {
    hmat_status st = ctx_create(*h, &sl.ctx[matrix]);
    if (st != HMAT_OK) return st;
  }
  EvalContext* c = sl.ctx[matrix];
  uint8_t* block = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync((void**)&block, (size_t)std::max<int64_t>(bytes, 256), pool, s);
  if (e != cudaSuccess) return cuda_status(e);
  uint8_t* dW = block;
  uint8_t* dY = block + align256(n * q_total * es);
  uint8_t* ws = block + 2 * align256(n * q_total * es);
  // W columns of the merged requests side by side (strided copies), evaluate, split Y back
  int64_t col = 0;
  for (int64_t id : ids) {
    const Request& r = requests[id];
    e = cudaMemcpy2DAsync(dW + col * es, (size_t)(q_total * es), r.W, (size_t)(r.ldw * es), (size_t)(r.q * es),
                          (size_t)n, cudaMemcpyDefault, s);
    if (e != cudaSuccess) break;
    col += r.q;
  }
  hmat_status st = cuda_status(e);
  if (st == HMAT_OK) {
    ctx_bind(*h, c, q_total, params.mode, ws, dtype);
    st = eval_impl(h, c, dW, dY, q_total, params.mode, dtype, s);
  }
  col = 0;
  for (int64_t id : ids) {
    if (st != HMAT_OK) break;
    const Request& r = requests[id];
    e = cudaMemcpy2DAsync(r.Y, (size_t)(r.ldy * es), dY + col * es, (size_t)(q_total * es), (size_t)(r.q * es),
                          (size_t)n, cudaMemcpyDefault, s);
    st = cuda_status(e);
    col += r.q;
  }
  cudaFreeAsync(block, s);
  if (st == HMAT_OK) st = cuda_status(cudaEventRecord(sl.done, s));
  if (st != HMAT_OK) return st;
  sl.members = ids;
  sl.bytes = bytes;
  sl.busy = true;
  in_flight_bytes += bytes;
  peak_bytes = std::max(peak_bytes, in_flight_bytes);
  evaluations += 1;
  batched_requests += (int64_t)ids.size();
  return HMAT_OK;
}

void hmat_server::retire(Slot& sl, hmat_status st) {
  const auto now = Clock::now();
  for (int64_t id : sl.members) {
    Request& r = requests[id];
    r.done = true;
    r.status = st;
    record(r, now);
  }
  in_flight_bytes -= sl.bytes;
  sl.members.clear();
  sl.bytes = 0;
  sl.busy = false;
}

void hmat_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    // completions
    bool any_busy = false, progressed = false;
    for (Slot& sl : slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      hmat_status st = cuda_status(q);
      if (st == HMAT_OK) {
        int word = 0;  // a kernel-side timeout of any evaluation on this handle is reported to its requests
        if (cudaMemcpyAsync(&word, handles[requests[sl.members[0]].matrix]->status, sizeof(int),
                            cudaMemcpyDeviceToHost, sl.stream) == cudaSuccess &&
            cudaStreamSynchronize(sl.stream) == cudaSuccess && word != 0)
          st = (hmat_status)word;
      }
      retire(sl, st);
      progressed = true;
    }
    if (progressed) cv_done.notify_all();
    // admissions: the oldest pending request, joined by the pending requests on the same matrix
    while (!pending.empty()) {
      Slot* free_slot = nullptr;
      for (Slot& sl : slots)
        if (!sl.busy) {
          free_slot = &sl;
          break;
        }
      if (!free_slot) break;
      const Request& head = requests[pending.front()];
      std::vector<int64_t> ids{head.id};
      int64_t q_total = head.q;
      for (size_t k = 1; k < pending.size(); ++k) {
        const Request& r = requests[pending[k]];
        if (r.matrix != head.matrix || r.dtype != head.dtype || q_total + r.q > params.max_q) continue;
        if (in_flight_bytes + need(head.matrix, q_total + r.q, head.dtype) > params.memory_budget) continue;
        ids.push_back(r.id);
        q_total += r.q;
      }
      if (in_flight_bytes + need(head.matrix, q_total, head.dtype) > params.memory_budget) break;  // wait for memory
      for (int64_t id : ids) pending.erase(std::find(pending.begin(), pending.end(), id));
      const hmat_status st = launch(*free_slot, head.matrix, head.dtype, ids, q_total);
      if (st != HMAT_OK) {
        const auto now = Clock::now();
        for (int64_t id : ids) {
          Request& r = requests[id];
          r.done = true;
          r.status = st;
          record(r, now);
        }
        cv_done.notify_all();
      } else {
        any_busy = true;
      }
    }
    if (stop && pending.empty() && !any_busy) break;
    if (any_busy) {  // poll the slots' events
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else {
      cv_submit.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

extern "C" hmat_status hmat_server_create(const hmat_t* handles, int count, const hmat_server_params* p,
                                          hmat_server_t* out) {
  if (!out) return HMAT_EINVAL;
  *out = nullptr;
  if (!handles || count <= 0 || count > 64 || !p || p->slots < 1 || p->slots > 64 || p->memory_budget <= 0 ||
      p->max_q < 1 || p->max_pending < 0)
    return HMAT_EINVAL;
  if (p->mode != HMAT_MODE_FP64 && p->mode != HMAT_MODE_MIXED) return HMAT_EUNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || handles[i]->device != dev) return HMAT_EINVAL;
    if (p->mode == HMAT_MODE_MIXED && !handles[i]->has_mixed) return HMAT_EUNSUPPORTED;
    if (p->mode == HMAT_MODE_FP64 && !handles[i]->has_fp64) return HMAT_EUNSUPPORTED;
  }
  hmat_server* sv = new (std::nothrow) hmat_server();
  if (!sv) return HMAT_ENOMEM;
  sv->device = dev;
  sv->params = *p;
  sv->handles.assign(handles, handles + count);
  sv->matrix_latencies_ms.resize(count);
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaError_t e = cudaMemPoolCreate(&sv->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = (uint64_t)p->memory_budget;  // keep freed blocks for reuse up to the budget
    e = cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  sv->slots.resize(p->slots);
  for (Slot& sl : sv->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    hmat_server_free(sv);
    return cuda_status(e);
  }
  sv->dispatcher = std::thread([sv]() { sv->run(); });
  *out = sv;
  return HMAT_OK;
}

namespace {

// Pinned host or device memory: copies to and from pageable memory would block the dispatcher.
bool copyable(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" hmat_status hmat_server_submit_typed(hmat_server_t sv, int matrix, const void* W, int64_t ldw, void* Y,
                                                int64_t ldy, int64_t q, int dtype, int64_t* id) {
  if (!sv || !id || matrix < 0 || matrix >= (int)sv->handles.size() || q < 1 || !W || !Y || ldw < q || ldy < q)
    return HMAT_EINVAL;
  if (dtype != HMAT_DTYPE_F64 && dtype != HMAT_DTYPE_F32) return HMAT_EINVAL;
  if (q > sv->params.max_q || !copyable(W) || !copyable(Y)) return HMAT_EINVAL;
  if (sv->need(matrix, q, dtype) > sv->params.memory_budget) return HMAT_ENOMEM;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return HMAT_EINVAL;
  if (sv->params.max_pending > 0 && (int64_t)sv->pending.size() >= sv->params.max_pending) {
    sv->rejected += 1;  // load shedding: the queue is full
    return HMAT_EBUSY;
  }
  Request r;
  r.id = sv->next_id++;
  r.matrix = matrix;
  r.dtype = dtype;
  r.W = W;
  r.Y = Y;
  r.ldw = ldw;
  r.ldy = ldy;
  r.q = q;
  r.submitted = Clock::now();
  sv->requests[r.id] = r;
  sv->pending.push_back(r.id);
  *id = r.id;
  sv->cv_submit.notify_one();
  return HMAT_OK;
}

extern "C" hmat_status hmat_server_submit(hmat_server_t sv, int matrix, const double* W, int64_t ldw, double* Y,
                                          int64_t ldy, int64_t q, int64_t* id) {
  return hmat_server_submit_typed(sv, matrix, W, ldw, Y, ldy, q, HMAT_DTYPE_F64, id);
}

extern "C" hmat_status hmat_server_wait(hmat_server_t sv, int64_t id, int timeout_ms) {
  if (!sv) return HMAT_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(id);
  if (it == sv->requests.end()) return HMAT_EINVAL;
  auto ready = [&]() { return sv->requests[id].done; };
  if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
  else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return HMAT_ETIMEOUT;
  const hmat_status st = sv->requests[id].status;
  sv->requests.erase(id);  // a completed request is forgotten once waited on
  return st;
}

namespace {

double percentile(const std::vector<double>& sorted, double p) {
  if (sorted.empty()) return 0.0;
  const size_t k = std::min(sorted.size() - 1, (size_t)(p * (double)(sorted.size() - 1) + 0.5));
  return sorted[k];
}

}  // namespace

extern "C" hmat_status hmat_server_stats(hmat_server_t sv, double* out, int n) {
  if (!sv || !out || n < 0) return HMAT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  std::vector<double> lat = sv->latencies_ms;
  std::sort(lat.begin(), lat.end());
  const double vals[7] = {(double)lat.size(), percentile(lat, 0.50), percentile(lat, 0.99),
                          sv->evaluations ? (double)sv->batched_requests / (double)sv->evaluations : 0.0,
                          (double)sv->evaluations, (double)sv->peak_bytes, (double)sv->rejected};
  for (int i = 0; i < n && i < 7; ++i) out[i] = vals[i];
  return HMAT_OK;
}

extern "C" hmat_status hmat_server_matrix_stats(hmat_server_t sv, int matrix, double* out, int n) {
  if (!sv || !out || n < 0 || matrix < 0 || matrix >= (int)sv->handles.size()) return HMAT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  std::vector<double> lat = sv->matrix_latencies_ms[matrix];
  std::sort(lat.begin(), lat.end());
  const double vals[3] = {(double)lat.size(), percentile(lat, 0.50), percentile(lat, 0.99)};
  for (int i = 0; i < n && i < 3; ++i) out[i] = vals[i];
  return HMAT_OK;
}

extern "C" hmat_status hmat_server_free(hmat_server_t sv) {
  if (!sv) return HMAT_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_submit.notify_all();
  if (sv->dispatcher.joinable()) sv->dispatcher.join();
  for (Slot& sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    for (EvalContext*& c : sl.ctx) {
      ctx_destroy(c);
      c = nullptr;
    }
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  if (sv->pool) cudaMemPoolDestroy(sv->pool);
  delete sv;
  return HMAT_OK;
}
