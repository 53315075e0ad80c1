// Evaluation runtime: Y = K~ W for one loaded HMatrix (Section 2.1, "Evaluation").
//
// FP64 mode: the phases in order (near field, upward leaves, upward transfers level by
// level, coupling, downward transfers level by level, downward leaves), each one
// grouped-GEMM launch per row-tile size on the caller's stream.
//
// Mixed mode: W is split into FP16 hi/lo tensor-core tiles (and an FP32 tree-order
// copy); the near field runs on the tensor cores on the caller's stream while the far
// chain (upward pass, coupling, downward transfers) runs on a high-priority side stream
// as persistent FP32 launches over every tree level (hmat_chain.cu), the coupling on the
// tensor cores between two of them when its ranks fill the tiles; the downward leaf
// step, which adds into Y, follows both as one more persistent launch.
//
// The per-evaluation state lives in an EvalContext, so several evaluations of the
// same HMatrix can be in flight at once (batches, the server).
#include <algorithm>
#include <cstring>
#include <new>

#include "hmat_internal.h"

namespace hmat {
namespace {

constexpr int64_t kAlignBytes = 256;
// hmat_eval_host pipelines the mixed mode in two column groups from this many columns each.
constexpr int64_t kHostSplitMinQ = 64;

int64_t align_up(int64_t x) { return (x + kAlignBytes - 1) / kAlignBytes * kAlignBytes; }

// Event records around one launch of the evaluation when the handle is profiling.
bool prof_begin(Handle* h, int32_t kind, cudaStream_t s, Handle::ProfRecord* rec) {
  rec->kind = kind;
  if (!h->profiling) return true;
  for (cudaEvent_t* ev : {&rec->start, &rec->stop}) {
    if (!h->event_pool.empty()) {
      *ev = h->event_pool.back();
      h->event_pool.pop_back();
    } else if (cudaEventCreate(ev) != cudaSuccess) {
      return false;
    }
  }
  return cudaEventRecord(rec->start, s) == cudaSuccess;
}

bool prof_end(Handle* h, const Handle::ProfRecord& rec, cudaStream_t s) {
  if (!h->profiling) return true;
  if (cudaEventRecord(rec.stop, s) != cudaSuccess) return false;
  h->prof.push_back(rec);
  return true;
}

hmat_status check_call(const Handle* h, const void* W, const void* Y, int64_t q, int mode, int dtype) {
  if (!h || q < 0) return HMAT_EINVAL;
  if (dtype != HMAT_DTYPE_F64 && dtype != HMAT_DTYPE_F32) return HMAT_EINVAL;
  if (mode != HMAT_MODE_FP64 && mode != HMAT_MODE_MIXED) return HMAT_EUNSUPPORTED;
  if (mode == HMAT_MODE_MIXED && !h->has_mixed) return HMAT_EUNSUPPORTED;
  if (mode == HMAT_MODE_FP64 && !h->has_fp64) return HMAT_EUNSUPPORTED;
  if (q == 0 || h->n_points == 0) return HMAT_OK;
  if (!W || !Y || W == Y) return HMAT_EINVAL;
  const char* w0 = (const char*)W;
  const char* y0 = (const char*)Y;
  const int64_t bytes = h->n_points * q * dtype_bytes(dtype);
  if (w0 < y0 + bytes && y0 < w0 + bytes) return HMAT_EINVAL;  // W and Y overlap
  if (mode == HMAT_MODE_MIXED && (q + 127) / 128 > 65535) return HMAT_EUNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (dev != h->device) return HMAT_EINVAL;
  return HMAT_OK;
}

}  // namespace

// Tensor-core column tiles: n_ct tiles of n_t columns (a multiple of 16, at most 128)
// cover q. The default is the fewest tiles, balanced; the tuner also tries one and two
// more tiles (more CTAs when a matrix has few leaves).
std::vector<int> mixed_nt_candidates(int64_t q) {
  std::vector<int> out;
  const int64_t base = std::max<int64_t>((q + 127) / 128, 1);
  for (int64_t n_ct : {base, base + 1, base + 2}) {
    const int64_t per = (q + n_ct - 1) / n_ct;
    const int n_t = (int)std::max<int64_t>(16, (per + 15) / 16 * 16);
    if (std::find(out.begin(), out.end(), n_t) == out.end()) out.push_back(n_t);
  }
  return out;
}

int64_t mixed_cols_bound(int64_t q) {
  int64_t best = 0;
  for (int n_t : mixed_nt_candidates(q)) best = std::max<int64_t>(best, (q + n_t - 1) / n_t * n_t);
  return best;
}

const TuneEntry* find_tuned(const Handle& h, int64_t q, int mode) {
  for (const TuneEntry& t : h.tuned)
    if (t.q == q && t.mode == mode) return &t;
  return nullptr;
}

void mixed_tiles(const Handle& h, int64_t q, int* n_t, int64_t* n_ct) {
  const TuneEntry* t = find_tuned(h, q, HMAT_MODE_MIXED);
  *n_t = t && t->n_t > 0 ? t->n_t : mixed_nt_candidates(q)[0];
  *n_ct = (q + *n_t - 1) / *n_t;
}

hmat_status ctx_create(const Handle& h, EvalContext** out) {
  *out = nullptr;
  EvalContext* c = new (std::nothrow) EvalContext();
  if (!c) return HMAT_ENOMEM;
  if (h.has_mixed) {
    // the far chain runs beside the near field at the lowest priority: the near field's
    // CTAs (one per SM) are placed first, and the chain's persistent CTAs fill the SMs its
    // last wave leaves (measured: N=65536 mixture 2.72 -> 2.66 ms, N=262144 1/r q=1 1.88 ->
    // 1.85 ms against the highest priority)
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      ctx_destroy(c);
      return cuda_status(e);
    }
  }
  *out = c;
  return HMAT_OK;
}

void ctx_destroy(EvalContext* c) {
  if (!c) return;
  if (c->aux) cudaStreamSynchronize(c->aux);
  cudaFree(c->block);
  cudaFree(c->host_w);
  cudaFree(c->host_y);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->copy) {
    cudaStreamSynchronize(c->copy);
    cudaStreamDestroy(c->copy);
  }
  for (cudaEvent_t ev : c->ev_copy)
    if (ev) cudaEventDestroy(ev);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

int64_t ctx_bytes(const Handle& h, int64_t q, int mode, int dtype) {
  const int64_t r = std::max<int64_t>(h.sum_rank, 1);
  if (mode == HMAT_MODE_MIXED) {
    const int64_t cols = mixed_cols_bound(q);
    return 2 * align_up(sizeof(unsigned long long)) + align_up(h.tc_near.n_chunks * cols * 256) +
           align_up(h.tc_far.n_chunks * cols * 256) +
           align_up(std::max<int64_t>(h.n_points, 1) * q * 4) + 2 * align_up(r * q * 4) +
           align_up(h.chain.n_ctr * 4);
  }
  const int64_t io = dtype == HMAT_DTYPE_F32 ? 2 * align_up(std::max<int64_t>(h.n_points, 1) * q * 8) : 0;
  return 2 * align_up(r * q * 8) + io + align_up(h.chain64.n_ctr * 4);
}

void ctx_bind(const Handle& h, EvalContext* c, int64_t q, int mode, uint8_t* base, int dtype) {
  const int64_t r = std::max<int64_t>(h.sum_rank, 1);
  uint8_t* p = base;
  auto take = [&](int64_t bytes) {
    uint8_t* x = p;
    p += align_up(bytes);
    return x;
  };
  c->ws = c->us = nullptr;
  c->w64 = c->y64 = nullptr;
  c->wmax = c->smax = nullptr;
  c->wsplit = c->ssplit = nullptr;
  c->w32 = c->ws32 = c->us32 = nullptr;
  c->chain_ctr = nullptr;
  if (mode == HMAT_MODE_MIXED) {
    const int64_t cols = mixed_cols_bound(q);
    c->wmax = (unsigned long long*)take(sizeof(unsigned long long));
    c->wsplit = take(h.tc_near.n_chunks * cols * 256);
    c->smax = (unsigned long long*)take(sizeof(unsigned long long));
    c->ssplit = take(h.tc_far.n_chunks * cols * 256);
    c->w32 = (float*)take(std::max<int64_t>(h.n_points, 1) * q * 4);
    c->ws32 = (float*)take(r * q * 4);
    c->us32 = (float*)take(r * q * 4);
    c->chain_ctr = (int32_t*)take(h.chain.n_ctr * 4);
  } else {
    c->ws = (double*)take(r * q * 8);
    c->us = (double*)take(r * q * 8);
    c->chain_ctr = (int32_t*)take(h.chain64.n_ctr * 4);
    if (dtype == HMAT_DTYPE_F32) {
      c->w64 = (double*)take(std::max<int64_t>(h.n_points, 1) * q * 8);
      c->y64 = (double*)take(std::max<int64_t>(h.n_points, 1) * q * 8);
    }
  }
}

hmat_status ctx_reserve(const Handle& h, EvalContext* c, int64_t q, int mode, int dtype) {
  const int64_t need = ctx_bytes(h, q, mode, dtype);
  if (need > c->block_bytes) {
    uint8_t* p = nullptr;
    cudaError_t e = cudaMalloc((void**)&p, (size_t)need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
    cudaDeviceSynchronize();  // earlier evaluations may still use the old block
    cudaFree(c->block);
    c->block = p;
    c->block_bytes = need;
  }
  ctx_bind(h, c, q, mode, c->block, dtype);
  return HMAT_OK;
}

ChainMember chain_member(const Handle& h, const EvalContext* c, void* Y, bool y_f32, int64_t q) {
  ChainMember m{};
  m.tiles = h.tiles;
  m.tasks = h.tasks;
  m.entries = h.entries32;
  m.arena = h.arena32;
  m.w32 = c->w32;
  m.ws32 = c->ws32;
  m.us32 = c->us32;
  m.Y = Y;
  m.perm = h.perm;
  m.far_rows = h.far_rows;
  m.items = h.chain.items;
  m.q = q;
  m.bn = chain_bn(q);
  m.n_ct = (int32_t)((q + m.bn - 1) / m.bn);
  m.first_leaf = (int32_t)(h.n_leaves - 1);
  m.sync = ChainSync{h.chain.expect, c->chain_ctr + kChainCtrHead, h.status, (int32_t)h.n_nodes, m.first_leaf,
                     m.n_ct, 0};
  m.xv = q % 4 == 0 ? 1 : 0;
  m.y_f32 = y_f32 ? 1 : 0;
  m.n_items = (int32_t)h.chain.host.size();
  m.n_tiles = (int32_t)h.n_tiles;
  return m;
}

ChainLaunch chain_launch(const Handle& h, const EvalContext* c, int part, int32_t extra, uint64_t limit_ns) {
  ChainLaunch l{};
  l.item_begin = h.chain.begin[part];
  l.n_items = h.chain.count[part];
  l.ticket = c->chain_ctr + part;
  l.abort_flag = c->chain_ctr + 3;
  l.waits = h.chain.waits[part];
  l.extra = extra;
  l.limit_ns = limit_ns;
  l.status = h.status;
  return l;
}

ChainMember64 chain_member64(const Handle& h, const EvalContext* c, const double* W, double* Y, int64_t q) {
  ChainMember64 m{};
  m.tiles = h.tiles;
  m.tasks = h.tasks;
  m.entries = h.entries;
  m.arena = h.arena;
  m.W = W;
  m.ws = c->ws;
  m.us = c->us;
  m.Y = Y;
  m.perm = h.perm;
  m.far_rows = h.far_rows;
  m.items = h.chain64.items;
  m.q = q;
  m.first_leaf = (int32_t)(h.n_leaves - 1);
  // the column tiles are those of the shape the launch uses; the counters count them
  const TuneEntry* t = find_tuned(h, q, HMAT_MODE_FP64);
  const int shape = t && t->chain_shape >= 0 ? t->chain_shape : fp64_default_shape(q);
  const int bn = fp64_shape_columns(shape);
  m.n_ct = (int32_t)((q + bn - 1) / bn);
  m.sync = ChainSync{h.chain64.expect, c->chain_ctr + kChainCtrHead, h.status, (int32_t)h.n_nodes, m.first_leaf,
                     m.n_ct, 0};
  m.n_items = (int32_t)h.chain64.host.size();
  m.n_tiles = (int32_t)h.n_tiles;
  return m;
}

ChainLaunch chain_launch64(const Handle& h, const EvalContext* c, int32_t extra, uint64_t limit_ns) {
  ChainLaunch l{};
  l.item_begin = h.chain64.begin[0];
  l.n_items = h.chain64.count[0];
  l.ticket = c->chain_ctr;
  l.abort_flag = c->chain_ctr + 3;
  l.waits = h.chain64.waits[0];
  l.extra = extra;
  l.limit_ns = limit_ns;
  l.status = h.status;
  return l;
}

int chain_grid_cap(const Handle& h, int64_t q) {
  const TuneEntry* t = find_tuned(h, q, HMAT_MODE_MIXED);
  return t ? t->chain_grid : 0;
}

hmat_status eval_impl(Handle* h, EvalContext* c, const void* W, void* Y, int64_t q, int mode, int dtype,
                      cudaStream_t s) {
  const bool f32 = dtype == HMAT_DTYPE_F32;
  Handle::ProfRecord rec{};
  hmat_status st = HMAT_OK;
  cudaError_t e = cudaSuccess;
  if (mode == HMAT_MODE_MIXED) {
    int n_t;
    int64_t n_ct;
    mixed_tiles(*h, q, &n_t, &n_ct);
    if (!prof_begin(h, HMAT_PHASE_SPLIT, s, &rec)) return HMAT_ECUDA;
    e = f32 ? launch_split_f32(h->tc_near, (const float*)W, h->n_points * q, h->perm, q, n_t, (int)n_ct, c->wmax,
                               c->wsplit, c->w32, s)
            : launch_split_f64(h->tc_near, (const double*)W, h->n_points * q, h->perm, q, n_t, (int)n_ct, c->wmax,
                               c->wsplit, c->w32, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (!prof_end(h, rec, s)) return HMAT_ECUDA;
    // the far chain on the side stream (beside the near field), or on s when profiling
    // serialised (each launch's events then time that launch alone)
    const bool serial = h->profiling == 2;
    cudaStream_t far = serial ? s : c->aux;
    if (!serial &&
        (cudaEventRecord(c->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(c->aux, c->ev_fork, 0) != cudaSuccess))
      return HMAT_ECUDA;
    ChainMember cm = chain_member(*h, c, Y, f32, q);
    auto chain = [&](int part, int32_t kind, cudaStream_t strm) -> hmat_status {
      if (h->chain.count[part] == 0) return HMAT_OK;
      if (!prof_begin(h, kind, strm, &rec)) return HMAT_ECUDA;
      e = launch_chain(cm, chain_launch(*h, c, part, 0, kChainWaitNs), chain_grid_cap(*h, q), strm);
      if (e != cudaSuccess) return cuda_status(e);
      return prof_end(h, rec, strm) ? HMAT_OK : HMAT_ECUDA;
    };
    if ((e = cudaMemsetAsync(c->chain_ctr, 0, (size_t)h->chain.n_ctr * 4, far)) != cudaSuccess) return cuda_status(e);
    // upward pass (with the FP32 coupling: also the coupling and the downward transfers)
    if ((st = chain(0, HMAT_PHASE_FAR_UP, far)) != HMAT_OK) return st;
    if (h->tc_coupling && h->tc_far.n_work > 0) {
      if (!prof_begin(h, HMAT_PHASE_SPLIT, far, &rec)) return HMAT_ECUDA;
      e = launch_split_f32(h->tc_far, c->ws32, std::max<int64_t>(h->sum_rank, 1) * q, nullptr, q, n_t, (int)n_ct,
                           c->smax, c->ssplit, nullptr, far);
      if (e != cudaSuccess) return cuda_status(e);
      if (!prof_end(h, rec, far)) return HMAT_ECUDA;
      if (!prof_begin(h, HMAT_PHASE_COUPLING, far, &rec)) return HMAT_ECUDA;
      e = launch_tc_far(h->tc_far, c->ssplit, c->smax, c->us32, q, n_t, (int)n_ct, h->status, far);
      if (e != cudaSuccess) return cuda_status(e);
      if (!prof_end(h, rec, far)) return HMAT_ECUDA;
    }
    // downward transfers after the tensor-core coupling
    if ((st = chain(1, HMAT_PHASE_FAR_DOWN, far)) != HMAT_OK) return st;
    if (!serial && cudaEventRecord(c->ev_join, c->aux) != cudaSuccess) return HMAT_ECUDA;
    if (!prof_begin(h, HMAT_PHASE_NEAR, s, &rec)) return HMAT_ECUDA;
    e = launch_tc_near(h->tc_near, c->wsplit, c->wmax, h->perm, Y, f32, q, n_t, (int)n_ct, h->status, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (!prof_end(h, rec, s)) return HMAT_ECUDA;
    if (!serial && cudaStreamWaitEvent(s, c->ev_join, 0) != cudaSuccess) return HMAT_ECUDA;
    // downward leaf step: adds into Y after the near field has written it
    return chain(2, HMAT_PHASE_DOWN_LEAF, s);
  }
  // FP64 mode: FP32 W is widened into the workspace and Y rounded from it at the end
  const double* W64 = f32 ? c->w64 : (const double*)W;
  double* Y64 = f32 ? c->y64 : (double*)Y;
  if (f32 && (e = launch_widen((const float*)W, c->w64, h->n_points * q, s)) != cudaSuccess) return cuda_status(e);
  const TuneEntry* tuned = find_tuned(*h, q, HMAT_MODE_FP64);
  // the near field, one launch per row-tile size; then the far field as one persistent launch
  for (size_t i = 0; i < h->phases.size(); ++i) {
    const Phase& ph = h->phases[i];
    if (ph.kind != PH_NEAR) continue;
    const double* X = ph.x == MAT_USER ? W64 : (ph.x == MAT_SKEL_W ? c->ws : c->us);
    double* Yd = ph.y == MAT_USER ? Y64 : (ph.y == MAT_SKEL_W ? c->ws : c->us);
    const int64_t* xm = phase_x_map(*h, ph);
    const int64_t* ym = ph.y == MAT_USER ? h->perm : nullptr;
    const int shape = tuned && i < tuned->shape.size() ? tuned->shape[i] : -1;
    if (!prof_begin(h, (int32_t)ph.kind, s, &rec)) return HMAT_ECUDA;
    e = launch_fp64_phase(*h, ph, X, xm, Yd, ym, q, shape, -1, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (!prof_end(h, rec, s)) return HMAT_ECUDA;
  }
  if (h->chain64.count[0] > 0) {
    if ((e = cudaMemsetAsync(c->chain_ctr, 0, (size_t)h->chain64.n_ctr * 4, s)) != cudaSuccess) return cuda_status(e);
    const ChainMember64 cm = chain_member64(*h, c, W64, Y64, q);
    const int shape = tuned && tuned->chain_shape >= 0 ? tuned->chain_shape : fp64_default_shape(q);
    if (!prof_begin(h, HMAT_PHASE_FAR_UP, s, &rec)) return HMAT_ECUDA;
    e = launch_chain64(cm, chain_launch64(*h, c, 0, kChainWaitNs), shape, tuned ? tuned->chain_grid : 0, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (!prof_end(h, rec, s)) return HMAT_ECUDA;
  }
  if (f32) return cuda_status(launch_narrow(c->y64, (float*)Y, h->n_points * q, s));
  return HMAT_OK;
}

}  // namespace hmat

using namespace hmat;

extern "C" hmat_status hmat_reserve(hmat_t h, int64_t q_max) {
  if (!h || q_max < 0) return HMAT_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (dev != h->device) return HMAT_EINVAL;
  if (q_max == 0) return HMAT_OK;
  const int mode = h->has_mixed && (!h->has_fp64 || ctx_bytes(*h, q_max, HMAT_MODE_MIXED) >
                                                          ctx_bytes(*h, q_max, HMAT_MODE_FP64))
                       ? HMAT_MODE_MIXED
                       : HMAT_MODE_FP64;
  return ctx_reserve(*h, h->ctx, q_max, mode);
}

extern "C" hmat_status hmat_eval_typed(hmat_t h, const void* W, void* Y, int64_t q, int mode, int dtype,
                                       void* stream) {
  hmat_status st = check_call(h, W, Y, q, mode, dtype);
  if (st != HMAT_OK || q == 0 || h->n_points == 0) return st;
  if ((st = ctx_reserve(*h, h->ctx, q, mode, dtype)) != HMAT_OK) return st;
  return eval_impl(h, h->ctx, W, Y, q, mode, dtype, (cudaStream_t)stream);
}

extern "C" hmat_status hmat_eval(hmat_t h, const double* W, double* Y, int64_t q, int mode, void* stream) {
  return hmat_eval_typed(h, W, Y, q, mode, HMAT_DTYPE_F64, stream);
}

extern "C" hmat_status hmat_eval_host_typed(hmat_t h, const void* W, void* Y, int64_t q, int mode, int dtype,
                                            void* stream) {
  if (!h || q < 0) return HMAT_EINVAL;
  if (dtype != HMAT_DTYPE_F64 && dtype != HMAT_DTYPE_F32) return HMAT_EINVAL;
  if (mode != HMAT_MODE_FP64 && mode != HMAT_MODE_MIXED) return HMAT_EUNSUPPORTED;
  if ((mode == HMAT_MODE_MIXED && !h->has_mixed) || (mode == HMAT_MODE_FP64 && !h->has_fp64))
    return HMAT_EUNSUPPORTED;
  if (q == 0 || h->n_points == 0) return HMAT_OK;
  if (!W || !Y) return HMAT_EINVAL;
  EvalContext* c = h->ctx;
  const int64_t es = dtype_bytes(dtype);
  const int64_t bytes = h->n_points * q * es;
  if (bytes > c->host_cap) {
    void *w = nullptr, *y = nullptr;
    cudaError_t e = cudaMalloc(&w, (size_t)bytes);
    if (e == cudaSuccess) e = cudaMalloc(&y, (size_t)bytes);
    if (e != cudaSuccess) {
      cudaFree(w);
      cudaGetLastError();
      return cuda_status(e);
    }
    cudaDeviceSynchronize();
    cudaFree(c->host_w);
    cudaFree(c->host_y);
    c->host_w = w;
    c->host_y = y;
    c->host_cap = bytes;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (mode == HMAT_MODE_MIXED && q >= 2 * kHostSplitMinQ) {
    // Two column groups, the copies on a stream of their own: the second group's upload
    // runs under the first group's evaluation and the first group's download under the
    // second's (the mixed evaluation takes milliseconds, like the copies).
    if (!c->copy) {
      cudaError_t e = cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking);
      for (cudaEvent_t& ev : c->ev_copy)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_status(e);
    }
    const int64_t n = h->n_points;
    const int64_t qa = std::min<int64_t>(q - 16, (q / 2 + 15) / 16 * 16), qb = q - qa;
    char* wa = (char*)c->host_w;
    char* wb = wa + n * qa * es;
    char* ya = (char*)c->host_y;
    char* yb = ya + n * qa * es;
    cudaEvent_t* ev = c->ev_copy;
    const size_t pitch = (size_t)(q * es);
    const char* Wc = (const char*)W;
    char* Yc = (char*)Y;
    cudaError_t e = cudaEventRecord(ev[0], s);  // earlier work on s that used these buffers
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy, ev[0], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(wa, qa * es, Wc, pitch, qa * es, n, cudaMemcpyHostToDevice, c->copy);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->copy);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(wb, qb * es, Wc + qa * es, pitch, qb * es, n, cudaMemcpyHostToDevice, c->copy);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], c->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
    if (e != cudaSuccess) return cuda_status(e);
    hmat_status st = hmat_eval_typed(h, wa, ya, qa, mode, dtype, stream);
    if (st != HMAT_OK) return st;
    if ((e = cudaEventRecord(ev[3], s)) != cudaSuccess || (e = cudaStreamWaitEvent(s, ev[2], 0)) != cudaSuccess)
      return cuda_status(e);
    if ((st = hmat_eval_typed(h, wb, yb, qb, mode, dtype, stream)) != HMAT_OK) return st;
    e = cudaEventRecord(ev[4], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy, ev[3], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Yc, pitch, ya, qa * es, qa * es, n, cudaMemcpyDeviceToHost, c->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy, ev[4], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Yc + qa * es, pitch, yb, qb * es, qb * es, n, cudaMemcpyDeviceToHost, c->copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->copy);
    return cuda_status(e);
  }
  cudaError_t e = cudaMemcpyAsync(c->host_w, W, (size_t)bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e);
  hmat_status st = hmat_eval_typed(h, c->host_w, c->host_y, q, mode, dtype, stream);
  if (st != HMAT_OK) return st;
  e = cudaMemcpyAsync(Y, c->host_y, (size_t)bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e);
}

extern "C" hmat_status hmat_eval_host(hmat_t h, const double* W, double* Y, int64_t q, int mode, void* stream) {
  return hmat_eval_host_typed(h, W, Y, q, mode, HMAT_DTYPE_F64, stream);
}

extern "C" hmat_status hmat_selftest_chain_timeout(hmat_t h, int64_t q, int mode, int64_t limit_ns, void* stream) {
  if (!h || q <= 0 || limit_ns <= 0 || limit_ns > 10000000000LL) return HMAT_EINVAL;
  if (mode != HMAT_MODE_FP64 && mode != HMAT_MODE_MIXED) return HMAT_EUNSUPPORTED;
  if ((mode == HMAT_MODE_MIXED && !h->has_mixed) || (mode == HMAT_MODE_FP64 && !h->has_fp64))
    return HMAT_EUNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (dev != h->device) return HMAT_EINVAL;
  const ChainPlan& plan = mode == HMAT_MODE_MIXED ? h->chain : h->chain64;
  if (plan.count[0] == 0) return HMAT_EINVAL;  // no far field: nothing to wait on
  hmat_status st = ctx_reserve(*h, h->ctx, q, mode);
  if (st != HMAT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(h->ctx->chain_ctr, 0, (size_t)plan.n_ctr * 4, s);
  if (e != cudaSuccess) return cuda_status(e);
  // the workspaces are not filled: the launch waits before it reads or writes any of them
  if (mode == HMAT_MODE_MIXED)
    return cuda_status(launch_chain(chain_member(*h, h->ctx, nullptr, false, q),
                                    chain_launch(*h, h->ctx, 0, 1, (uint64_t)limit_ns), 0, s));
  return cuda_status(launch_chain64(chain_member64(*h, h->ctx, nullptr, nullptr, q),
                                    chain_launch64(*h, h->ctx, 1, (uint64_t)limit_ns), fp64_default_shape(q), 0, s));
}

extern "C" hmat_status hmat_selftest_device_check(hmat_t h, int64_t q, int mode, void* stream) {
  if (!h || q <= 0) return HMAT_EINVAL;
  if (mode != HMAT_MODE_FP64 && mode != HMAT_MODE_MIXED) return HMAT_EUNSUPPORTED;
  if ((mode == HMAT_MODE_MIXED && !h->has_mixed) || (mode == HMAT_MODE_FP64 && !h->has_fp64))
    return HMAT_EUNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (dev != h->device) return HMAT_EINVAL;
  const ChainPlan& plan = mode == HMAT_MODE_MIXED ? h->chain : h->chain64;
  if (plan.host.empty()) return HMAT_EINVAL;  // no far field: no chain to check
  hmat_status st = ctx_reserve(*h, h->ctx, q, mode);
  if (st != HMAT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(h->ctx->chain_ctr, 0, (size_t)plan.n_ctr * 4, s);
  if (e != cudaSuccess) return cuda_status(e);
  // one ticket whose item index lies just past the item array: the launch's own index
  // check must catch it before any read
  if (mode == HMAT_MODE_MIXED) {
    ChainLaunch l = chain_launch(*h, h->ctx, 0, 0, kChainWaitNs);
    l.item_begin = (int32_t)plan.host.size();
    l.n_items = 1;
    ChainMember m = chain_member(*h, h->ctx, nullptr, false, q);
    m.n_ct = 1;
    m.sync.n_ct = 1;
    return cuda_status(launch_chain(m, l, 1, s));
  }
  ChainLaunch l = chain_launch64(*h, h->ctx, 0, kChainWaitNs);
  l.item_begin = (int32_t)plan.host.size();
  l.n_items = 1;
  ChainMember64 m = chain_member64(*h, h->ctx, nullptr, nullptr, q);
  m.n_ct = 1;
  m.sync.n_ct = 1;
  return cuda_status(launch_chain64(m, l, fp64_default_shape(q), 1, s));
}

extern "C" hmat_status hmat_profile(hmat_t h, int enable) {
  if (!h) return HMAT_EINVAL;
  for (auto& r : h->prof) {
    h->event_pool.push_back(r.start);
    h->event_pool.push_back(r.stop);
  }
  h->prof.clear();
  h->profiling = enable == 2 ? 2 : (enable != 0 ? 1 : 0);
  return HMAT_OK;
}

extern "C" hmat_status hmat_phase_times(hmat_t h, double* ms, int64_t* launches, int n) {
  if (!h || n < 0 || (n > 0 && (!ms || !launches))) return HMAT_EINVAL;
  for (int k = 0; k < n; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  hmat_status st = HMAT_OK;
  for (auto& r : h->prof) {
    float t = 0.0f;
    cudaError_t e = cudaEventSynchronize(r.stop);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.start, r.stop);
    if (e != cudaSuccess) st = HMAT_ECUDA;
    if (r.kind < n) {
      ms[r.kind] += t;
      launches[r.kind] += 1;
    }
    h->event_pool.push_back(r.start);
    h->event_pool.push_back(r.stop);
  }
  h->prof.clear();
  return st;
}
