// Batched evaluation: many HMatrices of uneven size, rank and q evaluated together,
// captured once as a CUDA graph and replayed with one launch.
//
// Every step of the evaluation is one launch over all members (a flattened work list
// with a member table and per-member block or ticket ranges), so a batch replays about
// ten kernels however many members it has:
//   mixed mode  - max |W| and the W split of every member; the far chain's upward pass
//                 (with the FP32 couplings and downward transfers) of every member in one
//                 persistent launch; for the members whose coupling runs on the tensor
//                 cores the w split, the coupling and the downward transfers; the
//                 tensor-core near field of every member; the downward leaf step;
//   FP64 mode   - the near field per member (its tuned column tile, on parallel graph
//                 branches), then the far field of every member in one persistent
//                 chain launch per column tile width.
// Each member's result is bitwise the one it gets alone: the same tiles summed in the
// same order, with its own workspaces and counters. hmat_batch_autotune may instead pick
// the branched schedule (each member's own evaluation as a graph branch: more launches,
// which overlap one another) when it replays faster.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "hmat_internal.h"

using namespace hmat;

namespace {

constexpr int kBranches = 8;  // FP64 near-field launches spread over this many graph branches
constexpr int kTickets = 64;  // ticket counters of the batch's chain launches; the last is the abort flag

int64_t al256(int64_t x) { return (x + 255) / 256 * 256; }

// One chain launch's tickets over the members, ordered by stage (then member, item,
// column tile): entry k of `items_of` lists member k's items of this launch.
struct TicketSrc {
  int32_t member;             // index into the launch's member table
  const ChainPlan* plan;
  int32_t begin, count;
  uint32_t waits;
  int32_t n_ct;
  int levels;
};
std::vector<ChainTicket> ticket_list(const std::vector<TicketSrc>& src, int max_levels) {
  struct Key {
    int stage, member, item, ct;
  };
  std::vector<std::pair<Key, ChainTicket>> all;
  for (const TicketSrc& t : src)
    for (int32_t i = t.begin; i < t.begin + t.count; ++i) {
      const int st = chain_stage(t.plan->host[i], t.levels, max_levels);
      for (int32_t c = 0; c < t.n_ct; ++c) all.push_back({Key{st, t.member, i, c}, ChainTicket{t.member, i, c, t.waits}});
    }
  std::stable_sort(all.begin(), all.end(), [](const auto& a, const auto& b) {
    if (a.first.stage != b.first.stage) return a.first.stage < b.first.stage;
    if (a.first.member != b.first.member) return a.first.member < b.first.member;
    if (a.first.item != b.first.item) return a.first.item < b.first.item;
    return a.first.ct < b.first.ct;
  });
  std::vector<ChainTicket> out;
  out.reserve(all.size());
  for (auto& p : all) out.push_back(p.second);
  return out;
}

}  // namespace

namespace hmat {

// Stages: the upward pass from the leaves up (each level's coupling right after it),
// then the downward transfers from the top down, then the downward leaf step. Every
// dependency of an item (children's upward items, its level's upward items, its own
// and its children's coupling, its parent's downward items) has a lower stage.
int chain_stage(const ChainItem& it, int levels, int max_levels) {
  switch (it.kind) {
    case CK_UP: return 2 * (levels - it.level);
    case CK_CPL: return 2 * (levels - it.level) + 1;
    case CK_DN: return 2 * max_levels + 2 + it.level;
    default: return 3 * max_levels + 3;
  }
}

}  // namespace hmat

struct hmat_batch {
  int device = -1;
  int mode = HMAT_MODE_FP64;
  std::vector<hmat_t> handles;
  std::vector<EvalContext*> ctx;      // per member: workspaces bound into `block`
  cudaStream_t capture = nullptr;     // the graph is captured on this stream (never the legacy default stream)
  cudaStream_t branch[kBranches] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kBranches] = {};
  uint8_t* block = nullptr;           // workspaces, counters and device tables of the captured graph
  int64_t block_bytes = 0;
  int kernels = 0;                    // kernel launches in the captured graph
  int chain_grid = 0;                 // CTAs of the chain launches (0: every resident CTA; hmat_batch_autotune)
  int branched = 0;                   // 1: every member's evaluation as a graph branch of its own (hmat_batch_autotune)
  int default_widths = 0;             // 1: mixed members at their default tensor-core column width, not
                                      // their own tuned one (hmat_batch_autotune)
  std::vector<cudaStream_t> member_stream;  // branched schedule: one stream per member
  std::vector<cudaEvent_t> member_join;
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
  for (cudaStream_t s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev_join)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t st : b->member_stream) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->member_join) cudaEventDestroy(ev);
  for (EvalContext* c : b->ctx) ctx_destroy(c);  // workspaces bound to b->block: only the streams are theirs
  cudaFree(b->block);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

// Host images of the device tables, laid out one after another in the batch's block.
struct Tables {
  std::vector<uint8_t> bytes;
  template <class T>
  int64_t add(const std::vector<T>& v) {
    const int64_t off = al256((int64_t)bytes.size());
    bytes.resize(off + std::max<size_t>(v.size(), 1) * sizeof(T), 0);
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

// Bind every member's workspaces into one block (allocated here, outside any capture)
// with the small per-member words that start at zero (max |W|, max |w|, the chains'
// counters) gathered at its front after the batch's own tickets, so that one memset
// clears them all; the device tables follow the workspaces.
hmat_status bind_members(hmat_batch* b, const int64_t* q, int dtype, int64_t table_bytes, int64_t* small_bytes,
                         int64_t* table_off) {
  const int n = (int)b->handles.size();
  const bool mixed = b->mode == HMAT_MODE_MIXED;
  int64_t small = al256(kTickets * 4);
  std::vector<int64_t> small_off(n), ws_off(n);
  for (int i = 0; i < n; ++i) {
    const Handle& h = *b->handles[i];
    small_off[i] = small;
    const int64_t n_ctr = mixed ? h.chain.n_ctr : h.chain64.n_ctr;
    small += al256(16 + n_ctr * 4);
  }
  int64_t off = small;
  for (int i = 0; i < n; ++i) {
    ws_off[i] = off;
    if (q[i] > 0 && b->handles[i]->n_points > 0) off += al256(ctx_bytes(*b->handles[i], q[i], b->mode, dtype));
  }
  const int64_t need = off + al256(table_bytes);
  if (need > b->block_bytes) {
    uint8_t* p = nullptr;
    cudaError_t e = cudaMalloc((void**)&p, (size_t)need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
    cudaDeviceSynchronize();  // an earlier replay may still use the old block
    cudaFree(b->block);
    b->block = p;
    b->block_bytes = need;
  }
  for (int i = 0; i < n; ++i) {
    EvalContext* c = b->ctx[i];
    if (q[i] == 0 || b->handles[i]->n_points == 0) continue;
    ctx_bind(*b->handles[i], c, q[i], b->mode, b->block + ws_off[i], dtype);
    uint8_t* sm = b->block + small_off[i];
    if (mixed) {
      c->wmax = (unsigned long long*)sm;
      c->smax = (unsigned long long*)(sm + 8);
    }
    c->chain_ctr = (int32_t*)(sm + 16);
  }
  *small_bytes = small;
  *table_off = off;
  return HMAT_OK;
}

// The device tables of a mixed-mode batch (built twice: for the sizes, then with the
// workspace pointers).
struct MixedTables {
  std::vector<AbsJob> absW, absS;
  std::vector<SplitJob> splW, splS;
  std::vector<TcArgs> near, far;
  std::vector<int64_t> endAbsW, endAbsS, endSplW, endSplS, endNear, endFar;
  std::vector<ChainMember> mem;               // the chain launches' member table
  std::vector<ChainTicket> listA, listB, listC;  // their tickets, by stage across members
  int64_t off[16] = {};

  void build(hmat_batch* b, const void* const* W, void* const* Y, const int64_t* q, bool f32,
             const std::vector<int>& live) {
    *this = MixedTables{};
    int64_t bAW = 0, bAS = 0, bSW = 0, bSS = 0, bN = 0, bF = 0;
    std::vector<TicketSrc> srcA, srcB, srcC;
    int max_levels = 0;
    for (int i : live) max_levels = std::max(max_levels, (int)b->handles[i]->levels);
    for (int i : live) {
      Handle* h = b->handles[i];
      EvalContext* c = b->ctx[i];
      int n_t;
      int64_t n_ct;
      if (b->default_widths) {
        n_t = mixed_nt_candidates(q[i])[0];
        n_ct = (q[i] + n_t - 1) / n_t;
      } else {
        mixed_tiles(*h, q[i], &n_t, &n_ct);
      }
      const int nct = (int)n_ct;
      const int64_t r = std::max<int64_t>(h->sum_rank, 1);
      absW.push_back(AbsJob{W[i], h->n_points * q[i], c->wmax});
      endAbsW.push_back(bAW += absmax_blocks(h->n_points * q[i]));
      splW.push_back(SplitJob{h->tc_near.dev, W[i], h->perm, q[i], n_t, nct, c->wmax, c->wsplit, c->w32});
      endSplW.push_back(bSW += h->tc_near.n_chunks * nct);
      near.push_back(TcArgs{h->tc_near.dev, c->wsplit, c->wmax, h->perm, Y[i], q[i], n_t, nct, h->status,
                            f32 ? 1 : 0});
      endNear.push_back(bN += h->tc_near.n_work * nct);
      if (h->tc_coupling && h->tc_far.n_work > 0) {
        absS.push_back(AbsJob{c->ws32, r * q[i], c->smax});
        endAbsS.push_back(bAS += absmax_blocks(r * q[i]));
        splS.push_back(SplitJob{h->tc_far.dev, c->ws32, nullptr, q[i], n_t, nct, c->smax, c->ssplit, nullptr});
        endSplS.push_back(bSS += h->tc_far.n_chunks * nct);
        far.push_back(TcArgs{h->tc_far.dev, c->ssplit, c->smax, nullptr, c->us32, q[i], n_t, nct, h->status, 0});
        endFar.push_back(bF += h->tc_far.n_work * nct);
      }
      const ChainMember cm = chain_member(*h, c, Y[i], f32, q[i]);
      const int32_t mi = (int32_t)mem.size();
      mem.push_back(cm);
      const ChainPlan& cp = h->chain;
      srcA.push_back(TicketSrc{mi, &cp, cp.begin[0], cp.count[0], cp.waits[0], cm.n_ct, h->levels});
      srcB.push_back(TicketSrc{mi, &cp, cp.begin[1], cp.count[1], cp.waits[1], cm.n_ct, h->levels});
      srcC.push_back(TicketSrc{mi, &cp, cp.begin[2], cp.count[2], cp.waits[2], cm.n_ct, h->levels});
    }
    listA = ticket_list(srcA, max_levels);
    listB = ticket_list(srcB, max_levels);
    listC = ticket_list(srcC, max_levels);
  }
  Tables layout() {
    Tables t;
    int k = 0;
    off[k++] = t.add(absW); off[k++] = t.add(absS); off[k++] = t.add(splW); off[k++] = t.add(splS);
    off[k++] = t.add(near); off[k++] = t.add(far);
    off[k++] = t.add(endAbsW); off[k++] = t.add(endAbsS); off[k++] = t.add(endSplW); off[k++] = t.add(endSplS);
    off[k++] = t.add(endNear); off[k++] = t.add(endFar);
    off[k++] = t.add(mem);
    off[k++] = t.add(listA); off[k++] = t.add(listB); off[k++] = t.add(listC);
    return t;
  }
};

int64_t last_or_zero(const std::vector<int64_t>& v) { return v.empty() ? 0 : v.back(); }

// Capture the mixed mode: about ten launches for the whole batch.
hmat_status capture_mixed(hmat_batch* b, const void* const* W, void* const* Y, const int64_t* q, int dtype) {
  const int n = (int)b->handles.size();
  const bool f32 = dtype == HMAT_DTYPE_F32;
  std::vector<int> live;
  for (int i = 0; i < n; ++i)
    if (q[i] > 0 && b->handles[i]->n_points > 0) live.push_back(i);
  MixedTables mt;
  mt.build(b, W, Y, q, f32, live);  // sizes only (the workspaces are not bound yet)
  int64_t small = 0, table_off = 0;
  hmat_status st = bind_members(b, q, dtype, (int64_t)mt.layout().bytes.size(), &small, &table_off);
  if (st != HMAT_OK) return st;
  mt.build(b, W, Y, q, f32, live);
  const Tables t = mt.layout();
  uint8_t* tb = b->block + table_off;
  cudaError_t e = cudaMemcpy(tb, t.bytes.data(), t.bytes.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  auto dp = [&](int k) { return (const void*)(tb + mt.off[k]); };
  int32_t* tickets = (int32_t*)b->block;
  auto chain_args = [&](int list_k, const std::vector<ChainTicket>& list, bool free_run) {
    return ChainMulti<ChainMember>{(const ChainMember*)dp(12), nullptr, (int32_t)mt.mem.size(), free_run ? 1 : 0,
                                   (int64_t)list.size(), (const ChainTicket*)dp(list_k)};
  };
  auto launch_of = [&](int k) {
    ChainLaunch l{};
    l.ticket = tickets + k;
    l.abort_flag = tickets + kTickets - 1;
    l.limit_ns = kChainWaitNs;
    l.status = live.empty() ? nullptr : b->handles[live[0]]->status;
    return l;
  };
  const int nW = (int)mt.absW.size(), nS = (int)mt.absS.size();
  cudaStream_t s = b->capture, aux = b->branch[0];
  int kernels = 0;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  auto step = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  step(cudaMemsetAsync(b->block, 0, (size_t)small, s));
  step(launch_absmax_multi(f32, (const AbsJob*)dp(0), (const int64_t*)dp(6), nW, last_or_zero(mt.endAbsW), s));
  step(launch_split_multi(f32, (const SplitJob*)dp(2), (const int64_t*)dp(8), nW, last_or_zero(mt.endSplW), s));
  kernels += 2;
  // the far field on a side branch, beside the near field
  step(cudaEventRecord(b->ev_fork, s));
  step(cudaStreamWaitEvent(aux, b->ev_fork, 0));
  if (!mt.listA.empty()) {
    step(launch_chain_multi(chain_args(13, mt.listA, false), launch_of(0), b->chain_grid, aux));
    ++kernels;
  }
  if (nS > 0) {
    step(launch_absmax_multi(true, (const AbsJob*)dp(1), (const int64_t*)dp(7), nS, last_or_zero(mt.endAbsS), aux));
    step(launch_split_multi(true, (const SplitJob*)dp(3), (const int64_t*)dp(9), nS, last_or_zero(mt.endSplS), aux));
    step(launch_tc_multi(true, (const TcArgs*)dp(5), (const int64_t*)dp(11), nS, last_or_zero(mt.endFar), aux));
    kernels += 3;
  }
  if (!mt.listB.empty()) {
    step(launch_chain_multi(chain_args(14, mt.listB, false), launch_of(1), b->chain_grid, aux));
    ++kernels;
  }
  step(cudaEventRecord(b->ev_join[0], aux));
  step(launch_tc_multi(false, (const TcArgs*)dp(4), (const int64_t*)dp(10), nW, last_or_zero(mt.endNear), s));
  ++kernels;
  step(cudaStreamWaitEvent(s, b->ev_join[0], 0));
  if (!mt.listC.empty()) {
    step(launch_chain_multi(chain_args(15, mt.listC, true), launch_of(2), 0, s));
    ++kernels;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s, &graph);
  if (e == cudaSuccess) e = ee;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_status(e);
  }
  b->kernels = kernels;
  return HMAT_OK;
}

// The device tables of an FP64 batch: per column shape of the far chain, its members
// and its tickets by stage across them.
struct Fp64Tables {
  std::map<int, std::vector<int>> by_shape;
  std::vector<int64_t> off;  // per group: members, tickets, ticket count

  Tables build(hmat_batch* b, const void* const* W, void* const* Y, const int64_t* q, bool f32) {
    Tables t;
    off.clear();
    for (auto& kv : by_shape) {
      std::vector<ChainMember64> mem;
      std::vector<TicketSrc> src;
      int max_levels = 0;
      for (int i : kv.second) max_levels = std::max(max_levels, (int)b->handles[i]->levels);
      for (int i : kv.second) {
        Handle* h = b->handles[i];
        EvalContext* c = b->ctx[i];
        const double* W64 = f32 ? c->w64 : (const double*)W[i];
        double* Y64 = f32 ? c->y64 : (double*)Y[i];
        const ChainMember64 m = chain_member64(*h, c, W64, Y64, q[i]);
        const ChainPlan& cp = h->chain64;
        src.push_back(TicketSrc{(int32_t)mem.size(), &cp, cp.begin[0], cp.count[0], cp.waits[0], m.n_ct, h->levels});
        mem.push_back(m);
      }
      const std::vector<ChainTicket> list = ticket_list(src, max_levels);
      off.push_back(t.add(mem));
      off.push_back(t.add(list));
      off.push_back((int64_t)list.size());
    }
    return t;
  }
};

// Capture the FP64 mode: the members' near fields on parallel branches, then one
// persistent far-chain launch per column tile width.
hmat_status capture_fp64(hmat_batch* b, const void* const* W, void* const* Y, const int64_t* q, int dtype) {
  const int n = (int)b->handles.size();
  const bool f32 = dtype == HMAT_DTYPE_F32;
  std::vector<int> live;
  for (int i = 0; i < n; ++i)
    if (q[i] > 0 && b->handles[i]->n_points > 0) live.push_back(i);
  Fp64Tables ft;
  for (int i : live) {  // far chains grouped by their column shape (a launch has one)
    const Handle& h = *b->handles[i];
    if (h.chain64.count[0] == 0) continue;
    const TuneEntry* te = find_tuned(h, q[i], HMAT_MODE_FP64);
    ft.by_shape[te && te->chain_shape >= 0 ? te->chain_shape : fp64_default_shape(q[i])].push_back(i);
  }
  if ((int)ft.by_shape.size() >= kTickets) return HMAT_EUNSUPPORTED;
  int64_t small = 0, table_off = 0;
  hmat_status st = bind_members(b, q, dtype, (int64_t)ft.build(b, W, Y, q, f32).bytes.size(), &small, &table_off);
  if (st != HMAT_OK) return st;
  const Tables t = ft.build(b, W, Y, q, f32);
  uint8_t* tb = b->block + table_off;
  cudaError_t e = cudaMemcpy(tb, t.bytes.data(), t.bytes.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  int32_t* tickets = (int32_t*)b->block;
  cudaStream_t s = b->capture;
  int kernels = 0;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  auto step = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  step(cudaMemsetAsync(b->block, 0, (size_t)small, s));
  step(cudaEventRecord(b->ev_fork, s));
  int k = 0;
  for (int i : live) {  // near fields, round-robin over the branches
    Handle* h = b->handles[i];
    EvalContext* c = b->ctx[i];
    cudaStream_t br = b->branch[k % kBranches];
    if (k < kBranches) step(cudaStreamWaitEvent(br, b->ev_fork, 0));
    ++k;
    if (f32) {
      step(launch_widen((const float*)W[i], c->w64, h->n_points * q[i], br));
      ++kernels;
    }
    const double* W64 = f32 ? c->w64 : (const double*)W[i];
    double* Y64 = f32 ? c->y64 : (double*)Y[i];
    const TuneEntry* te = find_tuned(*h, q[i], HMAT_MODE_FP64);
    for (size_t p = 0; p < h->phases.size(); ++p) {
      const Phase& ph = h->phases[p];
      if (ph.kind != PH_NEAR) continue;
      const int shape = te && p < te->shape.size() ? te->shape[p] : -1;
      step(launch_fp64_phase(*h, ph, W64, phase_x_map(*h, ph), Y64, h->perm, q[i], shape, -1, br));
      ++kernels;
    }
  }
  for (int j = 0; j < std::min(k, kBranches); ++j) {
    step(cudaEventRecord(b->ev_join[j], b->branch[j]));
    step(cudaStreamWaitEvent(s, b->ev_join[j], 0));
  }
  int g = 0;
  for (auto& kv : ft.by_shape) {
    ChainLaunch l{};
    l.ticket = tickets + g;
    l.abort_flag = tickets + kTickets - 1;
    l.limit_ns = kChainWaitNs;
    l.status = b->handles[kv.second[0]]->status;
    const ChainMulti<ChainMember64> mm{(const ChainMember64*)(tb + ft.off[3 * g]), nullptr,
                                       (int32_t)kv.second.size(), 0, ft.off[3 * g + 2],
                                       (const ChainTicket*)(tb + ft.off[3 * g + 1])};
    step(launch_chain64_multi(mm, l, kv.first, b->chain_grid, s));
    ++kernels;
    ++g;
  }
  if (f32)
    for (int i : live) {
      step(launch_narrow(b->ctx[i]->y64, (float*)Y[i], b->handles[i]->n_points * q[i], s));
      ++kernels;
    }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s, &graph);
  if (e == cudaSuccess) e = ee;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_status(e);
  }
  b->kernels = kernels;
  return HMAT_OK;
}

// Capture every member's evaluation (the single-handle path) as a branch of its own,
// forked from the capture stream: many small launches that overlap one another.
hmat_status capture_branched(hmat_batch* b, const void* const* W, void* const* Y, const int64_t* q, int dtype) {
  const int n = (int)b->handles.size();
  int64_t small = 0, table_off = 0;
  hmat_status st = bind_members(b, q, dtype, 0, &small, &table_off);
  if (st != HMAT_OK) return st;
  std::vector<int> profiling(n);
  for (int i = 0; i < n; ++i) {
    profiling[i] = b->handles[i]->profiling;
    b->handles[i]->profiling = 0;
  }
  int kernels = 0;
  cudaStream_t s = b->capture;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, s);
  for (int i = 0; i < n && e == cudaSuccess && st == HMAT_OK; ++i) {
    if (q[i] == 0 || b->handles[i]->n_points == 0) continue;
    e = cudaStreamWaitEvent(b->member_stream[i], b->ev_fork, 0);
    if (e != cudaSuccess) break;
    st = eval_impl(b->handles[i], b->ctx[i], W[i], Y[i], q[i], b->mode, dtype, b->member_stream[i]);
    if (st != HMAT_OK) break;
    kernels += b->mode == HMAT_MODE_MIXED ? 8 : 3;  // about: split (2), chains, [coupling], near, leaf chain
    e = cudaEventRecord(b->member_join[i], b->member_stream[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->member_join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s, &graph);
  for (int i = 0; i < n; ++i) b->handles[i]->profiling = profiling[i];
  if (e == cudaSuccess) e = ee;
  if (st == HMAT_OK && e == cudaSuccess) {
    size_t nodes = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nodes) == cudaSuccess) {
      std::vector<cudaGraphNode_t> all(nodes);
      if (nodes && cudaGraphGetNodes(graph, all.data(), &nodes) == cudaSuccess) {
        kernels = 0;
        for (cudaGraphNode_t nd : all) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
        }
      }
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
  }
  if (graph) cudaGraphDestroy(graph);
  if (st != HMAT_OK) return st;
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_status(e);
  }
  b->kernels = kernels;
  return HMAT_OK;
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
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int k = 0; k < kBranches && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
  }
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    EvalContext* c = nullptr;
    const hmat_status st = ctx_create(*handles[i], &c);  // its side stream serves the branched schedule
    if (st != HMAT_OK) {
      batch_release(b);
      return st;
    }
    b->ctx.push_back(c);
    cudaStream_t ms = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&ms, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->member_stream.push_back(ms);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->member_join.push_back(ev);
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
  if (!same) {
    if (b->exec) {
      cudaStreamSynchronize(b->capture);
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    const hmat_status st = b->branched ? capture_branched(b, W, Y, q, dtype)
                           : (b->mode == HMAT_MODE_MIXED ? capture_mixed(b, W, Y, q, dtype)
                                                         : capture_fp64(b, W, Y, q, dtype));
    if (st != HMAT_OK) return st;
    b->key_w.assign(W, W + n);
    b->key_y.assign(Y, Y + n);
    b->key_q.assign(q, q + n);
    b->key_dtype = dtype;
  }
  return cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

extern "C" hmat_status hmat_batch_eval(hmat_batch_t b, const double* const* W, double* const* Y, const int64_t* q,
                                       void* stream) {
  return hmat_batch_eval_typed(b, reinterpret_cast<const void* const*>(W), reinterpret_cast<void* const*>(Y), q,
                               HMAT_DTYPE_F64, stream);
}

extern "C" hmat_status hmat_batch_autotune(hmat_batch_t b, const void* const* W, void* const* Y, const int64_t* q,
                                           int dtype, void* stream, double* ms_default, double* ms_tuned) {
  if (!b) return HMAT_EINVAL;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) return HMAT_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return HMAT_ECUDA;
  }
  double best = 1e30, def = -1;
  int best_grid = 0;
  hmat_status st = HMAT_OK;
  // the chain launches run beside the near field, which needs whole SMs: fewer chain CTAs
  // leave it more of them; timed on whole replays of the batch's graph
  int best_branched = 0, best_widths = 0;
  // the flattened schedule with several chain grids, with the members' own tuned column
  // widths and (mixed) with every member at its default width (a width tuned for a member
  // alone need not suit it beside the others), then one branch per member
  struct Cand { int grid, widths; };
  std::vector<Cand> cands;
  for (int w = 0; w < (b->mode == HMAT_MODE_MIXED ? 2 : 1); ++w)
    for (int g : {0, 2 * sms, sms, sms / 2, sms / 4}) cands.push_back({g, w});
  cands.push_back({-1, 0});
  for (const Cand& cd : cands) {
    const int g = cd.grid;
    b->branched = g < 0 ? 1 : 0;
    b->chain_grid = g < 0 ? 0 : g;
    b->default_widths = cd.widths;
    if (b->exec) {  // recapture with this grid
      cudaStreamSynchronize(b->capture);
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    double t = 1e30;
    for (int r = 0; r < 4 && st == HMAT_OK; ++r) {
      if ((st = hmat_batch_eval_typed(b, W, Y, q, dtype, stream)) != HMAT_OK) break;
      if (cudaEventRecord(e0, s) != cudaSuccess) st = HMAT_ECUDA;
      if (st == HMAT_OK) st = hmat_batch_eval_typed(b, W, Y, q, dtype, stream);
      float ms = 0;
      if (st == HMAT_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = HMAT_ECUDA;
      if (st == HMAT_OK && r > 0) t = std::min(t, (double)ms);
    }
    if (st != HMAT_OK) break;
    if (g == 0 && cd.widths == 0) def = t;
    if (t < best) {
      best = t;
      best_grid = g < 0 ? 0 : g;
      best_branched = g < 0 ? 1 : 0;
      best_widths = cd.widths;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->chain_grid = st == HMAT_OK ? best_grid : 0;
  b->branched = st == HMAT_OK ? best_branched : 0;
  b->default_widths = st == HMAT_OK ? best_widths : 0;
  if (b->exec) {
    cudaStreamSynchronize(b->capture);
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (st != HMAT_OK) return st;
  if (ms_default) *ms_default = def;
  if (ms_tuned) *ms_tuned = best;
  return HMAT_OK;
}

extern "C" hmat_status hmat_batch_schedule(hmat_batch_t b, int branched, int chain_grid, int default_widths) {
  if (!b || branched < 0 || branched > 1 || chain_grid < 0 || default_widths < 0 || default_widths > 1)
    return HMAT_EINVAL;
  if (b->branched != branched || b->chain_grid != chain_grid || b->default_widths != default_widths) {
    if (b->exec) {  // the next call recaptures
      cudaStreamSynchronize(b->capture);
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    b->branched = branched;
    b->chain_grid = chain_grid;
    b->default_widths = default_widths;
  }
  return HMAT_OK;
}

extern "C" hmat_status hmat_batch_info(hmat_batch_t b, int64_t* out, int n) {
  if (!b || !out || n < 0) return HMAT_EINVAL;
  const int64_t vals[6] = {(int64_t)b->handles.size(), b->exec ? b->kernels : 0, b->block_bytes, b->chain_grid,
                           b->branched, b->default_widths};
  for (int i = 0; i < n && i < 6; ++i) out[i] = vals[i];
  return HMAT_OK;
}

extern "C" hmat_status hmat_batch_free(hmat_batch_t b) {
  if (!b) return HMAT_OK;
  batch_release(b);
  return HMAT_OK;
}
