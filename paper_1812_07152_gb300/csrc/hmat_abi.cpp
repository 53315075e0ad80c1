// libhmat C ABI: validation and level-packed upload of an HMatrix (hmat_load),
// the evaluation runtime (hmat_eval) and the handle's lifetime.
//
// The phases follow the evaluation of Section 2.1: the near-field reduction over
// D, the bottom-up tree loop over the bases, the far-field reduction over B and
// the top-down tree loop. Every phase is one grouped-GEMM launch over a work list
// built here once per handle; the gather of W into tree order and the scatter of
// Y back to the caller's order are folded into the row indexing of the first and
// last phases (perm maps a tree-order row to the caller's row).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>

#include "hmat_internal.h"

using namespace hmat;

namespace {

constexpr int64_t kAlignValues = 16;  // every packed block starts on a 128-byte boundary

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct Validated {
  int64_t n_nodes, n_leaves, first_leaf, n_near, n_far;
};

int level_of(int64_t a) {
  int l = 0;
  while (((int64_t)2 << l) - 1 <= a) ++l;
  return l;
}

hmat_status validate(const hmat_desc* d, bool host_blocks, Validated* v) {
  if (!d || d->levels < 0 || d->levels > 24 || d->n_points < 0) return HMAT_EINVAL;
  const int64_t n_nodes = ((int64_t)2 << d->levels) - 1;
  const int64_t n_leaves = (int64_t)1 << d->levels;
  const int64_t first_leaf = n_leaves - 1;
  if (!d->node_begin || !d->node_size || !d->rank || !d->near_ptr || !d->far_ptr) return HMAT_EINVAL;
  if (d->n_points > 0 && !d->perm) return HMAT_EINVAL;
  if (d->node_begin[0] != 0 || d->node_size[0] != d->n_points) return HMAT_EINVAL;
  for (int64_t a = 0; a < n_nodes; ++a) {
    if (d->node_size[a] < 0 || d->rank[a] < 0 || d->rank[a] > (1 << 20)) return HMAT_EINVAL;
    if (d->node_size[a] > INT32_MAX) return HMAT_EINVAL;
    if (a < first_leaf) {
      const int64_t l = 2 * a + 1, r = 2 * a + 2;
      if (d->node_begin[l] != d->node_begin[a]) return HMAT_EINVAL;
      if (d->node_size[l] + d->node_size[r] != d->node_size[a]) return HMAT_EINVAL;
      if (d->node_begin[r] != d->node_begin[a] + d->node_size[l]) return HMAT_EINVAL;
    }
  }
  // perm: a bijection of 0..n_points-1
  if (d->n_points > 0) {
    std::vector<uint8_t> seen((size_t)d->n_points, 0);
    for (int64_t k = 0; k < d->n_points; ++k) {
      const int64_t p = d->perm[k];
      if (p < 0 || p >= d->n_points || seen[(size_t)p]) return HMAT_EINVAL;
      seen[(size_t)p] = 1;
    }
  }
  // near CSR over leaves
  if (d->near_ptr[0] != 0) return HMAT_EINVAL;
  for (int64_t i = 0; i < n_leaves; ++i)
    if (d->near_ptr[i + 1] < d->near_ptr[i]) return HMAT_EINVAL;
  const int64_t n_near = d->near_ptr[n_leaves];
  if (n_near > INT32_MAX) return HMAT_EINVAL;
  if (n_near > 0 && (!d->near_idx || (host_blocks && !d->near))) return HMAT_EINVAL;
  for (int64_t e = 0; e < n_near; ++e) {
    if (d->near_idx[e] < 0 || d->near_idx[e] >= n_leaves) return HMAT_EINVAL;
  }
  for (int64_t i = 0; i < n_leaves; ++i)
    for (int64_t e = d->near_ptr[i]; e < d->near_ptr[i + 1]; ++e) {
      const int64_t j = d->near_idx[e];
      if (host_blocks && d->node_size[first_leaf + i] * d->node_size[first_leaf + j] > 0 && !d->near[e])
        return HMAT_EINVAL;
    }
  // far CSR over nodes
  if (d->far_ptr[0] != 0) return HMAT_EINVAL;
  for (int64_t a = 0; a < n_nodes; ++a)
    if (d->far_ptr[a + 1] < d->far_ptr[a]) return HMAT_EINVAL;
  const int64_t n_far = d->far_ptr[n_nodes];
  if (n_far > INT32_MAX) return HMAT_EINVAL;
  if (n_far > 0 && (!d->far_idx || (host_blocks && !d->coupling))) return HMAT_EINVAL;
  for (int64_t a = 0; a < n_nodes; ++a)
    for (int64_t e = d->far_ptr[a]; e < d->far_ptr[a + 1]; ++e) {
      const int64_t b = d->far_idx[e];
      if (b < 0 || b >= n_nodes || b == a || level_of(a) != level_of(b)) return HMAT_EINVAL;
      if (host_blocks && (int64_t)d->rank[a] * d->rank[b] > 0 && !d->coupling[e]) return HMAT_EINVAL;
    }
  // bases
  for (int64_t a = 0; a < n_nodes; ++a) {
    if (d->rank[a] == 0) continue;
    if (!d->basis) return HMAT_EINVAL;
    const int64_t rows = a >= first_leaf ? d->node_size[a] : (int64_t)d->rank[2 * a + 1] + d->rank[2 * a + 2];
    if (rows > 0 && !d->basis[a]) return HMAT_EINVAL;
  }
  v->n_nodes = n_nodes;
  v->n_leaves = n_leaves;
  v->first_leaf = first_leaf;
  v->n_near = n_near;
  v->n_far = n_far;
  return HMAT_OK;
}

// Streams host blocks into a device arena through two pinned staging buffers.
class Uploader {
 public:
  Uploader() = default;
  ~Uploader() { release(); }
  cudaError_t init(double* dst, size_t stage_values) {
    dst_ = dst;
    cap_ = stage_values;
    for (int b = 0; b < 2; ++b) {
      cudaError_t e = cudaMallocHost(&buf_[b], cap_ * sizeof(double));
      if (e != cudaSuccess) return e;
      e = cudaEventCreateWithFlags(&ev_[b], cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    return cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking);
  }
  // Copy `count` values of `src` (row-major rows x cols with row stride cols) to
  // arena offset `off`; returns false when a value is not finite.
  bool put(int64_t off, const double* src, int64_t count, cudaError_t* err) {
    if (count == 0) return true;
    if (count > (int64_t)cap_) {  // a block larger than the staging buffer: copy in pieces
      if ((*err = flush()) != cudaSuccess) return true;
      bool finite = true;
      for (int64_t s = 0; s < count && *err == cudaSuccess; s += (int64_t)cap_) {
        const int64_t c = std::min<int64_t>(cap_, count - s);
        finite &= put(off + s, src + s, c, err);
        if (*err == cudaSuccess) *err = flush();
      }
      return finite;
    }
    if (fill_ > 0) {  // extend the staged range across the alignment gap, or flush it
      const int64_t gap = off - (start_ + (int64_t)fill_);
      if (gap < 0 || (int64_t)fill_ + gap + count > (int64_t)cap_) {
        if ((*err = flush()) != cudaSuccess) return true;
      } else {
        std::memset(buf_[cur_] + fill_, 0, (size_t)gap * sizeof(double));
        fill_ += (size_t)gap;
      }
    }
    if (fill_ == 0) start_ = off;
    double* b = buf_[cur_] + fill_;
    bool finite = true;
    for (int64_t i = 0; i < count; ++i) {
      const double x = src[i];
      finite &= std::isfinite(x);
      b[i] = x;
    }
    fill_ += (size_t)count;
    return finite;
  }
  cudaError_t flush() {
    if (fill_ == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dst_ + start_, buf_[cur_], fill_ * sizeof(double), cudaMemcpyHostToDevice, stream_);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev_[cur_], stream_);
    if (e != cudaSuccess) return e;
    cur_ ^= 1;
    fill_ = 0;
    return cudaEventSynchronize(ev_[cur_]);  // the other buffer's copy has finished
  }
  cudaError_t finish() {
    cudaError_t e = flush();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(stream_);
  }
  void release() {
    if (stream_) { cudaStreamSynchronize(stream_); cudaStreamDestroy(stream_); stream_ = nullptr; }
    for (int b = 0; b < 2; ++b) {
      if (buf_[b]) { cudaFreeHost(buf_[b]); buf_[b] = nullptr; }
      if (ev_[b]) { cudaEventDestroy(ev_[b]); ev_[b] = nullptr; }
    }
  }

 private:
  double* dst_ = nullptr;
  double* buf_[2] = {nullptr, nullptr};
  cudaEvent_t ev_[2] = {nullptr, nullptr};
  cudaStream_t stream_ = nullptr;
  size_t cap_ = 0, fill_ = 0;
  int64_t start_ = 0;
  int cur_ = 0;
};

void free_tc(TcProduct* p) {
  cudaFree(p->tiles);
  cudaFree(p->meta);
  *p = TcProduct{};
}

void free_device(Handle* h) {
  for (auto& r : h->prof) {
    h->event_pool.push_back(r.start);
    h->event_pool.push_back(r.stop);
  }
  h->prof.clear();
  for (cudaEvent_t ev : h->event_pool) cudaEventDestroy(ev);
  h->event_pool.clear();
  ctx_destroy(h->ctx);
  h->ctx = nullptr;
  free_tc(&h->tc_near);
  free_tc(&h->tc_far);
  cudaFree(h->arena32);
  cudaFree(h->entries32);
  cudaFree(h->chain.items);
  cudaFree(h->chain.expect);
  h->chain = ChainPlan{};
  cudaFree(h->chain64.items);
  cudaFree(h->chain64.expect);
  h->chain64 = ChainPlan{};
  h->arena32 = nullptr; h->entries32 = nullptr; h->has_mixed = false;
  cudaFree(h->arena);
  cudaFree(h->pts_tree);
  h->pts_tree = nullptr;
  cudaFree(h->far_rows);
  h->far_rows = nullptr;
  cudaFree(h->perm);
  cudaFree(h->tasks);
  cudaFree(h->entries);
  cudaFree(h->tiles);
  cudaFree(h->status);
  h->arena = nullptr; h->perm = nullptr; h->tasks = nullptr; h->entries = nullptr;
  h->tiles = nullptr; h->status = nullptr;
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src, int64_t* bytes) {
  const size_t n = std::max<size_t>(src.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)dst, n);
  if (e != cudaSuccess) return e;
  *bytes += (int64_t)n;
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}



// Host description of one tensor-core product family (see TcLists): a CSR list of
// (target, source) blocks over one node index space and where each block sits in
// the FP64 arena.
struct TcSpec {
  int64_t n_nodes = 0;
  std::vector<int64_t> ptr;      // per target: CSR into the entries (n_nodes + 1)
  std::vector<int32_t> idx;      // per entry: source node
  std::vector<int64_t> blk_off;  // per entry: arena offset of the block's (row 0, column 0)
  std::vector<int32_t> blk_ld;   // per entry: row stride of the block
  std::vector<int32_t> size;     // per node: rows
  std::vector<int64_t> begin;    // per node: first row
  std::vector<char> target;      // per node: gets (target, m-tile) work items
};

// Packs one product family on the device: per-m-tile scale exponents, then the hi/lo
// tile pairs of every (entry, m-tile of its target, k-chunk of its source), and
// uploads the metadata and the (target, m-tile) work list, longest lists first.
hmat_status build_tc(Handle* h, const TcSpec& sp, TcProduct* out) {
  const int64_t nn = sp.n_nodes;
  std::vector<int32_t> kc(nn), mt_base(nn + 1), n_mt(nn);
  std::vector<int64_t> kcum(nn + 1);
  mt_base[0] = 0;
  kcum[0] = 0;
  for (int64_t i = 0; i < nn; ++i) {
    kc[i] = (sp.size[i] + kTcK - 1) / kTcK;
    n_mt[i] = sp.target[i] ? (sp.size[i] + kTcRows - 1) / kTcRows : 0;
    mt_base[i + 1] = mt_base[i] + n_mt[i];
    kcum[i + 1] = kcum[i] + kc[i];
  }
  const int64_t n_mtiles = mt_base[nn];
  out->n_chunks = kcum[nn];
  std::vector<int32_t> mtile_node(n_mtiles), mtile_mt(n_mtiles), chunk_node(out->n_chunks), chunk_c(out->n_chunks);
  for (int64_t i = 0; i < nn; ++i) {
    for (int32_t m = 0; m < n_mt[i]; ++m) {
      mtile_node[mt_base[i] + m] = (int32_t)i;
      mtile_mt[mt_base[i] + m] = m;
    }
    for (int32_t c = 0; c < kc[i]; ++c) {
      chunk_node[kcum[i] + c] = (int32_t)i;
      chunk_c[kcum[i] + c] = c;
    }
  }
  const int64_t n_entries = sp.ptr[nn];
  std::vector<int64_t> a_off(n_entries, 0);
  std::vector<TcPackJob> jobs;
  int64_t bytes = 0;
  for (int64_t i = 0; i < nn; ++i)
    for (int64_t e = sp.ptr[i]; e < sp.ptr[i + 1]; ++e) {
      const int32_t j = sp.idx[e];
      a_off[e] = bytes;
      for (int32_t m = 0; m < n_mt[i]; ++m)
        for (int32_t c = 0; c < kc[j]; ++c)
          jobs.push_back(TcPackJob{bytes + ((int64_t)m * kc[j] + c) * 2 * kTcTileBytes, sp.blk_off[e], sp.size[i],
                                   sp.size[j], m * kTcRows, c * kTcK, mt_base[i] + m, sp.blk_ld[e]});
      bytes += (int64_t)n_mt[i] * kc[j] * 2 * kTcTileBytes;
    }
  std::vector<std::pair<int64_t, TcTile>> work;
  for (int64_t i = 0; i < nn; ++i) {
    int64_t cost = 0;
    for (int64_t e = sp.ptr[i]; e < sp.ptr[i + 1]; ++e) cost += kc[sp.idx[e]];
    for (int32_t m = 0; m < n_mt[i]; ++m) work.push_back({cost, TcTile{(int32_t)i, m}});
  }
  // longest lists first by half-octave class of their length (no long list in the last
  // wave), tree order within a class: targets that run side by side are neighbours and
  // share most of their sources, whose right-hand-side tiles then come from L2
  // (measured: N=262144 inverse multiquadric near field 4.83 -> 4.57 ms; strict
  // longest-first is needed where list lengths spread, the N=65536 mixture's 98..512)
  auto cls = [](int64_t c) { return c > 0 ? (int)std::floor(2.0 * std::log2((double)c)) : 0; };
  std::stable_sort(work.begin(), work.end(), [&](const auto& x, const auto& y) { return cls(x.first) > cls(y.first); });
  std::vector<TcTile> work_list;
  for (auto& w : work) work_list.push_back(w.second);
  out->n_work = (int64_t)work_list.size();

  // one allocation for the permanent metadata
  struct Part { const void* src; size_t bytes; void** dst; };
  int64_t* d_a_off; int64_t* d_ptr; int32_t* d_idx; int32_t* d_kc; int64_t* d_kcum; int64_t* d_begin;
  int32_t* d_size; int32_t* d_mt_base; int32_t* d_scale; TcTile* d_work; int32_t* d_chunk_node; int32_t* d_chunk_c;
  std::vector<int32_t> scale_zero(std::max<int64_t>(n_mtiles, 1), 0);
  Part parts[] = {
      {a_off.data(), a_off.size() * 8, (void**)&d_a_off},
      {sp.ptr.data(), sp.ptr.size() * 8, (void**)&d_ptr},
      {sp.idx.data(), sp.idx.size() * 4, (void**)&d_idx},
      {kc.data(), kc.size() * 4, (void**)&d_kc},
      {kcum.data(), kcum.size() * 8, (void**)&d_kcum},
      {sp.begin.data(), sp.begin.size() * 8, (void**)&d_begin},
      {sp.size.data(), sp.size.size() * 4, (void**)&d_size},
      {mt_base.data(), mt_base.size() * 4, (void**)&d_mt_base},
      {scale_zero.data(), scale_zero.size() * 4, (void**)&d_scale},
      {work_list.data(), work_list.size() * sizeof(TcTile), (void**)&d_work},
      {chunk_node.data(), chunk_node.size() * 4, (void**)&d_chunk_node},
      {chunk_c.data(), chunk_c.size() * 4, (void**)&d_chunk_c},
  };
  size_t total = 0;
  for (auto& p : parts) total += (p.bytes + 255) / 256 * 256 + 256;
  uint8_t* meta = nullptr;
  cudaError_t e = cudaMalloc((void**)&meta, total);
  if (e != cudaSuccess) return cuda_status(e);
  out->meta = meta;
  h->device_bytes += (int64_t)total;
  size_t o = 0;
  for (auto& p : parts) {
    *p.dst = meta + o;
    if (p.bytes && (e = cudaMemcpy(meta + o, p.src, p.bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_status(e);
    o += (p.bytes + 255) / 256 * 256 + 256;
  }
  out->dev = TcLists{nullptr, d_a_off, d_ptr, d_idx, d_kc, d_kcum, d_begin, d_size, d_mt_base, d_scale,
                     d_work, d_chunk_node, d_chunk_c};

  // tiles: scale exponents, then the packed hi/lo pairs
  if ((e = cudaMalloc((void**)&out->tiles, (size_t)std::max<int64_t>(bytes, 256))) != cudaSuccess)
    return cuda_status(e);
  out->tile_bytes = bytes;
  h->device_bytes += bytes;
  out->dev.tiles = out->tiles;
  int64_t* d_blk_off = nullptr; int32_t* d_blk_ld = nullptr; int32_t* d_mnode = nullptr; int32_t* d_mmt = nullptr;
  TcPackJob* d_jobs = nullptr;
  int64_t scratch = 0;
  e = upload(&d_blk_off, sp.blk_off, &scratch);
  if (e == cudaSuccess) e = upload(&d_blk_ld, sp.blk_ld, &scratch);
  if (e == cudaSuccess) e = upload(&d_mnode, mtile_node, &scratch);
  if (e == cudaSuccess) e = upload(&d_mmt, mtile_mt, &scratch);
  if (e == cudaSuccess) e = upload(&d_jobs, jobs, &scratch);
  if (e == cudaSuccess) e = launch_tc_scale(out->dev, d_blk_off, d_blk_ld, h->arena, n_mtiles, d_mnode, d_mmt, d_scale, 0);
  if (e == cudaSuccess) e = launch_tc_pack(d_jobs, (int64_t)jobs.size(), h->arena, d_scale, out->tiles, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_blk_off);
  cudaFree(d_blk_ld);
  cudaFree(d_mnode);
  cudaFree(d_mmt);
  cudaFree(d_jobs);
  return e == cudaSuccess ? HMAT_OK : cuda_status(e);
}

// Mixed-precision copies of a loaded HMatrix (HMAT_LOAD_MIXED): the near blocks and
// the coupling blocks as FP16 hi/lo tensor-core tiles (packed on the device from the
// FP64 arena, one scale exponent per 128-row m-tile of a target), and the operand of
// every FP32 entry (the bases, and the coupling blocks when the coupling runs in FP32)
// as an FP32 block of its own in the k-major padded layout the FP32 kernel copies 16
// bytes at a time (a basis is held twice: as read by the upward and by the downward pass).
hmat_status build_mixed(Handle* h, const hmat_desc* d, const Validated& v, const std::vector<int64_t>& near_off,
                        const std::vector<int64_t>& far_task_off, const std::vector<int64_t>& far_off,
                        const std::vector<int64_t>& far_k, const std::vector<GemmTask>& tasks,
                        const std::vector<GemmEntry>& entries, const std::vector<GemmTile>& tiles) {
  const int64_t nl = v.n_leaves, fl = v.first_leaf;
  {  // near field: targets and sources are the leaves
    TcSpec sp;
    sp.n_nodes = nl;
    sp.ptr.assign(d->near_ptr, d->near_ptr + nl + 1);
    sp.idx.assign(d->near_idx, d->near_idx + v.n_near);
    sp.size.resize(nl);
    sp.begin.resize(nl);
    sp.target.assign(nl, 1);
    for (int64_t i = 0; i < nl; ++i) {
      sp.size[i] = (int32_t)h->size[fl + i];
      sp.begin[i] = h->begin[fl + i];
    }
    sp.blk_off = near_off;
    sp.blk_ld.resize(v.n_near);
    for (int64_t e = 0; e < v.n_near; ++e) sp.blk_ld[e] = sp.size[sp.idx[e]];
    hmat_status st = build_tc(h, sp, &h->tc_near);
    if (st != HMAT_OK) return st;
  }
  if (h->tc_coupling) {  // coupling: targets are the nodes with a basis, sources their
                        // far partners; B_ab is the column slice of B_a starting at far_off
    TcSpec sp;
    const int64_t nn = v.n_nodes;
    sp.n_nodes = nn;
    sp.ptr.assign(d->far_ptr, d->far_ptr + nn + 1);
    sp.idx.assign(d->far_idx, d->far_idx + v.n_far);
    sp.size.resize(nn);
    sp.begin.resize(nn);
    sp.target.assign(nn, 0);
    for (int64_t a = 0; a < nn; ++a) {
      sp.size[a] = h->rank[a];
      sp.begin[a] = h->skel_off[a];
      sp.target[a] = a >= 1 && h->rank[a] > 0;
    }
    sp.blk_off.assign(v.n_far, 0);
    sp.blk_ld.assign(v.n_far, 1);
    for (int64_t a = 0; a < nn; ++a) {
      if (far_task_off[a] < 0) continue;
      for (int64_t e = d->far_ptr[a]; e < d->far_ptr[a + 1]; ++e) {
        sp.blk_off[e] = far_task_off[a] + far_off[e];
        sp.blk_ld[e] = (int32_t)far_k[a];
      }
    }
    hmat_status st = build_tc(h, sp, &h->tc_far);
    if (st != HMAT_OK) return st;
  }

  // FP32 operands: one k-major block per entry of an FP32 phase (each task belongs to
  // one phase; the FP32 coupling phase has tiles of its own over the coupling tasks)
  // (an entry of another phase keeps k = 0 there: it contributes nothing)
  std::vector<GemmEntry> e32(entries.size(), GemmEntry{0, 0, 0, 4, 1, 0});
  std::vector<F32Job> jobs;
  std::vector<char> seen(tasks.size(), 0);
  int64_t n32 = 0;
  for (const Phase& ph : h->phases32)
    for (int64_t i = ph.tile_begin; i < ph.tile_begin + ph.n_tiles; ++i) {
      const int32_t t = tiles[i].task;
      if (seen[t]) continue;
      seen[t] = 1;
      const GemmTask& tk = tasks[t];
      const int32_t ld = (tk.m + 3) / 4 * 4;
      for (int32_t e = tk.e_begin; e < tk.e_end; ++e) {
        const GemmEntry& en = entries[e];
        jobs.push_back(F32Job{en.a_off, n32, tk.m, en.k, en.lda, ld, en.trans, 0});
        e32[e] = GemmEntry{n32, en.x_row, en.k, ld, 1, 0};
        n32 += (int64_t)ld * en.k;
      }
    }
  cudaError_t e;
  if ((e = cudaMalloc((void**)&h->arena32, (size_t)std::max<int64_t>(n32, 4) * sizeof(float))) != cudaSuccess)
    return cuda_status(e);
  h->device_bytes += std::max<int64_t>(n32, 4) * (int64_t)sizeof(float);
  if ((e = upload(&h->entries32, e32, &h->device_bytes)) != cudaSuccess) return cuda_status(e);
  F32Job* d_jobs = nullptr;
  int64_t scratch = 0;
  if ((e = upload(&d_jobs, jobs, &scratch)) != cudaSuccess) return cuda_status(e);
  e = launch_relayout_f32(h->arena, d_jobs, (int64_t)jobs.size(), h->arena32, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_jobs);
  if (e != cudaSuccess) return cuda_status(e);
  h->has_mixed = true;
  return HMAT_OK;
}

// Counts per node of the items a dependent item waits for (the expect layout of ChainSync).
std::vector<int32_t> chain_expect(const std::vector<ChainItem>& items, int64_t n, int L) {
  std::vector<int32_t> expect(3 * n + L + 1, 0);
  for (const ChainItem& it : items) {
    if (it.kind == CK_UP) {
      expect[it.node] += 1;
      expect[3 * n + it.level] += 1;
    } else if (it.kind == CK_CPL) {
      expect[n + it.node] += 1;
    } else if (it.kind == CK_DN) {
      expect[2 * n + it.node] += 1;
    }
  }
  return expect;
}

// The FP64 far field as one chain launch: the upward pass, each level's coupling after
// the next level up, the downward transfers, the downward leaf step.
hmat_status build_chain64(Handle* h, const Validated& v, const std::vector<ChainItem> (&by_kind)[4]) {
  const int L = h->levels;
  std::vector<ChainItem> items;
  auto level_range = [&](int ck, int l) {
    for (const ChainItem& it : by_kind[ck])
      if (it.level == l) items.push_back(it);
  };
  level_range(CK_UP, L);
  for (int l = L - 1; l >= 1; --l) {
    level_range(CK_UP, l);
    level_range(CK_CPL, l + 1);
  }
  if (L >= 1) level_range(CK_CPL, 1);
  for (int l = 1; l < L; ++l) level_range(CK_DN, l);
  level_range(CK_LEAF, L);
  if (items.size() > (size_t)INT32_MAX) return HMAT_EUNSUPPORTED;
  ChainPlan& cp = h->chain64;
  cp.begin[0] = 0;
  cp.count[0] = (int32_t)items.size();
  cp.waits[0] = kWaitUp | kWaitLevel | kWaitCpl | kWaitDn;
  const std::vector<int32_t> expect = chain_expect(items, v.n_nodes, L);
  cp.n_ctr = kChainCtrHead + (int64_t)expect.size();
  cp.host = items;
  cudaError_t e = chain64_prepare();
  if (e == cudaSuccess) e = upload(&cp.items, items, &h->device_bytes);
  if (e == cudaSuccess) e = upload(&cp.expect, expect, &h->device_bytes);
  return cuda_status(e);
}

// The far field of the mixed mode as chain items (hmat_chain.cu): every tile of the
// FP32 phases, ordered so that every item's dependencies come before it, and the
// number of items per node and kind that a dependent item waits for.
hmat_status build_chain(Handle* h, const Validated& v, const std::vector<GemmTile>& tiles,
                        const std::vector<int32_t>& task_node) {
  const int L = h->levels;
  const int64_t n = v.n_nodes;
  std::vector<std::vector<ChainItem>> up(L + 1), cpl(L + 1), dn(L + 1);
  std::vector<ChainItem> leaf;
  for (const Phase& ph : h->phases32) {
    const uint8_t cls = ph.tile_rows == 16 ? 0 : (ph.tile_rows == 32 ? 1 : 2);
    for (int64_t i = ph.tile_begin; i < ph.tile_begin + ph.n_tiles; ++i) {
      const int32_t node = task_node[tiles[i].task];
      const int lvl = level_of(node);
      ChainItem it{(int32_t)i, node, 0, cls, (uint8_t)lvl, (uint8_t)(ph.xmap == XMAP_FAR ? 1 : 0)};
      switch (ph.kind) {
        case PH_UP_LEAF:
        case PH_UP_TRANS: it.kind = CK_UP; up[lvl].push_back(it); break;
        case PH_COUPLING: it.kind = CK_CPL; cpl[lvl].push_back(it); break;
        case PH_DOWN_TRANS: it.kind = CK_DN; dn[lvl].push_back(it); break;
        case PH_DOWN_LEAF: it.kind = CK_LEAF; leaf.push_back(it); break;
        default: return HMAT_EINVAL;
      }
    }
  }
  std::vector<ChainItem> items;
  auto append = [&](const std::vector<ChainItem>& b) { items.insert(items.end(), b.begin(), b.end()); };
  ChainPlan& cp = h->chain;
  // A: the upward pass, each level's coupling after the next level up has been queued
  // (so that the CTAs that take it find its inputs ready), then the downward transfers
  cp.begin[0] = 0;
  append(up[L]);
  for (int l = L - 1; l >= 1; --l) {
    append(up[l]);
    if (!h->tc_coupling) append(cpl[l + 1]);
  }
  if (!h->tc_coupling && L >= 1) append(cpl[1]);
  if (!h->tc_coupling)
    for (int l = 1; l < L; ++l) append(dn[l]);
  cp.count[0] = (int32_t)items.size();
  cp.waits[0] = h->tc_coupling ? kWaitUp : (kWaitUp | kWaitLevel | kWaitCpl | kWaitDn);
  // B: the downward transfers after the tensor-core coupling (which the stream orders)
  cp.begin[1] = (int32_t)items.size();
  if (h->tc_coupling)
    for (int l = 1; l < L; ++l) append(dn[l]);
  cp.count[1] = (int32_t)items.size() - cp.begin[1];
  cp.waits[1] = kWaitDn;
  // C: the downward leaf step, after the near field has written Y (ordered by the stream)
  cp.begin[2] = (int32_t)items.size();
  append(leaf);
  cp.count[2] = (int32_t)items.size() - cp.begin[2];
  cp.waits[2] = 0;
  if (items.size() > (size_t)INT32_MAX) return HMAT_EUNSUPPORTED;
  const std::vector<int32_t> expect = chain_expect(items, n, L);
  cp.n_ctr = kChainCtrHead + (int64_t)expect.size();
  cp.host = items;
  cudaError_t e = chain_prepare(nullptr, nullptr);
  if (e == cudaSuccess) e = upload(&cp.items, items, &h->device_bytes);
  if (e == cudaSuccess) e = upload(&cp.expect, expect, &h->device_bytes);
  return cuda_status(e);
}

}  // namespace

namespace hmat {

hmat_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HMAT_OK;
  if (e == cudaErrorMemoryAllocation) return HMAT_ENOMEM;
  return HMAT_ECUDA;
}

hmat_status load_impl(const hmat_desc* d, const DeviceBlockSource* src, int flags, hmat_handle** out) {
  *out = nullptr;
  if (flags & ~(HMAT_LOAD_MIXED | HMAT_LOAD_MIXED_ONLY | HMAT_BUILD_NEAR_OTF)) return HMAT_EUNSUPPORTED;
  if (flags & HMAT_LOAD_MIXED_ONLY) flags |= HMAT_LOAD_MIXED;
  // blocks evaluated on the fly need the points (a build), and the FP64 mode
  if ((flags & HMAT_BUILD_NEAR_OTF) && (!src || (flags & HMAT_LOAD_MIXED))) return HMAT_EUNSUPPORTED;
  const bool near_otf = (flags & HMAT_BUILD_NEAR_OTF) != 0;
  Validated v;
  hmat_status st = validate(d, src == nullptr, &v);
  if (st != HMAT_OK) return st;

  std::unique_ptr<hmat_handle> h(new (std::nothrow) hmat_handle());
  if (!h) return HMAT_ENOMEM;
  if (cudaGetDevice(&h->device) != cudaSuccess) return HMAT_ECUDA;
  h->n_points = d->n_points;
  h->levels = d->levels;
  h->n_nodes = v.n_nodes;
  h->n_leaves = v.n_leaves;
  h->n_near = v.n_near;
  h->n_far = v.n_far;
  h->begin.assign(d->node_begin, d->node_begin + v.n_nodes);
  h->size.assign(d->node_size, d->node_size + v.n_nodes);
  h->rank.assign(d->rank, d->rank + v.n_nodes);
  h->perm_host.assign(d->perm, d->perm + d->n_points);
  h->near_ptr.assign(d->near_ptr, d->near_ptr + v.n_leaves + 1);
  h->near_idx.assign(d->near_idx, d->near_idx + v.n_near);
  h->far_ptr.assign(d->far_ptr, d->far_ptr + v.n_nodes + 1);
  h->far_idx.assign(d->far_idx, d->far_idx + v.n_far);
  h->skel_off.resize(v.n_nodes + 1);
  h->skel_off[0] = 0;
  for (int64_t a = 0; a < v.n_nodes; ++a) h->skel_off[a + 1] = h->skel_off[a] + h->rank[a];
  h->sum_rank = h->skel_off[v.n_nodes];
  const int64_t fl = v.first_leaf;
  auto rows_of = [&](int64_t a) -> int64_t {
    return a >= fl ? h->size[a] : (int64_t)h->rank[2 * a + 1] + h->rank[2 * a + 2];
  };

  // ---- arena layout: near blocks (CSR order), bases (node order), coupling (CSR order)
  std::vector<int64_t> near_off(v.n_near), basis_off(v.n_nodes, -1), far_off(v.n_far);
  int64_t off = 0;
  for (int64_t i = 0; i < v.n_leaves; ++i)
    for (int64_t e = d->near_ptr[i]; e < d->near_ptr[i + 1]; ++e) {
      const int64_t cnt = h->size[fl + i] * h->size[fl + d->near_idx[e]];
      h->near_values += cnt;
      near_off[e] = near_otf ? 0 : off;  // on the fly: nothing stored, the offset unused
      if (!near_otf) off = align_up(off + cnt, kAlignValues);
    }
  for (int64_t a = 0; a < v.n_nodes; ++a) {
    if (h->rank[a] == 0) continue;
    basis_off[a] = off;
    const int64_t cnt = rows_of(a) * h->rank[a];
    h->basis_values += cnt;
    off = align_up(off + cnt, kAlignValues);
  }
  // coupling: the blocks of one target node side by side, B_a = [B_ab1 | B_ab2 | ...]
  // (s_a x K_a, K_a = sum of the partners' ranks), so the far-field reduction of a
  // node is one product B_a [w_b1; w_b2; ...] whose right operand is gathered through
  // the row map far_rows.
  std::vector<int64_t> far_task_off(v.n_nodes, -1), far_k(v.n_nodes, 0), far_rows_off(v.n_nodes, 0);
  std::vector<int64_t> far_rows_host;
  for (int64_t a = 0; a < v.n_nodes; ++a) {
    far_rows_off[a] = (int64_t)far_rows_host.size();
    for (int64_t e = d->far_ptr[a]; e < d->far_ptr[a + 1]; ++e) {
      const int64_t b = d->far_idx[e];
      far_off[e] = far_k[a];  // column offset of B_ab inside B_a
      far_k[a] += h->rank[b];
      for (int32_t r = 0; r < h->rank[b]; ++r) far_rows_host.push_back(h->skel_off[b] + r);
    }
    if (h->rank[a] == 0 || far_k[a] == 0) continue;
    far_task_off[a] = off;
    const int64_t cnt = (int64_t)h->rank[a] * far_k[a];
    h->coupling_values += cnt;
    off = align_up(off + cnt, kAlignValues);
  }
  h->arena_values = std::max<int64_t>(off, 1);

  // ---- mixed mode: coupling on the tensor cores when the 128 x 64 tiles are well
  // filled (ranks of about 64 and more); small ranks would leave most of every tile
  // padding, and then the FP32 grouped GEMM on the CUDA cores is faster
  if (flags & HMAT_LOAD_MIXED) {
    double padded = 0.0;
    for (int64_t a = 1; a < v.n_nodes; ++a) {
      if (h->rank[a] == 0) continue;
      const double rows = (double)((h->rank[a] + kTcRows - 1) / kTcRows * kTcRows);
      for (int64_t e = d->far_ptr[a]; e < d->far_ptr[a + 1]; ++e)
        padded += rows * (double)((h->rank[d->far_idx[e]] + kTcK - 1) / kTcK * kTcK);
    }
    h->tc_coupling = padded > 0.0 && (double)h->coupling_values >= kTcCouplingFill * padded;
  }

  // ---- work lists
  std::vector<GemmTask> tasks;
  std::vector<GemmEntry> entries;
  std::vector<GemmTile> tiles;
  std::vector<int64_t> tile_cost;
  // One launch per row-tile size: tasks of at most 16 or 32 rows get smaller tiles so
  // that the FP64 kernels spend no DFMA on padding rows of small skeleton blocks.
  auto add_phase = [&](PhaseKind kind, int32_t level, MatrixKind x, MatrixKind y,
                       const std::vector<int32_t>& task_ids, XMap xmap) {
    for (int32_t rows_cls : {64, 32, 16}) {
      Phase ph{kind, level, x, y, xmap, (int64_t)tiles.size(), 0, 0, rows_cls};
      std::vector<std::pair<int64_t, GemmTile>> list;
      for (int32_t t : task_ids) {
        const GemmTask& tk = tasks[t];
        const int32_t cls = tk.m <= 16 ? 16 : (tk.m <= 32 ? 32 : 64);
        if (cls != rows_cls) continue;
        int64_t kk = 0;
        for (int32_t e = tk.e_begin; e < tk.e_end; ++e) kk += entries[e].k;
        ph.max_m = std::max(ph.max_m, tk.m);
        for (int32_t m0 = 0; m0 < tk.m; m0 += rows_cls) {
          const int64_t rows = std::min(rows_cls, tk.m - m0);
          list.push_back({rows * std::max<int64_t>(kk, 1), GemmTile{t, m0}});
        }
      }
      // longest tiles first, so that the last wave of CTAs is short
      std::stable_sort(list.begin(), list.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
      for (auto& p : list) tiles.push_back(p.second);
      ph.n_tiles = (int64_t)tiles.size() - ph.tile_begin;
      if (ph.n_tiles > 0) h->phases.push_back(ph);
    }
    // The mixed mode runs the upward and downward passes as FP32 launches of the same
    // tiles; the near field runs on the tensor cores, and so does the coupling when
    // its tiles fill well. The FP32 kernel splits each task's K over warp groups, so
    // an FP32 coupling (long K: hundreds of partners) is bound by its longest task:
    // one launch of 16-row tiles for all its tasks, longest K first.
    if (kind == PH_NEAR || (kind == PH_COUPLING && h->tc_coupling)) return;
    if (kind != PH_COUPLING) {
      for (const Phase& p : h->phases)
        if (p.kind == kind && p.level == level) h->phases32.push_back(p);
      return;
    }
    Phase ph{kind, level, x, y, xmap, (int64_t)tiles.size(), 0, 0, 16};
    std::vector<std::pair<int64_t, GemmTile>> list;
    for (int32_t t : task_ids) {
      const GemmTask& tk = tasks[t];
      int64_t kk = 0;
      for (int32_t e = tk.e_begin; e < tk.e_end; ++e) kk += entries[e].k;
      ph.max_m = std::max(ph.max_m, tk.m);
      for (int32_t m0 = 0; m0 < tk.m; m0 += 16) list.push_back({std::max<int64_t>(kk, 1), GemmTile{t, m0}});
    }
    std::stable_sort(list.begin(), list.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (auto& p : list) tiles.push_back(p.second);
    ph.n_tiles = (int64_t)tiles.size() - ph.tile_begin;
    if (ph.n_tiles > 0) h->phases32.push_back(ph);
  };
  std::vector<int32_t> task_node;  // the tree node of each task (the chains' counters)
  std::vector<PhaseKind> task_kind;
  auto new_task = [&](int64_t out_row, int64_t m, int accumulate, int64_t node, PhaseKind kind) -> int32_t {
    tasks.push_back(GemmTask{out_row, (int32_t)m, (int32_t)entries.size(), (int32_t)entries.size(), accumulate});
    task_node.push_back((int32_t)node);
    task_kind.push_back(kind);
    return (int32_t)tasks.size() - 1;
  };
  auto add_entry = [&](int32_t t, int64_t a_off, int64_t x_row, int64_t k, int64_t lda, int trans) {
    if (k == 0) return;
    entries.push_back(GemmEntry{a_off, x_row, (int32_t)k, (int32_t)lda, trans, 0});
    tasks[t].e_end = (int32_t)entries.size();
  };

  {  // near field: every leaf, so that every row of Y is written
    std::vector<int32_t> ids;
    for (int64_t i = 0; i < v.n_leaves; ++i) {
      const int64_t a = fl + i;
      if (h->size[a] == 0) continue;
      const int32_t t = new_task(h->begin[a], h->size[a], 0, a, PH_NEAR);
      for (int64_t e = d->near_ptr[i]; e < d->near_ptr[i + 1]; ++e) {
        const int64_t b = fl + d->near_idx[e];
        add_entry(t, near_off[e], h->begin[b], h->size[b], h->size[b], 0);
      }
      ids.push_back(t);
    }
    add_phase(PH_NEAR, d->levels, MAT_USER, MAT_USER, ids, XMAP_PERM);
  }
  {  // upward pass, leaves
    std::vector<int32_t> ids;
    for (int64_t a = fl; a < v.n_nodes; ++a) {
      if (h->rank[a] == 0) continue;
      const int32_t t = new_task(h->skel_off[a], h->rank[a], 0, a, PH_UP_LEAF);
      add_entry(t, basis_off[a], h->begin[a], h->size[a], h->rank[a], 1);
      ids.push_back(t);
    }
    add_phase(PH_UP_LEAF, d->levels, MAT_USER, MAT_SKEL_W, ids, XMAP_PERM);
  }
  for (int32_t level = d->levels - 1; level >= 1; --level) {  // upward pass, inner levels
    std::vector<int32_t> ids;
    for (int64_t a = ((int64_t)1 << level) - 1; a < ((int64_t)2 << level) - 1; ++a) {
      if (h->rank[a] == 0) continue;
      const int32_t t = new_task(h->skel_off[a], h->rank[a], 0, a, PH_UP_TRANS);
      add_entry(t, basis_off[a], h->skel_off[2 * a + 1], rows_of(a), h->rank[a], 1);
      ids.push_back(t);
    }
    add_phase(PH_UP_TRANS, level, MAT_SKEL_W, MAT_SKEL_W, ids, XMAP_NONE);
  }
  {  // far field: every node with a basis (also initialises u for the downward pass)
    std::vector<int32_t> ids;
    for (int64_t a = 1; a < v.n_nodes; ++a) {
      if (h->rank[a] == 0) continue;
      const int32_t t = new_task(h->skel_off[a], h->rank[a], 0, a, PH_COUPLING);
      if (far_task_off[a] >= 0) add_entry(t, far_task_off[a], far_rows_off[a], far_k[a], far_k[a], 0);
      ids.push_back(t);
    }
    add_phase(PH_COUPLING, 0, MAT_SKEL_W, MAT_SKEL_U, ids, XMAP_FAR);
  }
  for (int32_t level = 1; level < d->levels; ++level) {  // downward pass, inner levels
    std::vector<int32_t> ids;
    for (int64_t a = ((int64_t)1 << level) - 1; a < ((int64_t)2 << level) - 1; ++a) {
      if (h->rank[a] == 0 || rows_of(a) == 0) continue;
      const int32_t t = new_task(h->skel_off[2 * a + 1], rows_of(a), 1, a, PH_DOWN_TRANS);
      add_entry(t, basis_off[a], h->skel_off[a], h->rank[a], h->rank[a], 0);
      ids.push_back(t);
    }
    add_phase(PH_DOWN_TRANS, level, MAT_SKEL_U, MAT_SKEL_U, ids, XMAP_NONE);
  }
  {  // downward pass, leaves (adds into Y)
    std::vector<int32_t> ids;
    for (int64_t a = fl; a < v.n_nodes; ++a) {
      if (h->rank[a] == 0 || h->size[a] == 0) continue;
      const int32_t t = new_task(h->begin[a], h->size[a], 1, a, PH_DOWN_LEAF);
      add_entry(t, basis_off[a], h->skel_off[a], h->rank[a], h->rank[a], 0);
      ids.push_back(t);
    }
    add_phase(PH_DOWN_LEAF, d->levels, MAT_SKEL_U, MAT_USER, ids, XMAP_NONE);
  }

  // ---- the FP64 far chain: 16-row tiles of every far-field task (appended to the tile
  // array), longest first within a (step, level)
  std::vector<ChainItem> items64[4];  // per ChainKind, in (level, cost) order within
  {
    const int L = d->levels;
    std::vector<std::vector<std::pair<int64_t, int32_t>>> by(4 * (L + 1));
    for (size_t t = 0; t < tasks.size(); ++t) {
      const PhaseKind k = task_kind[t];
      if (k == PH_NEAR) continue;
      const int ck = (k == PH_UP_LEAF || k == PH_UP_TRANS) ? CK_UP
                     : k == PH_COUPLING ? CK_CPL : (k == PH_DOWN_TRANS ? CK_DN : CK_LEAF);
      int64_t kk = 0;
      for (int32_t e = tasks[t].e_begin; e < tasks[t].e_end; ++e) kk += entries[e].k;
      by[ck * (L + 1) + level_of(task_node[t])].push_back({std::max<int64_t>(kk, 1), (int32_t)t});
    }
    for (int ck = 0; ck < 4; ++ck)
      for (int l = 0; l <= L; ++l) {
        auto& b = by[ck * (L + 1) + l];
        std::stable_sort(b.begin(), b.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
        for (const auto& p : b) {
          const int32_t t = p.second;
          for (int32_t m0 = 0; m0 < tasks[t].m; m0 += 16) {
            items64[ck].push_back(ChainItem{(int32_t)tiles.size(), task_node[t], (uint8_t)ck, 0, (uint8_t)l,
                                            (uint8_t)(ck == CK_CPL ? 1 : 0)});
            tiles.push_back(GemmTile{t, m0});
          }
        }
      }
  }

  // ---- device allocations and upload
  auto fail = [&](cudaError_t e) -> hmat_status {
    free_device(h.get());
    return cuda_status(e);
  };
  cudaError_t e = cudaMalloc((void**)&h->arena, (size_t)h->arena_values * sizeof(double));
  if (e != cudaSuccess) return fail(e);
  h->device_bytes += h->arena_values * (int64_t)sizeof(double);
  {
    Uploader up;
    if ((e = up.init(h->arena, (size_t)1 << 23)) != cudaSuccess) return fail(e);
    bool finite = true;
    cudaError_t ce = cudaSuccess;
    if (!src) {
      for (int64_t i = 0; i < v.n_leaves && ce == cudaSuccess; ++i)
        for (int64_t ee = d->near_ptr[i]; ee < d->near_ptr[i + 1] && ce == cudaSuccess; ++ee) {
          const int64_t cnt = h->size[fl + i] * h->size[fl + d->near_idx[ee]];
          finite &= up.put(near_off[ee], d->near[ee], cnt, &ce);
        }
    }
    for (int64_t a = 0; a < v.n_nodes && ce == cudaSuccess; ++a)
      if (h->rank[a] > 0) finite &= up.put(basis_off[a], d->basis[a], rows_of(a) * h->rank[a], &ce);
    if (!src) {
      for (int64_t a = 0; a < v.n_nodes && ce == cudaSuccess; ++a) {
        if (far_task_off[a] < 0) continue;
        for (int32_t r = 0; r < h->rank[a] && ce == cudaSuccess; ++r)
          for (int64_t ee = d->far_ptr[a]; ee < d->far_ptr[a + 1] && ce == cudaSuccess; ++ee) {
            const int32_t sb = h->rank[d->far_idx[ee]];
            if (sb > 0)
              finite &= up.put(far_task_off[a] + r * far_k[a] + far_off[ee], d->coupling[ee] + (int64_t)r * sb, sb,
                               &ce);
          }
      }
    }
    if (ce == cudaSuccess) ce = up.finish();
    if (ce != cudaSuccess) return fail(ce);
    if (!finite) { free_device(h.get()); return HMAT_EINVAL; }
  }
  if (src) {  // evaluate D (unless on the fly) and B on the device from the points
    std::vector<BlockJob> jobs;
    for (int64_t i = 0; i < v.n_leaves && !near_otf; ++i)
      for (int64_t ee = d->near_ptr[i]; ee < d->near_ptr[i + 1]; ++ee) {
        const int64_t a = fl + i, b = fl + d->near_idx[ee];
        if (h->size[a] * h->size[b] == 0) continue;
        jobs.push_back(BlockJob{near_off[ee], h->size[b], h->begin[a], h->begin[b], (int32_t)h->size[a],
                                (int32_t)h->size[b], 0, 0});
      }
    for (int64_t a = 0; a < v.n_nodes; ++a)
      for (int64_t ee = d->far_ptr[a]; ee < d->far_ptr[a + 1]; ++ee) {
        const int64_t b = d->far_idx[ee];
        if ((int64_t)h->rank[a] * h->rank[b] == 0) continue;
        jobs.push_back(BlockJob{far_task_off[a] + far_off[ee], far_k[a], h->skel_off[a], h->skel_off[b], h->rank[a],
                                h->rank[b], 1, 1});
      }
    std::vector<double> pts(src->points_tree, src->points_tree + d->n_points * (int64_t)src->dim);
    std::vector<int64_t> skel(src->skel_points, src->skel_points + h->sum_rank);
    double* dpts = nullptr;
    int64_t* dskel = nullptr;
    BlockJob* djobs = nullptr;
    int64_t scratch = 0;
    cudaError_t ce = upload(&dpts, pts, &scratch);
    if (ce == cudaSuccess) ce = upload(&dskel, skel, &scratch);
    if (ce == cudaSuccess) ce = upload(&djobs, jobs, &scratch);
    if (ce == cudaSuccess && !jobs.empty())
      ce = launch_eval_blocks(djobs, (int64_t)jobs.size(), dpts, src->dim, dskel, src->kernel, src->kernel_param,
                              h->arena, 0);
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    if (ce == cudaSuccess && near_otf) {  // the near field keeps the points
      h->near_otf = true;
      h->pts_tree = dpts;
      h->dim = src->dim;
      h->kernel = src->kernel;
      h->kernel_param = src->kernel_param;
      h->device_bytes += (int64_t)pts.size() * (int64_t)sizeof(double);
    } else {
      cudaFree(dpts);
    }
    cudaFree(dskel);
    cudaFree(djobs);
    if (ce != cudaSuccess) return fail(ce);
  }
  std::vector<int64_t> perm(d->perm, d->perm + d->n_points);
  if ((e = upload(&h->perm, perm, &h->device_bytes)) != cudaSuccess) return fail(e);
  if ((e = upload(&h->far_rows, far_rows_host, &h->device_bytes)) != cudaSuccess) return fail(e);
  if ((e = upload(&h->tasks, tasks, &h->device_bytes)) != cudaSuccess) return fail(e);
  if ((e = upload(&h->entries, entries, &h->device_bytes)) != cudaSuccess) return fail(e);
  if ((e = upload(&h->tiles, tiles, &h->device_bytes)) != cudaSuccess) return fail(e);
  h->n_tiles = (int64_t)tiles.size();
  std::vector<int> zero(1, 0);
  if ((e = upload(&h->status, zero, &h->device_bytes)) != cudaSuccess) return fail(e);
  if (flags & HMAT_LOAD_MIXED) {
    hmat_status ms = build_mixed(h.get(), d, v, near_off, far_task_off, far_off, far_k, tasks, entries, tiles);
    if (ms == HMAT_OK) ms = build_chain(h.get(), v, tiles, task_node);
    if (ms == HMAT_OK && (flags & HMAT_LOAD_MIXED_ONLY)) {
      // the mixed mode reads only its own copies: the FP64 blocks are dropped
      cudaFree(h->arena);
      h->arena = nullptr;
      h->device_bytes -= h->arena_values * (int64_t)sizeof(double);
      h->has_fp64 = false;
    }
    if (ms != HMAT_OK) {
      free_device(h.get());
      return ms;
    }
  }
  {
    hmat_status cs = build_chain64(h.get(), v, items64);
    if (cs != HMAT_OK) {
      free_device(h.get());
      return cs;
    }
  }
  if ((e = noalloc_scratch_address(&h->noalloc_scratch)) != cudaSuccess) return fail(e);
  {
    hmat_status cs = ctx_create(*h, &h->ctx);
    if (cs != HMAT_OK) {
      free_device(h.get());
      return cs;
    }
  }
  *out = h.release();
  return HMAT_OK;
}

}  // namespace hmat

extern "C" hmat_status hmat_load(const hmat_desc* d, int flags, hmat_t* out) {
  if (!out) return HMAT_EINVAL;
  *out = nullptr;
  return load_impl(d, nullptr, flags, out);
}

extern "C" hmat_status hmat_structure(hmat_t h, int64_t* perm, int32_t* rank, int64_t* near_ptr, int32_t* near_idx,
                                      int64_t* far_ptr, int32_t* far_idx) {
  if (!h) return HMAT_EINVAL;
  auto put = [](auto* dst, const auto& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  put(perm, h->perm_host);
  put(rank, h->rank);
  put(near_ptr, h->near_ptr);
  put(near_idx, h->near_idx);
  put(far_ptr, h->far_ptr);
  put(far_idx, h->far_idx);
  return HMAT_OK;
}

extern "C" hmat_status hmat_status_poll(hmat_t h, void* stream) {
  if (!h) return HMAT_EINVAL;
  int word = 0;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(&word, h->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word != 0) e = cudaMemset(h->status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_status(e);
  return (hmat_status)word;
}

extern "C" hmat_status hmat_selftest_timeout(hmat_t h, int64_t limit_ns, void* stream) {
  if (!h || limit_ns <= 0 || limit_ns > 10000000000LL) return HMAT_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (dev != h->device) return HMAT_EINVAL;
  return cuda_status(launch_wait_selftest(h->status, (uint64_t)limit_ns, (cudaStream_t)stream));
}

extern "C" hmat_status hmat_info(hmat_t h, int64_t* out, int n_out) {
  if (!h || !out || n_out < 0) return HMAT_EINVAL;
  const int64_t held = h->device_bytes + (h->ctx ? h->ctx->block_bytes + 2 * h->ctx->host_cap : 0);
  const int64_t engine = !h->has_mixed ? 0 : (h->tc_coupling ? 2 : 1);
  const int64_t vals[11] = {h->n_points, h->levels,          h->n_near,          h->n_far,
                            h->near_values, h->basis_values, h->coupling_values, h->sum_rank,
                            held,           engine,          h->near_otf ? 1 : 0};
  for (int i = 0; i < n_out && i < 11; ++i) out[i] = vals[i];
  return HMAT_OK;
}

extern "C" hmat_status hmat_free(hmat_t h) {
  if (!h) return HMAT_OK;
  cudaDeviceSynchronize();
  free_device(h);
  delete h;
  return HMAT_OK;
}

extern "C" const char* hmat_strerror(hmat_status s) {
  switch (s) {
    case HMAT_OK: return "success";
    case HMAT_EINVAL: return "invalid argument or HMatrix description";
    case HMAT_ENOMEM: return "out of memory";
    case HMAT_ECUDA: return "CUDA runtime error";
    case HMAT_ETIMEOUT: return "a bounded device-side wait gave up";
    case HMAT_EUNSUPPORTED: return "unsupported request";
    case HMAT_EDEVICE: return "a kernel found an inconsistent index or size";
    case HMAT_EBUSY: return "the server's queue is full";
  }
  return "unknown status";
}
