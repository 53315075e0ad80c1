// hmat_autotune: picks the tile shapes of one HMatrix's evaluation for one q and mode
// by timing the candidates on the device (CUDA events on the caller's stream).
//
// FP64 mode: per near-field launch (one per row-tile size), the column tile of the
// grouped GEMM among the widths 1..64 that waste less than half of a tile on padding,
// then the column tile of the far chain timed on whole chain launches. Mixed mode: the column width of the tensor-core near-field
// CTAs (the number of CTAs that share one D tile), then the number of CTAs of the
// persistent far chain, timed on whole evaluations. Every candidate sums each output
// in the same order, so a tuned evaluation gives bitwise the result of an untuned one;
// only launch shapes change.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hmat_internal.h"

using namespace hmat;

namespace {

// A long launch is timed on a prefix of its tiles (the longest ones, tiles are sorted
// by cost) sized to about this many milliseconds with the default shape, but never
// fewer tiles than give the widest candidate kSampleWaves CTAs per SM (a prefix that
// does not fill the GPU would time latency, not throughput).
constexpr double kSampleMs = 20.0;
constexpr int kSampleWaves = 4;
constexpr int kRepeats = 3;

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {}
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  bool init() { return cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess; }
  // best of kRepeats runs of fn (after one untimed run), in ms; < 0 on error
  template <typename F>
  double best(F fn) {
    if (fn() != cudaSuccess) return -1;
    double t = 1e30;
    for (int r = 0; r < kRepeats; ++r) {
      if (cudaEventRecord(a, s) != cudaSuccess || fn() != cudaSuccess || cudaEventRecord(b, s) != cudaSuccess ||
          cudaEventSynchronize(b) != cudaSuccess)
        return -1;
      float ms = 0;
      if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return -1;
      t = std::min(t, (double)ms);
    }
    return t;
  }
};

// Column shapes worth trying for q: no more than half a tile of padding, and not
// narrower than min(8, q) rounded down to a power of two (narrower tiles re-read A).
std::vector<int> fp64_candidates(int64_t q) {
  std::vector<int> out;
  int64_t floor2 = 1;
  while (floor2 * 2 <= std::min<int64_t>(q, 8)) floor2 *= 2;
  for (int c = 0;; ++c) {
    const int bn = fp64_shape_columns(c);
    if (bn == 0) break;
    if (bn >= floor2 && bn < 2 * q) out.push_back(c);
  }
  const int def = fp64_default_shape(q);
  if (std::find(out.begin(), out.end(), def) == out.end()) out.push_back(def);
  return out;
}

}  // namespace

extern "C" hmat_status hmat_autotune(hmat_t h, int64_t q, int mode, void* stream, hmat_tune_report* report) {
  if (!h || q <= 0) return HMAT_EINVAL;
  if (mode != HMAT_MODE_FP64 && mode != HMAT_MODE_MIXED) return HMAT_EUNSUPPORTED;
  if (mode == HMAT_MODE_MIXED && !h->has_mixed) return HMAT_EUNSUPPORTED;
  if (mode == HMAT_MODE_FP64 && !h->has_fp64) return HMAT_EUNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HMAT_ECUDA;
  if (dev != h->device) return HMAT_EINVAL;
  if (report) *report = hmat_tune_report{q, mode, 0, 0.0, 0.0, 0, 0};
  if (h->n_points == 0) return HMAT_OK;
  cudaStream_t s = (cudaStream_t)stream;

  // private workspaces and operands (contents only need to be finite)
  EvalContext* c = nullptr;
  hmat_status st = ctx_create(*h, &c);
  if (st != HMAT_OK) return st;
  double* W = nullptr;
  double* Y = nullptr;
  const size_t bytes = (size_t)h->n_points * (size_t)q * sizeof(double);
  cudaError_t e = cudaSuccess;
  auto cleanup = [&]() {
    if (s) cudaStreamSynchronize(s);
    cudaFree(W);
    cudaFree(Y);
    ctx_destroy(c);
  };
  if ((st = ctx_reserve(*h, c, q, mode)) != HMAT_OK) {
    cleanup();
    return st;
  }
  if ((e = cudaMalloc((void**)&W, bytes)) != cudaSuccess || (e = cudaMalloc((void**)&Y, bytes)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return cuda_status(e);
  }
  // 0x3F in every byte is a normal double (about 4.8e-4)
  if ((e = cudaMemsetAsync(W, 0x3F, bytes, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(Y, 0, bytes, s)) != cudaSuccess) {
    cleanup();
    return cuda_status(e);
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cleanup();
    return HMAT_ECUDA;
  }
  Timer timer(s);
  if (!timer.init()) {
    cleanup();
    return HMAT_ECUDA;
  }

  TuneEntry entry;
  entry.q = q;
  entry.mode = mode;
  int32_t n_tuned = 0;
  int32_t near_cols = 0;
  if (mode == HMAT_MODE_FP64) {
    entry.shape.assign(h->phases.size(), -1);
    const std::vector<int> cand = fp64_candidates(q);
    for (size_t i = 0; i < h->phases.size(); ++i) {
      const Phase& ph = h->phases[i];
      if (ph.kind != PH_NEAR) continue;  // the far field runs as one chain launch (below)
      const double* X = ph.x == MAT_USER ? W : (ph.x == MAT_SKEL_W ? c->ws : c->us);
      double* Yd = ph.y == MAT_USER ? Y : (ph.y == MAT_SKEL_W ? c->ws : c->us);
      const int64_t* xm = phase_x_map(*h, ph);
      const int64_t* ym = ph.y == MAT_USER ? h->perm : nullptr;
      const int def = fp64_default_shape(q);
      int64_t n_tiles = ph.n_tiles;
      auto run = [&](int shape) { return launch_fp64_phase(*h, ph, X, xm, Yd, ym, q, shape, n_tiles, s); };
      // one timed run of the default on all tiles decides the sample
      if (cudaEventRecord(timer.a, s) != cudaSuccess || run(def) != cudaSuccess ||
          cudaEventRecord(timer.b, s) != cudaSuccess || cudaEventSynchronize(timer.b) != cudaSuccess) {
        cleanup();
        return HMAT_ECUDA;
      }
      float full_ms = 0;
      cudaEventElapsedTime(&full_ms, timer.a, timer.b);
      if (full_ms > kSampleMs) {
        int widest = 0;
        for (int shape : cand) widest = std::max(widest, fp64_shape_columns(shape));
        const int64_t n_col = (q + widest - 1) / widest;
        const int64_t fill = ((int64_t)kSampleWaves * sms + n_col - 1) / n_col;
        n_tiles = std::max<int64_t>((int64_t)std::ceil(ph.n_tiles * (kSampleMs / full_ms)), fill);
        n_tiles = std::min<int64_t>(n_tiles, ph.n_tiles);
      }
      const double scale = (double)ph.n_tiles / (double)n_tiles;
      double t_def = -1, t_best = 1e30;
      int best = def;
      for (int shape : cand) {
        const double t = timer.best([&] { return run(shape); });
        if (t < 0) {
          cleanup();
          return HMAT_ECUDA;
        }
        if (shape == def) t_def = t;
        if (t < t_best) {
          t_best = t;
          best = shape;
        }
      }
      entry.shape[i] = (int8_t)best;
      entry.default_ms += t_def * scale;
      entry.tuned_ms += t_best * scale;
      if (ph.kind == PH_NEAR) near_cols = std::max(near_cols, fp64_shape_columns(best));
      ++n_tuned;
    }
    // the far chain: its column width, timed on whole launches (near field untouched); a
    // short chain (latency-bound: thin levels, few tiles per level) also tries narrower
    // tiles, which spread each level over more CTAs
    if (h->chain64.count[0] > 0) {
      auto prev = std::find_if(h->tuned.begin(), h->tuned.end(),
                               [&](const TuneEntry& t) { return t.q == q && t.mode == mode; });
      const bool had = prev != h->tuned.end();
      const TuneEntry saved = had ? *prev : TuneEntry{};
      if (!had) h->tuned.push_back(entry);
      TuneEntry* live = &*std::find_if(h->tuned.begin(), h->tuned.end(),
                                       [&](const TuneEntry& t) { return t.q == q && t.mode == mode; });
      *live = entry;
      int grid_cap = 0;
      auto run_chain = [&](int shape) -> cudaError_t {
        live->chain_shape = shape;
        cudaError_t ce = cudaMemsetAsync(c->chain_ctr, 0, (size_t)h->chain64.n_ctr * 4, s);
        if (ce != cudaSuccess) return ce;
        return launch_chain64(chain_member64(*h, c, W, Y, q), chain_launch64(*h, c, 0, kChainWaitNs), shape,
                              grid_cap, s);
      };
      const int def = fp64_default_shape(q);
      std::vector<int> cand = fp64_candidates(q);
      const double t_def = timer.best([&] { return run_chain(def); });
      if (t_def >= 0 && t_def < 5.0)
        for (int sh = 0; sh < def; ++sh)
          if (std::find(cand.begin(), cand.end(), sh) == cand.end()) cand.push_back(sh);
      double t_best = t_def;
      int best = def;
      for (int sh : cand) {
        if (t_def < 0) break;
        if (sh == def) continue;
        const double t = timer.best([&] { return run_chain(sh); });
        if (t < 0) {
          t_best = -1;
          break;
        }
        if (t < t_best) {
          t_best = t;
          best = sh;
        }
      }
      // then the grid: fewer CTAs than the default (less waiting) or more (more warps per SM)
      int best_grid = 0;
      for (int g : {sms, 2 * sms, 4 * sms, 16 * sms, 64 * sms}) {
        if (t_best < 0) break;
        grid_cap = g;
        const double t = timer.best([&] { return run_chain(best); });
        if (t < 0) {
          t_best = -1;
          break;
        }
        if (t < t_best) {
          t_best = t;
          best_grid = g;
        }
      }
      if (had) {
        *live = saved;
      } else {
        h->tuned.erase(h->tuned.begin() + (live - &h->tuned[0]));
      }
      if (t_def < 0 || t_best < 0) {
        cleanup();
        return HMAT_ECUDA;
      }
      entry.chain_shape = best;
      entry.chain_grid = best_grid;
      entry.default_ms += t_def;
      entry.tuned_ms += t_best;
      ++n_tuned;
    }
  } else {
    const std::vector<int> cand = mixed_nt_candidates(q);
    double t_def = -1, t_best = 1e30;
    int best = cand[0];
    for (int n_t : cand) {
      const int n_ct = (int)((q + n_t - 1) / n_t);
      e = launch_split_f64(h->tc_near, W, h->n_points * q, h->perm, q, n_t, n_ct, c->wmax, c->wsplit, c->w32, s);
      if (e != cudaSuccess) {
        cleanup();
        return cuda_status(e);
      }
      const double t = timer.best([&] {
        return launch_tc_near(h->tc_near, c->wsplit, c->wmax, h->perm, Y, false, q, n_t, n_ct, h->status, s);
      });
      if (t < 0) {
        cleanup();
        return HMAT_ECUDA;
      }
      if (n_t == cand[0]) t_def = t;
      if (t < t_best) {
        t_best = t;
        best = n_t;
      }
    }
    entry.n_t = best;
    entry.default_ms = t_def;
    entry.tuned_ms = t_best;
    near_cols = best;
    n_tuned = 1;
    // the persistent far chain runs beside the near field and holds its CTAs until its
    // last item: how many it should take is timed on whole evaluations (the default is
    // every resident CTA); the result does not depend on it
    if (h->chain.count[0] + h->chain.count[1] + h->chain.count[2] > 0) {
      auto prev = std::find_if(h->tuned.begin(), h->tuned.end(),
                               [&](const TuneEntry& t) { return t.q == q && t.mode == mode; });
      const bool had = prev != h->tuned.end();
      const TuneEntry saved = had ? *prev : TuneEntry{};
      if (!had) h->tuned.push_back(entry);
      TuneEntry* live = &*std::find_if(h->tuned.begin(), h->tuned.end(),
                                       [&](const TuneEntry& t) { return t.q == q && t.mode == mode; });
      *live = entry;
      const int prof = h->profiling;
      h->profiling = 0;
      double c_def = -1, c_best = 1e30;
      int g_best = 0;
      for (int g : {0, 2 * sms, sms, sms / 2, sms / 4}) {
        live->chain_grid = g;
        const double t = timer.best([&] { return eval_impl(h, c, W, Y, q, mode, HMAT_DTYPE_F64, s) == HMAT_OK ? cudaSuccess
                                                                                              : cudaErrorUnknown; });
        if (t < 0) break;
        if (g == 0) c_def = t;
        if (t < c_best) {
          c_best = t;
          g_best = g;
        }
      }
      h->profiling = prof;
      if (had) {
        *live = saved;
      } else {
        h->tuned.erase(h->tuned.begin() + (live - &h->tuned[0]));
      }
      if (c_def < 0) {
        cleanup();
        return HMAT_ECUDA;
      }
      entry.chain_grid = g_best;
      entry.default_ms = c_def;
      entry.tuned_ms = c_best;
      n_tuned = 2;
    }
  }
  cleanup();
  // a wait that ran out inside a timed launch is an error of the call
  int dev_status = HMAT_OK;
  if (cudaMemcpy(&dev_status, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HMAT_ECUDA;
  if (dev_status != HMAT_OK) return (hmat_status)dev_status;

  auto it = std::find_if(h->tuned.begin(), h->tuned.end(),
                         [&](const TuneEntry& t) { return t.q == q && t.mode == mode; });
  if (it != h->tuned.end())
    *it = entry;
  else
    h->tuned.push_back(entry);
  if (report)
    *report = hmat_tune_report{q, mode, n_tuned, entry.default_ms, entry.tuned_ms, near_cols, entry.chain_grid};
  return HMAT_OK;
}

extern "C" hmat_status hmat_tune_apply(hmat_t h, const hmat_tune_report* choice) {
  if (!h || !choice || choice->q <= 0) return HMAT_EINVAL;
  if (choice->mode != HMAT_MODE_MIXED) return HMAT_EUNSUPPORTED;
  if (!h->has_mixed) return HMAT_EUNSUPPORTED;
  const std::vector<int> cand = mixed_nt_candidates(choice->q);
  const int n_t = choice->near_cols == 0 ? cand[0] : choice->near_cols;
  if (std::find(cand.begin(), cand.end(), n_t) == cand.end() || choice->chain_grid < 0) return HMAT_EINVAL;
  TuneEntry entry;
  entry.q = choice->q;
  entry.mode = choice->mode;
  entry.n_t = n_t;
  entry.chain_grid = choice->chain_grid;
  auto it = std::find_if(h->tuned.begin(), h->tuned.end(),
                         [&](const TuneEntry& t) { return t.q == entry.q && t.mode == entry.mode; });
  if (it != h->tuned.end())
    *it = entry;
  else
    h->tuned.push_back(entry);
  return HMAT_OK;
}
