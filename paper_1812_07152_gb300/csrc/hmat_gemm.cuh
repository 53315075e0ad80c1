// Grouped ("owner computes") GEMM shared by every phase of the evaluation
// (Section 2.1): the near-field reduction over D, the upward pass over the bases,
// the far-field reduction over B and the downward pass. A CTA owns one row tile of
// one output block and one column tile of the right-hand side and walks the
// block's list of terms, so no two CTAs write the same output and no atomics are
// needed (the role blocking plays in Algorithm 1).
#pragma once

#include <cuda_runtime.h>

#include "hmat_internal.h"
#include "hmat_kernels.cuh"

namespace hmat {
namespace gemm {

// Near blocks evaluated on the fly: A(m, k) of a near entry is K(x_{out_row + m},
// x_{x_row + k}) over the tree-ordered points.
struct OtfArgs {
  const double* pts;
  int32_t dim;
  KernelSpec ks;
};

// out of line: inlined into every unrolled operand load of every tile shape, the kernel
// functions made the translation unit take minutes to compile; an entry costs tens of
// FP64 operations, so the call adds little
static __device__ __noinline__ double otf_entry(const OtfArgs& otf, int64_t row, int64_t col) {
  return kernel_entry(otf.ks, otf.pts + row * otf.dim, otf.pts + col * otf.dim, otf.dim);
}

constexpr int BK = 16;   // depth of one operand chunk
constexpr int TM = 4;    // FP32 kernel: outputs per thread, TM rows x TN columns
constexpr int TN = 4;

// FP64 kernel column tiles: BN right-hand-side columns per CTA, each thread holding
// CTM rows x CTN columns of the output tile. The narrow shapes (BN < 16) serve small
// q, where a 16-wide tile would spend most DFMAs on padding columns. Every shape
// sums each output over the same depth order, so all give bitwise the same result.
constexpr int kColShapes = 7;
constexpr int kColBN[kColShapes] = {1, 2, 4, 8, 16, 32, 64};

// BM rows (the launch's tile_rows) x BN columns per CTA, CTM x CTN outputs per thread.
template <int BM, int BN, int CTM, int CTN>
struct Cfg {
  static constexpr int kThreads = (BM / CTM) * (BN / CTN);
  static constexpr int kAPer = BM * BK / kThreads;                   // A values loaded per thread per chunk
  static constexpr int kXPer = (BN * BK + kThreads - 1) / kThreads;  // X values (the last ones guarded)
  static_assert(BM * BK % kThreads == 0, "whole A chunk per thread");
};

__device__ __forceinline__ int64_t map_row(const int64_t* __restrict__ m, int64_t r) { return m ? m[r] : r; }

// One CTA tile: output rows m0 .. m0 + BM - 1 of the tile's task, columns q0 .. q0 + BN - 1;
// the CTA has exactly Cfg::kThreads threads.
//
// TA: stored block type, TX / TY: input / output matrix types, TC: the type of the
// products and sums. Entry offsets index the FP64 arena; a_shift maps them into an
// arena that holds only the values from a_shift on. kOtf: the blocks are not read but
// evaluated from the points (`otf`), entry by entry, as the build evaluates them.
template <typename TA, typename TX, typename TY, typename TC, int BM, int BN, int CTM, int CTN, bool kOtf>
__device__ __forceinline__ void gemm_tile(const GemmTile tile, const GemmTask* __restrict__ tasks,
                                          const GemmEntry* __restrict__ entries, const TA* __restrict__ arena,
                                          int64_t a_shift, const TX* X, const int64_t* __restrict__ x_map, TY* Y,
                                          const int64_t* __restrict__ y_map, int64_t q, int64_t q0,
                                          const OtfArgs& otf) {
  using C = Cfg<BM, BN, CTM, CTN>;
  constexpr int NT = C::kThreads;
  constexpr int TM = CTM, TN = CTN;
  constexpr int CX = BN / TN;  // threads along the columns
  __shared__ TC As[2][BK][BM + 1];
  __shared__ TC Xs[2][BK][BN];

  const GemmTask task = tasks[tile.task];
  const int m0 = tile.m0;
  const int tid = threadIdx.x;
  const int ty = tid / CX, tx = tid % CX;

  TC acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = TC(0);

  TC ra[C::kAPer], rx[C::kXPer];
  int e = task.e_begin;
  int k0 = 0;

  // Load the chunk (entry e, depth k0 .. k0+BK) into registers, zero outside the block.
  auto load_chunk = [&](int ee, int kk0) {
    const GemmEntry en = entries[ee];
    const TA* a = arena + (en.a_off - a_shift);
#pragma unroll
    for (int t = 0; t < C::kAPer; ++t) {
      const int idx = tid + t * NT;
      int m, k;
      if (en.trans) { k = idx / BM; m = idx % BM; } else { m = idx / BK; k = idx % BK; }
      const int gm = m0 + m, gk = kk0 + k;
      TC v = TC(0);
      if (gm < task.m && gk < en.k) {
        if constexpr (kOtf)
          v = (TC)otf_entry(otf, task.out_row + gm, en.x_row + gk);
        else
          v = (TC)(en.trans ? a[(int64_t)gk * en.lda + gm] : a[(int64_t)gm * en.lda + gk]);
      }
      ra[t] = v;
    }
#pragma unroll
    for (int t = 0; t < C::kXPer; ++t) {
      const int idx = tid + t * NT;
      const int k = idx / BN, n = idx % BN;
      const int gk = kk0 + k;
      const int64_t gq = q0 + n;
      TC v = TC(0);
      if (idx < BN * BK && gk < en.k && gq < q) v = (TC)X[map_row(x_map, en.x_row + gk) * q + gq];
      rx[t] = v;
    }
  };
  auto store_chunk = [&](int buf, int trans) {
#pragma unroll
    for (int t = 0; t < C::kAPer; ++t) {
      const int idx = tid + t * NT;
      int m, k;
      if (trans) { k = idx / BM; m = idx % BM; } else { m = idx / BK; k = idx % BK; }
      As[buf][k][m] = ra[t];
    }
#pragma unroll
    for (int t = 0; t < C::kXPer; ++t) {
      const int idx = tid + t * NT;
      if (idx < BN * BK) Xs[buf][idx / BN][idx % BN] = rx[t];
    }
  };

  if (e < task.e_end) {
    load_chunk(e, k0);
    int buf = 0;
    while (true) {
      store_chunk(buf, entries[e].trans);
      __syncthreads();
      // advance to the next chunk and start its loads before computing this one
      k0 += BK;
      if (k0 >= entries[e].k) { ++e; k0 = 0; }
      const bool more = e < task.e_end;
      if (more) load_chunk(e, k0);
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        TC av[TM], xv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = As[buf][k][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) xv[j] = Xs[buf][k][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], xv[j], acc[i][j]);
      }
      if (!more) break;
      buf ^= 1;
    }
  }

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + ty * TM + i;
    if (r >= task.m) continue;
    TY* dst = Y + map_row(y_map, task.out_row + r) * q;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t c = q0 + tx * TN + j;
      if (c < q) dst[c] = task.accumulate ? (TY)(dst[c] + (TY)acc[i][j]) : (TY)acc[i][j];
    }
  }
}

// The grid is one-dimensional: CTA b works on tile b / n_col_tiles and column tile
// b % n_col_tiles, so the column tiles of one output block run side by side and
// read each block of A from HBM once (the others hit L2).
template <typename TA, typename TX, typename TY, typename TC, int BM, int BN, int CTM, int CTN, bool kOtf>
__global__ void __launch_bounds__(Cfg<BM, BN, CTM, CTN>::kThreads)
k_grouped_gemm(const GemmTile* __restrict__ tiles, const GemmTask* __restrict__ tasks,
               const GemmEntry* __restrict__ entries, const TA* __restrict__ arena, int64_t a_shift,
               const TX* X, const int64_t* __restrict__ x_map,
               TY* Y, const int64_t* __restrict__ y_map, int64_t q, int n_col_tiles, OtfArgs otf) {
  gemm_tile<TA, TX, TY, TC, BM, BN, CTM, CTN, kOtf>(tiles[blockIdx.x / n_col_tiles], tasks, entries, arena, a_shift,
                                                     X, x_map, Y, y_map, q,
                                                     (int64_t)(blockIdx.x % n_col_tiles) * BN, otf);
}

template <typename TA, typename TX, typename TY, typename TC, int BM, int BN, int CTM, int CTN, bool kOtf>
cudaError_t launch(const Handle& h, const Phase& ph, int64_t n_tiles, const TA* arena, int64_t a_shift, const TX* X,
                   const int64_t* x_map, TY* Y, const int64_t* y_map, int64_t q, cudaStream_t s) {
  const int64_t n_col = (q + BN - 1) / BN;
  const int64_t blocks = n_tiles * n_col;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  if (kOtf && !h.pts_tree) return cudaErrorInvalidValue;
  const OtfArgs otf{h.pts_tree, h.dim, kernel_spec(h.kernel, h.kernel_param)};
  k_grouped_gemm<TA, TX, TY, TC, BM, BN, CTM, CTN, kOtf><<<(unsigned)blocks, Cfg<BM, BN, CTM, CTN>::kThreads, 0, s>>>(
      h.tiles + ph.tile_begin, h.tasks, h.entries, arena, a_shift, X, x_map, Y, y_map, q, (int)n_col, otf);
  return cudaGetLastError();
}

// The column shape used when none was tuned: the narrowest tile that holds q.
inline int default_col_shape(int64_t q) {
  for (int c = 0; c < kColShapes; ++c)
    if (kColBN[c] >= q) return c;
  return kColShapes - 1;
}

// One launch of a phase: the tile-row class of the launch picks BM, `shape` (an index
// into kColBN, or -1 for the default) the column tile. `n_tiles` (at most the phase's)
// limits the launch to the first tiles of the phase, the longest ones (the tuner times
// such prefixes of long phases).
template <typename TA, typename TX, typename TY, typename TC, bool kOtf = false>
cudaError_t launch_phase(const Handle& h, const Phase& ph, int shape, int64_t n_tiles, const TA* arena,
                         int64_t a_shift, const TX* X, const int64_t* x_map, TY* Y, const int64_t* y_map, int64_t q,
                         cudaStream_t s) {
  if (n_tiles < 0 || n_tiles > ph.n_tiles) n_tiles = ph.n_tiles;
  if (n_tiles == 0 || q == 0) return cudaSuccess;
  if (q > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  if (shape < 0) shape = default_col_shape(q);
  if (shape >= kColShapes) return cudaErrorInvalidValue;
#define HMAT_GEMM_L(BMV, BNV, TMV, TNV) \
  return launch<TA, TX, TY, TC, BMV, BNV, TMV, TNV, kOtf>(h, ph, n_tiles, arena, a_shift, X, x_map, Y, y_map, q, s)
#define HMAT_GEMM_BN(BMV)                      \
  switch (shape) {                             \
    case 0: HMAT_GEMM_L(BMV, 1, 1, 1);         \
    case 1: HMAT_GEMM_L(BMV, 2, 1, 1);         \
    case 2: HMAT_GEMM_L(BMV, 4, 2, 1);         \
    case 3: HMAT_GEMM_L(BMV, 8, 2, 2);         \
    case 4: HMAT_GEMM_L(BMV, 16, 4, 4);        \
    case 5: HMAT_GEMM_L(BMV, 32, 4, 4);        \
    default: HMAT_GEMM_L(BMV, 64, 4, 4);       \
  }
  switch (ph.tile_rows) {
    case 16: HMAT_GEMM_BN(16)
    case 32: HMAT_GEMM_BN(32)
    default: HMAT_GEMM_BN(64)
  }
#undef HMAT_GEMM_BN
#undef HMAT_GEMM_L
}

}  // namespace gemm
}  // namespace hmat
