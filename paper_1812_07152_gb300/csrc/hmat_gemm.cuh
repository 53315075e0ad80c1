// Grouped ("owner computes") GEMM shared by every phase of the evaluation
// (Section 2.1): the near-field reduction over D, the upward pass over the bases,
// the far-field reduction over B and the downward pass. A CTA owns one row tile of
// one output block and one column tile of the right-hand side and walks the
// block's list of terms, so no two CTAs write the same output and no atomics are
// needed (the role blocking plays in Algorithm 1).
#pragma once

#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace hmat {
namespace gemm {

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

// The grid is one-dimensional: CTA b works on tile b / n_col_tiles and column tile
// b % n_col_tiles, so the column tiles of one output block run side by side and
// read each block of A from HBM once (the others hit L2).
//
// TA: stored block type, TX / TY: input / output matrix types, TC: the type of the
// products and sums. Entry offsets index the FP64 arena; a_shift maps them into an
// arena that holds only the values from a_shift on (the FP32 far-field copy).
template <typename TA, typename TX, typename TY, typename TC, int BM, int BN, int CTM, int CTN>
__global__ void __launch_bounds__(Cfg<BM, BN, CTM, CTN>::kThreads)
k_grouped_gemm(const GemmTile* __restrict__ tiles, const GemmTask* __restrict__ tasks,
               const GemmEntry* __restrict__ entries, const TA* __restrict__ arena, int64_t a_shift,
               const TX* X, const int64_t* __restrict__ x_map,
               TY* Y, const int64_t* __restrict__ y_map, int64_t q, int n_col_tiles) {
  using C = Cfg<BM, BN, CTM, CTN>;
  constexpr int NT = C::kThreads;
  constexpr int TM = CTM, TN = CTN;
  constexpr int CX = BN / TN;  // threads along the columns
  __shared__ TC As[2][BK][BM + 1];
  __shared__ TC Xs[2][BK][BN];

  const GemmTile tile = tiles[blockIdx.x / n_col_tiles];
  const GemmTask task = tasks[tile.task];
  const int m0 = tile.m0;
  const int64_t q0 = (int64_t)(blockIdx.x % n_col_tiles) * BN;
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
      if (gm < task.m && gk < en.k)
        v = (TC)(en.trans ? a[(int64_t)gk * en.lda + gm] : a[(int64_t)gm * en.lda + gk]);
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

template <typename TA, typename TX, typename TY, typename TC, int BM, int BN, int CTM, int CTN>
cudaError_t launch(const Handle& h, const Phase& ph, int64_t n_tiles, const TA* arena, int64_t a_shift, const TX* X,
                   const int64_t* x_map, TY* Y, const int64_t* y_map, int64_t q, cudaStream_t s) {
  const int64_t n_col = (q + BN - 1) / BN;
  const int64_t blocks = n_tiles * n_col;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  k_grouped_gemm<TA, TX, TY, TC, BM, BN, CTM, CTN><<<(unsigned)blocks, Cfg<BM, BN, CTM, CTN>::kThreads, 0, s>>>(
      h.tiles + ph.tile_begin, h.tasks, h.entries, arena, a_shift, X, x_map, Y, y_map, q, (int)n_col);
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
template <typename TA, typename TX, typename TY, typename TC>
cudaError_t launch_phase(const Handle& h, const Phase& ph, int shape, int64_t n_tiles, const TA* arena,
                         int64_t a_shift, const TX* X, const int64_t* x_map, TY* Y, const int64_t* y_map, int64_t q,
                         cudaStream_t s) {
  if (n_tiles < 0 || n_tiles > ph.n_tiles) n_tiles = ph.n_tiles;
  if (n_tiles == 0 || q == 0) return cudaSuccess;
  if (q > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  if (shape < 0) shape = default_col_shape(q);
  if (shape >= kColShapes) return cudaErrorInvalidValue;
#define HMAT_GEMM_L(BMV, BNV, TMV, TNV) \
  return launch<TA, TX, TY, TC, BMV, BNV, TMV, TNV>(h, ph, n_tiles, arena, a_shift, X, x_map, Y, y_map, q, s)
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

// FP32 variant for the far field of the mixed mode. FP32 arithmetic is 64x faster
// than FP64 on GB300, so these launches are bound by memory latency along each
// task's K loop (coupling lists reach hundreds of partners). Every task of the mixed
// far field has at most one entry (the coupling blocks of a node are concatenated),
// so chunk c of a task covers depth c * BK. The entries index the FP32 arena, where
// every operand is k-major (A(m, k) at a[k * lda + m]) with lda a multiple of 4,
// zero-padded rows up to lda and a 16-byte aligned start, so A is copied 16 bytes
// (four rows m) at a time. The CTA splits the chunks round-robin
// over up to four groups of warps; each group copies its chunks straight into shared
// memory with cp.async, kAsyncStages - 1 chunks ahead (the row-map indices one more
// chunk ahead), and at the end the groups' partial sums are added in a fixed order.
// Up to 4 slices, at most 256 threads per CTA.
constexpr int kAsyncStages = 3;

__device__ __forceinline__ void cp_async4(uint32_t smem_dst, const void* gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_dst), "l"(gsrc), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t smem_dst, const void* gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_dst), "l"(gsrc), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int BM, int BN>
struct CfgF32 {
  static constexpr int kSliceThreads = (BM / TM) * (BN / TN);
  static constexpr int kSlices = kSliceThreads >= 256 ? 1 : (256 / kSliceThreads > 4 ? 4 : 256 / kSliceThreads);
  static constexpr int kThreads = kSliceThreads * kSlices;
  static constexpr int kAPer = BM * BK / kSliceThreads;
  static constexpr int kXPer = BN * BK / kSliceThreads;
  static constexpr int kAStride = BM + 4;
  static constexpr int kStageFloats = BK * kAStride + BK * BN;
  static constexpr int kSmemBytes = kSlices * kAsyncStages * kStageFloats * 4;
  static_assert(kSliceThreads % 32 == 0, "a K slice is whole warps");
  static_assert(kXPer <= BK, "one map index per row of the chunk");
};

// XV: the rows of X are copied 16 bytes (four columns) at a time; needs q a multiple of 4
// and X 16-byte aligned.
template <typename TY, int BM, int BN, bool XV>
__global__ void __launch_bounds__(CfgF32<BM, BN>::kThreads)
k_grouped_gemm_f32(const GemmTile* __restrict__ tiles, const GemmTask* __restrict__ tasks,
                   const GemmEntry* __restrict__ entries, const float* __restrict__ arena,
                   const float* X, const int64_t* __restrict__ x_map, TY* Y, const int64_t* __restrict__ y_map,
                   int64_t q, int n_col_tiles) {
  using C = CfgF32<BM, BN>;
  constexpr int NTS = C::kSliceThreads;
  constexpr int CX = BN / TN;
  constexpr int S = kAsyncStages;
  extern __shared__ __align__(16) float smf[];

  const GemmTile tile = tiles[blockIdx.x / n_col_tiles];
  const GemmTask task = tasks[tile.task];
  const int m0 = tile.m0;
  const int64_t q0 = (int64_t)(blockIdx.x % n_col_tiles) * BN;
  const int slice = threadIdx.x / NTS, lt = threadIdx.x % NTS;
  const int ty = lt / CX, tx = lt % CX;
  float* my = smf + slice * S * C::kStageFloats;  // this slice's stages
  auto a_st = [&](int st) { return my + st * C::kStageFloats; };
  auto x_st = [&](int st) { return my + st * C::kStageFloats + BK * C::kAStride; };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;

  const bool has = task.e_begin < task.e_end;
  GemmEntry en{};
  if (has) en = entries[task.e_begin];
  const int n_chunks = has ? (en.k + BK - 1) / BK : 0;
  const int my_chunks = n_chunks > slice ? (n_chunks - slice + C::kSlices - 1) / C::kSlices : 0;
  const float* a = arena + en.a_off;

  // X row of depth gk (through the row map when there is one); one per copy of XW floats
  constexpr int AV = BM * BK / 4;           // 16-byte A copies per chunk
  constexpr int AN = (AV + NTS - 1) / NTS;  // per thread (the last ones masked when NTS > AV)
  constexpr int XW = XV ? 4 : 1;
  constexpr int XN = C::kXPer / XW;  // X copies per thread and chunk
  static_assert(C::kXPer % XW == 0 && BN % XW == 0, "whole vectors");
  int64_t rows_next[XN];
  auto load_rows = [&](int j, int64_t* rows) {
    const int c = slice + j * C::kSlices;
#pragma unroll
    for (int t = 0; t < XN; ++t) {
      const int k = (lt + t * NTS) / (BN / XW);
      const int gk = c * BK + k;
      rows[t] = (j < my_chunks && gk < en.k) ? map_row(x_map, en.x_row + gk) : 0;
    }
  };
  auto issue = [&](int j, int st, const int64_t* rows) {
    if (j >= my_chunks) return;
    const int k0 = (slice + j * C::kSlices) * BK;
    const uint32_t as = (uint32_t)__cvta_generic_to_shared(a_st(st));
    const uint32_t xs = (uint32_t)__cvta_generic_to_shared(x_st(st));
#pragma unroll
    for (int t = 0; t < AN; ++t) {
      const int idx = lt + t * NTS;
      if (AV % NTS != 0 && idx >= AV) break;
      const int k = idx / (BM / 4), m = (idx % (BM / 4)) * 4;
      const int gm = m0 + m, gk = k0 + k;
      const bool ok = gm < task.m && gk < en.k;  // gm < task.m <= lda, both multiples of 4
      const float* src = ok ? a + (int64_t)gk * en.lda + gm : arena;
      cp_async16(as + 4u * (uint32_t)(k * C::kAStride + m), src, ok);
    }
#pragma unroll
    for (int t = 0; t < XN; ++t) {
      const int idx = lt + t * NTS;
      const int k = idx / (BN / XW), n = (idx % (BN / XW)) * XW;
      const int64_t gq = q0 + n;
      const bool ok = k0 + k < en.k && gq < q;  // XV: gq < q implies gq + 3 < q
      const float* src = ok ? X + rows[t] * q + gq : X;
      if (XV)
        cp_async16(xs + 4u * (uint32_t)(k * BN + n), src, ok);
      else
        cp_async4(xs + 4u * (uint32_t)(k * BN + n), src, ok);
    }
  };

  int64_t rows_cur[XN];
  load_rows(0, rows_cur);
#pragma unroll
  for (int st = 0; st < S - 1; ++st) {
    load_rows(st + 1, rows_next);
    issue(st, st, rows_cur);
    cp_async_commit();
#pragma unroll
    for (int t = 0; t < XN; ++t) rows_cur[t] = rows_next[t];
  }
  for (int j = 0; j < my_chunks; ++j) {
    load_rows(j + S, rows_next);  // indices one chunk ahead of the next copy
    cp_async_wait<S - 2>();
    bar_sync(1 + slice, NTS);     // chunk j landed for the slice; stage (j - 1) % S is free
    issue(j + S - 1, (j + S - 1) % S, rows_cur);
    cp_async_commit();
#pragma unroll
    for (int t = 0; t < XN; ++t) rows_cur[t] = rows_next[t];
    const float* As = a_st(j % S);
    const float* Xs = x_st(j % S);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float av[TM], xv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[k * C::kAStride + ty * TM + i];
#pragma unroll
      for (int jj = 0; jj < TN; ++jj) xv[jj] = Xs[k * BN + tx * TN + jj];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) acc[i][jj] = fmaf(av[i], xv[jj], acc[i][jj]);
    }
  }
  cp_async_wait<0>();
  __syncthreads();

  // add the slices' partial sums in a fixed order (slice 0 + 1 + 2 + 3)
  float* red = smf;  // kSlices - 1 partial tiles, reusing the stage buffers
  if (slice > 0) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int jj = 0; jj < TN; ++jj) red[((slice - 1) * TM * TN + i * TN + jj) * NTS + lt] = acc[i][jj];
  }
  __syncthreads();
  if (slice == 0) {
#pragma unroll
    for (int sl = 1; sl < C::kSlices; ++sl)
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) acc[i][jj] += red[((sl - 1) * TM * TN + i * TN + jj) * NTS + lt];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int r = m0 + ty * TM + i;
      if (r >= task.m) continue;
      TY* dst = Y + map_row(y_map, task.out_row + r) * q;
#pragma unroll
      for (int jj = 0; jj < TN; ++jj) {
        const int64_t c = q0 + tx * TN + jj;
        if (c < q) dst[c] = task.accumulate ? (TY)(dst[c] + (TY)acc[i][jj]) : (TY)acc[i][jj];
      }
    }
  }
}

template <typename TY, int BM, int BN>
cudaError_t launch_f32(const Handle& h, const Phase& ph, const float* arena, const float* X,
                       const int64_t* x_map, TY* Y, const int64_t* y_map, int64_t q, cudaStream_t s) {
  using C = CfgF32<BM, BN>;
  static_assert(C::kSmemBytes >= (C::kSlices - 1) * TM * TN * C::kSliceThreads * 4, "room for the partial sums");
  const int64_t n_col = (q + BN - 1) / BN;
  const int64_t blocks = ph.n_tiles * n_col;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  const bool xv = q % 4 == 0 && ((uintptr_t)X & 15u) == 0;
  auto kern = xv ? k_grouped_gemm_f32<TY, BM, BN, true> : k_grouped_gemm_f32<TY, BM, BN, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, C::kThreads, C::kSmemBytes, s>>>(h.tiles + ph.tile_begin, h.tasks, h.entries32, arena, X,
                                                            x_map, Y, y_map, q, (int)n_col);
  return cudaGetLastError();
}

// One launch of a far-field phase in FP32 (tasks with at most one entry each): 32, 64 or
// (64-row tiles, q > 256) 128 columns per CTA.
template <typename TY>
cudaError_t launch_phase_f32(const Handle& h, const Phase& ph, const float* arena, const float* X,
                             const int64_t* x_map, TY* Y, const int64_t* y_map, int64_t q, cudaStream_t s) {
  if (ph.n_tiles == 0 || q == 0) return cudaSuccess;
  if (q > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
#define HMAT_GEMM_BN32(BMV)                                                                       \
  if (q <= 32) return launch_f32<TY, BMV, 32>(h, ph, arena, X, x_map, Y, y_map, q, s);  \
  return launch_f32<TY, BMV, 64>(h, ph, arena, X, x_map, Y, y_map, q, s);
  switch (ph.tile_rows) {
    case 16: { HMAT_GEMM_BN32(16) }
    case 32: { HMAT_GEMM_BN32(32) }
    default: {
      // wide q: 128-column tiles read each block of A half as often (measured faster for
      // q = 512, no different for q = 256)
      if (q > 256) return launch_f32<TY, 64, 128>(h, ph, arena, X, x_map, Y, y_map, q, s);
      HMAT_GEMM_BN32(64)
    }
  }
#undef HMAT_GEMM_BN32
}

}  // namespace gemm
}  // namespace hmat
