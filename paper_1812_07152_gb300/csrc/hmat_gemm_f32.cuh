// FP32 grouped GEMM of the mixed mode's upward and downward passes (and of its
// coupling reduction when the ranks are small): the owner-computes schedule of
// hmat_gemm.cuh in FP32 with operands copied into shared memory by cp.async.
#pragma once

#include <cstdint>

#include "hmat_fp.cuh"
#include "hmat_gemm.cuh"

namespace hmat {
namespace gemm {

// FP32 variant for the far field of the mixed mode. FP32 arithmetic is 64x faster
// than FP64 on GB300, so these launches are bound by memory latency along each
// task's K loop (coupling lists reach hundreds of partners). Every task of the mixed
// far field has at most one entry (the coupling blocks of a node are concatenated),
// so chunk c of a task covers depth c * BK (BK = 32 for 64 x 64 tiles, which halves their
// barriers and copy rounds per FMA, else 16). The entries index the FP32 arena, where
// every operand is k-major (A(m, k) at a[k * lda + m]) with lda a multiple of 4,
// zero-padded rows up to lda and a 16-byte aligned start, so A is copied 16 bytes
// (four rows m) at a time. The CTA splits the chunks round-robin over up to four
// groups of warps; each group copies its chunks straight into shared memory with
// cp.async, kAsyncStages - 1 chunks ahead (the row-map indices one more chunk ahead),
// and at the end the groups' partial sums are added in a fixed order. Up to 4 slices,
// at most 256 threads per CTA.
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
  static constexpr int BK = (BM >= 64 && BN >= 64) ? 32 : gemm::BK;
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

// One CTA tile of the FP32 grouped GEMM: output rows m0 .. m0 + BM - 1 of the tile's
// task, columns q0 .. q0 + BN - 1. Threads from C::kThreads on (when the CTA is wider
// than the shape) take no part but pass the CTA-wide barriers, so the persistent far
// chain can run every shape with one block size. smf: C::kSmemBytes of shared memory.
// XV: the rows of X are copied 16 bytes (four columns) at a time; needs q a multiple of 4
// and X 16-byte aligned.
template <typename TY, int BM, int BN, bool XV>
__device__ __forceinline__ void gemm_tile_f32(const GemmTile tile, const GemmTask* __restrict__ tasks,
                                              const GemmEntry* __restrict__ entries,
                                              const float* __restrict__ arena, const float* X,
                                              const int64_t* __restrict__ x_map, TY* Y,
                                              const int64_t* __restrict__ y_map, int64_t q, int64_t q0,
                                              float* smf) {
  using C = CfgF32<BM, BN>;
  constexpr int BK = C::BK;
  constexpr int NTS = C::kSliceThreads;
  constexpr int CX = BN / TN;
  constexpr int S = kAsyncStages;

  const GemmTask task = tasks[tile.task];
  const int m0 = tile.m0;
  const bool active = threadIdx.x < C::kThreads;
  const int slice = threadIdx.x / NTS, lt = threadIdx.x % NTS;
  const int ty = lt / CX, tx = lt % CX;
  float* my = smf + (active ? slice : 0) * S * C::kStageFloats;  // this slice's stages
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
  const int my_chunks = active && n_chunks > slice ? (n_chunks - slice + C::kSlices - 1) / C::kSlices : 0;
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

  if (active) {
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
  }
  __syncthreads();

  // add the slices' partial sums in a fixed order (slice 0 + 1 + 2 + 3)
  float* red = smf;  // kSlices - 1 partial tiles, reusing the stage buffers
  if (active && slice > 0) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int jj = 0; jj < TN; ++jj) red[((slice - 1) * TM * TN + i * TN + jj) * NTS + lt] = acc[i][jj];
  }
  __syncthreads();
  if (active && slice == 0) {
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
        if (c >= q) continue;
        if constexpr (sizeof(TY) == 8) {  // FP64 Y: widened on the integer units, one DADD
          const double w = widen_f32(acc[i][jj]);
          dst[c] = task.accumulate ? dst[c] + w : w;
        } else {
          dst[c] = task.accumulate ? dst[c] + acc[i][jj] : acc[i][jj];
        }
      }
    }
  }
}

}  // namespace gemm
}  // namespace hmat
