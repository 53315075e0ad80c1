// FP64 evaluation kernels: one grouped ("owner computes") GEMM that serves every
// step of the evaluation (Section 2.1): the near-field reduction over D, the
// upward pass over the bases, the far-field reduction over B and the downward
// pass. A CTA owns one row tile of one output block and one column tile of the
// right-hand side and walks the block's list of terms, so no two CTAs write the
// same output and no atomics are needed (the role blocking plays in Algorithm 1).
//
// On GB300 the FP64 pipe retires about 2 DFMA per clock per SM, 1/64 of FP32,
// so these kernels are bound by DFMA issue and not by memory: register tiles of
// 4x4 outputs per thread, double-buffered shared-memory operand tiles, and
// column tiles matched to q so that no DFMA is spent on padding columns.
#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace hmat {
namespace {

constexpr int BK = 16;   // depth of one operand chunk
constexpr int TM = 4;    // outputs per thread: TM rows x TN columns
constexpr int TN = 4;

// BM rows (the phase's tile_rows) x BN right-hand-side columns per CTA.
template <int BM, int BN>
struct Cfg {
  static constexpr int kThreads = (BM / TM) * (BN / TN);
  static constexpr int kAPer = BM * BK / kThreads;  // A values loaded per thread per chunk
  static constexpr int kXPer = BN * BK / kThreads;  // X values loaded per thread per chunk
};

__device__ __forceinline__ int64_t map_row(const int64_t* __restrict__ m, int64_t r) { return m ? m[r] : r; }

// The grid is one-dimensional: CTA b works on tile b / n_col_tiles and column tile
// b % n_col_tiles, so the column tiles of one output block run side by side and
// read each block of A from HBM once (the others hit L2).
template <int BM, int BN>
__global__ void __launch_bounds__(Cfg<BM, BN>::kThreads)
k_fp64_grouped_gemm(const GemmTile* __restrict__ tiles, const GemmTask* __restrict__ tasks,
                    const GemmEntry* __restrict__ entries, const double* __restrict__ arena,
                    const double* X, const int64_t* __restrict__ x_map,
                    double* Y, const int64_t* __restrict__ y_map, int64_t q, int n_col_tiles) {
  using C = Cfg<BM, BN>;
  constexpr int NT = C::kThreads;
  constexpr int TX = BN / TN;
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Xs[2][BK][BN];

  const GemmTile tile = tiles[blockIdx.x / n_col_tiles];
  const GemmTask task = tasks[tile.task];
  const int m0 = tile.m0;
  const int64_t q0 = (int64_t)(blockIdx.x % n_col_tiles) * BN;
  const int tid = threadIdx.x;
  const int ty = tid / TX, tx = tid % TX;

  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  double ra[C::kAPer], rx[C::kXPer];
  int e = task.e_begin;
  int k0 = 0;

  // Load the chunk (entry e, depth k0 .. k0+BK) into registers, zero outside the block.
  auto load_chunk = [&](int ee, int kk0) {
    const GemmEntry en = entries[ee];
    const double* a = arena + en.a_off;
#pragma unroll
    for (int t = 0; t < C::kAPer; ++t) {
      const int idx = tid + t * NT;
      int m, k;
      if (en.trans) { k = idx / BM; m = idx % BM; } else { m = idx / BK; k = idx % BK; }
      const int gm = m0 + m, gk = kk0 + k;
      double v = 0.0;
      if (gm < task.m && gk < en.k)
        v = en.trans ? a[(int64_t)gk * en.lda + gm] : a[(int64_t)gm * en.lda + gk];
      ra[t] = v;
    }
#pragma unroll
    for (int t = 0; t < C::kXPer; ++t) {
      const int idx = tid + t * NT;
      const int k = idx / BN, n = idx % BN;
      const int gk = kk0 + k;
      const int64_t gq = q0 + n;
      double v = 0.0;
      if (gk < en.k && gq < q) v = X[map_row(x_map, en.x_row + gk) * q + gq];
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
      Xs[buf][idx / BN][idx % BN] = rx[t];
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
        double av[TM], xv[TN];
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
    double* dst = Y + map_row(y_map, task.out_row + r) * q;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t c = q0 + tx * TN + j;
      if (c < q) dst[c] = task.accumulate ? dst[c] + acc[i][j] : acc[i][j];
    }
  }
}

template <int BM, int BN>
cudaError_t launch(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map, double* Y,
                   const int64_t* y_map, int64_t q, cudaStream_t s) {
  const int64_t n_col = (q + BN - 1) / BN;
  const int64_t blocks = ph.n_tiles * n_col;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  k_fp64_grouped_gemm<BM, BN><<<(unsigned)blocks, Cfg<BM, BN>::kThreads, 0, s>>>(
      h.tiles + ph.tile_begin, h.tasks, h.entries, h.arena, X, x_map, Y, y_map, q, (int)n_col);
  return cudaGetLastError();
}

template <int BM>
cudaError_t launch_bn(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map, double* Y,
                      const int64_t* y_map, int64_t q, cudaStream_t s) {
  if (q <= 16) return launch<BM, 16>(h, ph, X, x_map, Y, y_map, q, s);
  if (q <= 32) return launch<BM, 32>(h, ph, X, x_map, Y, y_map, q, s);
  return launch<BM, 64>(h, ph, X, x_map, Y, y_map, q, s);
}

}  // namespace

cudaError_t launch_fp64_phase(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map,
                              double* Y, const int64_t* y_map, int64_t q, cudaStream_t stream) {
  if (ph.n_tiles == 0 || q == 0) return cudaSuccess;
  if (q > (int64_t)INT32_MAX) return cudaErrorInvalidValue;
  switch (ph.tile_rows) {
    case 16: return launch_bn<16>(h, ph, X, x_map, Y, y_map, q, stream);
    case 32: return launch_bn<32>(h, ph, X, x_map, Y, y_map, q, stream);
    default: return launch_bn<64>(h, ph, X, x_map, Y, y_map, q, stream);
  }
}

}  // namespace hmat
