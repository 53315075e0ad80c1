// Mixed-precision products on the tcgen05 tensor cores (HMAT_MODE_MIXED): the
// near-field reduction Y_i = sum_j D_ij W_j and the far-field coupling reduction
// u_a = sum_b B_ab w_b (Section 2.1, "Evaluation"). Both are lists of dense
// contractions per target, so one kernel serves both:
//
//  * A (D or B) and X (W or w) are split into two FP16 terms, x ~= hi + lo with
//    hi = fp16(x) and lo = fp16(x - hi), after a power-of-two scaling that puts the
//    largest |value| of an A m-tile (128 rows of one target, over its whole list) and
//    of X into [2^13, 2^14): 22 significant bits per value, no overflow, no
//    subnormal lo for values down to 2^-16 of the maximum;
//  * Y_t = sum_s (Ah Xh + Ah Xl + Al Xh), the dropped Al Xl term is 2^-22 relative;
//  * the tensor core's FP32 accumulator truncates (rounds toward zero, measured on
//    this GPU), so the dominant Ah Xh product is accumulated in TMEM over a few blocks
//    only (near field: whole blocks up to 512 summed terms; coupling: two blocks) and then
//    drained by the epilogue warps into a compensated FP32 (hi, lo)
//    pair per output (hi in registers, lo in TMEM columns 384..511); the two small
//    cross terms (2^-11 of the result) accumulate over the whole list in a second
//    TMEM accumulator.
//
// Operands are packed once (A at load, X per evaluation) in the canonical K-major
// 128-byte-swizzled tcgen05 layout, so one cp.async.bulk (TMA) copy per tile lands
// it in shared memory. Warp roles: warp 0 issues the bulk copies of the A tiles and
// warp 10 those of the X tiles (bulk copies issued by one thread are processed about
// one at a time, ~0.2 us each, so two issuers nearly double the copy rate), warp 1
// issues the MMAs (one thread) and owns the TMEM allocation, warps 2..9 drain the
// accumulators and write the output. All waits are bounded; on a timeout the kernel
// records HMAT_ETIMEOUT in the status word, lets its own copies and MMAs finish,
// frees its TMEM and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "hmat_fp.cuh"
#include "hmat_internal.h"

namespace hmat {
namespace {

constexpr int kStages = 3;
constexpr int kStageBytes = 65536;           // A hi+lo (32 KB) + B hi+lo (<= 32 KB)
constexpr int kTcThreads = 352;              // warps 0/10 copies, warp 1 MMAs, warps 2..9 epilogue
constexpr int kMaxNt = 128;                  // columns of W per CTA (MMA N)
constexpr uint32_t kTmemCols = 512;          // main[0], main[1], cross, compensation terms
constexpr uint64_t kWaitNs = 2000000000ull;  // give up a wait after 2 s
constexpr int kScaleTop = 13;                // scaled maxima land in [2^13, 2^14)
constexpr int kDrainChunks = 8;              // near field: a drain follows the block that brings the
                                             // accumulator to 8 k-chunks (512 summed terms)
constexpr int kDrainBlocksFar = 2;           // coupling: a drain every 2 blocks (its partners' ranks
                                             // vary; longer groups cost accuracy where it is tightest)
constexpr int kStagedEntries = 1024;         // list entries whose metadata a CTA keeps in shared memory

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `bar` with the given parity; false after limit_ns or when
// another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t limit_ns = kWaitNs) {
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 31) == 31) {
      if (*abort_flag) return false;
      const uint64_t t = gtimer();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both K-major.
__device__ __forceinline__ uint32_t idesc_f16(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this warp's 32 lanes: one FP32 value per column per
// thread. The registers pass through the wait so that no use is scheduled before it.
#define HMAT_R16(r) "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
    "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
#define HMAT_RW16(r) "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), \
    "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
#define HMAT_LD16 "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(HMAT_LD16 : HMAT_R16(r) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" : HMAT_RW16(r)::"memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float* va, float* vb) {
  uint32_t r[16], t[16];
  asm volatile(HMAT_LD16 : HMAT_R16(r) : "r"(ta));
  asm volatile(HMAT_LD16 : HMAT_R16(t) : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" : HMAT_RW16(r), HMAT_RW16(t)::"memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    va[j] = __uint_as_float(r[j]);
    vb[j] = __uint_as_float(t[j]);
  }
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Exact sum of two FP32 values as s + err (Knuth's TwoSum), err added to the low part.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// The scale exponent from the bits of a non-negative maximum (as k_absmax stores it), on the
// integer units: the exponent field of a normal value is ilogb + 1023; zero, subnormal and
// non-finite maxima take the FP64 path.
__device__ __forceinline__ int scale_exponent_bits(unsigned long long bits);

__device__ __forceinline__ int scale_exponent(double maxabs) {
  return maxabs > 0.0 ? kScaleTop - ilogb(maxabs) : 0;
}

static __device__ __noinline__ double pow2_hw(int k) { return ldexp(1.0, k); }

__device__ __forceinline__ int scale_exponent_bits(unsigned long long bits) {
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex != 0 && ex != 0x7FF) return kScaleTop - (ex - 1023);
  return scale_exponent(__longlong_as_double((long long)bits));
}

// Byte offset of FP16 value (row r, column k) inside a 128-row x 64-column SW128 tile.
__device__ __forceinline__ int sw128_chunk(int r, int chunk) { return r * 128 + ((chunk ^ (r & 7)) << 4); }

__device__ __forceinline__ void split_fp16(double x, __half& hi, __half& lo) {
  hi = __double2half(x);
  lo = __double2half(x - (double)__half2float(hi));
}

__device__ double block_max_d(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
  if (threadIdx.x < 32)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------------ load-time packing

// Scale exponent of one m-tile: the largest |value| over the tile's rows of every
// block of the target's list.
__global__ void __launch_bounds__(256) k_tc_scale(TcLists tc, const int64_t* __restrict__ blk_off,
                                                  const int32_t* __restrict__ blk_ld, const double* __restrict__ arena,
                                                  const int32_t* __restrict__ mtile_node,
                                                  const int32_t* __restrict__ mtile_mt, int32_t* __restrict__ out) {
  const int t = blockIdx.x;
  const int node = mtile_node[t], mt = mtile_mt[t];
  const int n_i = tc.size[node];
  const int r0 = mt * kTcRows, r1 = min(n_i, r0 + kTcRows);
  double m = 0.0;
  for (int64_t e = tc.ptr[node]; e < tc.ptr[node + 1]; ++e) {
    const int n_j = tc.size[tc.idx[e]];
    if (n_j == 0) continue;
    const double* B = arena + blk_off[e];
    const int64_t ld = blk_ld[e];
    const int64_t cnt = (int64_t)(r1 - r0) * n_j;
    for (int64_t x = threadIdx.x; x < cnt; x += blockDim.x) {
      const int64_t r = r0 + x / n_j, c = x % n_j;
      m = fmax(m, fabs(B[r * ld + c]));
    }
  }
  m = block_max_d(m);
  if (threadIdx.x == 0) out[t] = scale_exponent(m);
}

// One (entry, m-tile, k-chunk): scaled FP64 values -> FP16 hi and lo SW128 tiles.
__global__ void __launch_bounds__(256) k_tc_pack(const TcPackJob* __restrict__ jobs, const double* __restrict__ arena,
                                                 const int32_t* __restrict__ scale, uint8_t* __restrict__ tiles) {
  const TcPackJob job = jobs[blockIdx.x];
  const int k = scale[job.scale_idx];
  uint8_t* hi_t = tiles + job.dst;
  uint8_t* lo_t = hi_t + kTcTileBytes;
  for (int task = threadIdx.x; task < kTcRows * 8; task += blockDim.x) {
    const int r = task >> 3, ck = task & 7;
    const int gr = job.r0 + r;
    __align__(16) __half hv[8], lv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int gk = job.k0 + ck * 8 + t;
      double x = 0.0;
      if (gr < job.rows && gk < job.cols) x = ldexp(arena[job.src + (int64_t)gr * job.ld + gk], k);
      split_fp16(x, hv[t], lv[t]);
    }
    const int off = sw128_chunk(r, ck);
    *reinterpret_cast<uint4*>(hi_t + off) = *reinterpret_cast<const uint4*>(hv);
    *reinterpret_cast<uint4*>(lo_t + off) = *reinterpret_cast<const uint4*>(lv);
  }
}

// one CTA per block
__global__ void k_relayout_f32(const double* __restrict__ arena, const F32Job* __restrict__ jobs,
                               float* __restrict__ dst) {
  const F32Job j = jobs[blockIdx.x];
  const double* src = arena + j.src_off;
  float* out = dst + j.dst_off;
  const int64_t n = (int64_t)j.k * j.ld;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t k = i / j.ld, m = i % j.ld;
    out[i] = m < j.m_rows ? (float)(j.trans ? src[k * j.lda + m] : src[m * j.lda + k]) : 0.0f;
  }
}

// ------------------------------------------------------------------ per-evaluation W split

// |x| as an unsigned integer that orders like |x| (IEEE magnitudes order as their bit
// patterns), NaN as 0 so that it sets no scale: the maximum then runs on the integer
// units (FP64 compares and conversions run at 1/64 rate on this GPU).
__device__ __forceinline__ uint64_t abs_key_bits(uint64_t bits) {
  const uint64_t b = bits & 0x7FFFFFFFFFFFFFFFull;
  return b <= 0x7FF0000000000000ull ? b : 0;
}
__device__ __forceinline__ uint32_t abs_key_bits(uint32_t bits) {
  const uint32_t b = bits & 0x7FFFFFFFu;
  return b <= 0x7F800000u ? b : 0;
}
__device__ __forceinline__ uint64_t abs_key(double x) { return abs_key_bits((uint64_t)__double_as_longlong(x)); }
__device__ __forceinline__ uint32_t abs_key(float x) { return abs_key_bits(__float_as_uint(x)); }
__device__ __forceinline__ double key_value(uint64_t k) { return __longlong_as_double((long long)k); }
__device__ __forceinline__ double key_value(uint32_t k) { return (double)__uint_as_float(k); }

// max |X| over n values: 16-byte loads, four in flight per thread and iteration (few
// registers, so that every SM holds enough loads in flight to stream at HBM rate)
// (block bid of nb blocks working on X)
template <typename T>
__device__ __forceinline__ void absmax_body(const T* __restrict__ X, int64_t n, unsigned long long* __restrict__ out,
                                            int64_t bid, int64_t nb) {
  using Key = decltype(abs_key(T{}));
  constexpr int kPer = 16 / (int)sizeof(T);
  const int64_t stride = nb * blockDim.x;
  const int64_t tid = bid * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n_vec = ((uintptr_t)X & 15u) == 0 ? n / kPer : 0;
  const uint4* V = reinterpret_cast<const uint4*>(X);
  Key m = 0;
  auto upd = [&m](const uint4& u) {
    Key k[kPer];
    if constexpr (sizeof(T) == 8) {
      k[0] = abs_key_bits((uint64_t)u.x | ((uint64_t)u.y << 32));
      k[1] = abs_key_bits((uint64_t)u.z | ((uint64_t)u.w << 32));
    } else {
      k[0] = abs_key_bits(u.x);
      k[1] = abs_key_bits(u.y);
      k[2] = abs_key_bits(u.z);
      k[3] = abs_key_bits(u.w);
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) m = k[j] > m ? k[j] : m;
  };
  int64_t i = tid;
  for (; i + 3 * stride < n_vec; i += 4 * stride) {
    const uint4 a = V[i], b = V[i + stride], c = V[i + 2 * stride], d = V[i + 3 * stride];
    upd(a);
    upd(b);
    upd(c);
    upd(d);
  }
  for (; i < n_vec; i += stride) upd(V[i]);
  for (int64_t j = n_vec * kPer + tid; j < n; j += stride) {
    const Key k = abs_key(X[j]);
    m = k > m ? k : m;
  }
  const double mm = block_max_d(key_value(m));
  if (threadIdx.x == 0 && mm > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mm));
}

template <typename T>
__global__ void __launch_bounds__(256) k_absmax(const T* __restrict__ X, int64_t n,
                                                unsigned long long* __restrict__ out) {
  absmax_body<T>(X, n, out, blockIdx.x, gridDim.x);
}

// The member of a multi-member launch that block b belongs to: the first j with
// block_end[j] > b; *first receives the block's index within the member.
__device__ __forceinline__ int member_of(const int64_t* __restrict__ block_end, int n, int64_t b, int64_t* first) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (block_end[mid] > b) hi = mid;
    else lo = mid + 1;
  }
  *first = lo > 0 ? block_end[lo - 1] : 0;
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) k_absmax_multi(const AbsJob* __restrict__ jobs,
                                                      const int64_t* __restrict__ block_end, int n_jobs) {
  int64_t first;
  const int j = member_of(block_end, n_jobs, blockIdx.x, &first);
  const AbsJob job = jobs[j];
  absmax_body<T>(static_cast<const T*>(job.X), job.n, job.out, blockIdx.x - first, block_end[j] - first);
}

// One (source k-chunk, column tile): 64 rows of X x n_t columns -> B-operand tiles:
// n_t rows (columns of X) x 64 values (rows of X), hi then lo. The near field's X is
// W (FP64 or FP32, caller order, rows through perm); there the same values, rounded to
// FP32, also go unscaled into x32, the FP32 tree-order copy the far field reads. The
// coupling's X is the FP32 skeleton weights in node order. A thread owns one column and 8 consecutive
// rows: one 16-byte chunk of each tile. FP64 arithmetic is 1/64 rate on this GPU, so
// the split itself is done in FP32 after one conversion on the integer units (24 bits
// kept, 22 needed),
// scaled in FP32: the scale is a power of two, so RN32(v) * 2^k = RN32(v * 2^k) unless
// RN32(v) is subnormal, and such values (|v| < 2^-126) scale to below half the smallest
// FP16 subnormal (both sides give 0) for every k <= 100; larger k take the FP64 path.
template <typename T>
__device__ __forceinline__ void split_body(const SplitJob& j, int64_t b) {
  const TcLists& tc = j.tc;
  const T* __restrict__ X = static_cast<const T*>(j.X);
  const int64_t* __restrict__ perm = j.perm;
  const int64_t q = j.q;
  const int n_t = j.n_t, n_ct = j.n_ct;
  const unsigned long long* __restrict__ xmax = j.xmax;
  uint8_t* __restrict__ out = j.out;
  float* __restrict__ x32 = j.x32;
  const int64_t g = b / n_ct;
  const int ct = b % n_ct;
  const int node = tc.chunk_node[g], c = tc.chunk_c[g];
  const int n_j = tc.size[node];
  const int64_t row0 = tc.begin[node] + (int64_t)c * kTcK;
  // the scale 2^k_x as FP64 and FP32 bit patterns (every thread of the split computes it:
  // FP64 ilogb, ldexp and conversions would keep the 1/64-rate FP64 pipe a quarter busy)
  const int k_x = scale_exponent_bits(*xmax);
  const double sd = k_x >= -1022 && k_x <= 1023 ? __longlong_as_double((long long)(k_x + 1023) << 52) : pow2_hw(k_x);
  const float sf = k_x >= -126 && k_x <= 127 ? __int_as_float((k_x + 127) << 23) : narrow_f64_hw(sd);
  const bool f32_scale = k_x <= 100;
  const int64_t q0 = (int64_t)ct * n_t;
  uint8_t* hi_t = out + (g * n_ct + ct) * (int64_t)(2 * n_t * 128);
  // the tile pair is assembled in shared memory and written out with linear 16-byte
  // stores (a thread's own chunks are one per 128-byte row)
  __shared__ __align__(128) uint8_t tile[2 * kMaxNt * 128];
  // the chunk's source rows, looked up once (each X load then waits on shared memory only)
  __shared__ int64_t src_row[kTcK];
  if (threadIdx.x < kTcK) {
    const int k = threadIdx.x;
    src_row[k] = c * kTcK + k < n_j ? (perm ? perm[row0 + k] : row0 + k) : -1;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < n_t * 8; x += blockDim.x) {
    const int kc = x / n_t, n = x % n_t;
    const int64_t gq = q0 + n;
    __align__(16) __half hv[8], lv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = kc * 8 + t;
      float xs = 0.0f;
      const int64_t src = src_row[k];
      if (src >= 0 && gq < q) {
        const T v = X[src * q + gq];
        float f;
        if constexpr (sizeof(T) == 8)
          f = narrow_f64<true>((double)v);
        else
          f = v;
        xs = f32_scale ? f * sf : narrow_f64_hw(mul_f64_hw((double)v, sd));
        if (x32) x32[(row0 + k) * q + gq] = f;
      }
      hv[t] = __float2half_rn(xs);
      lv[t] = __float2half_rn(xs - __half2float(hv[t]));
    }
    const int off = sw128_chunk(n, kc);
    *reinterpret_cast<uint4*>(tile + off) = *reinterpret_cast<const uint4*>(hv);
    *reinterpret_cast<uint4*>(tile + n_t * 128 + off) = *reinterpret_cast<const uint4*>(lv);
  }
  __syncthreads();
  const uint4* src = reinterpret_cast<const uint4*>(tile);
  uint4* dst = reinterpret_cast<uint4*>(hi_t);
  for (int i = threadIdx.x; i < n_t * 16; i += blockDim.x) dst[i] = src[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_split(const SplitJob j) {
  split_body<T>(j, blockIdx.x);
}

// one 32-bit word per thread: a job or argument block copied into shared memory
template <typename S>
__device__ __forceinline__ void copy_words(S* dst, const S* src) {
  const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d32 = reinterpret_cast<uint32_t*>(dst);
  for (int w = threadIdx.x; w < (int)(sizeof(S) / 4); w += blockDim.x) d32[w] = s32[w];
}

template <typename T>
__global__ void __launch_bounds__(256) k_split_multi(const SplitJob* __restrict__ jobs,
                                                     const int64_t* __restrict__ block_end, int n_jobs) {
  __shared__ SplitJob sj;
  int64_t first;
  const int jx = member_of(block_end, n_jobs, blockIdx.x, &first);
  copy_words(&sj, jobs + jx);
  __syncthreads();
  split_body<T>(sj, blockIdx.x - first);
}

// ------------------------------------------------------------------ the tensor-core product kernel

// coupling output when 2^-(k_a + k_x) is no normal FP32 number (out of line: see hmat_fp.cuh)
static __device__ __noinline__ float far_out_hw(float hi, float t, double sc) {
  return __double2float_rn(((double)hi + (double)t) * sc);
}



// Y_t = sum over the list of target t of A_ts X_s, for one (target, m-tile, column
// tile). kFar = false: the near field (A = D, X = W, Y FP64 in caller order);
// kFar = true: the coupling reduction (A = B, X = skeleton weights w, Y = the FP32
// skeleton potentials u, written in node order).
// Many products in one launch (batches): block b works for the member j with
// block_end[j - 1] <= b < block_end[j] (each member's blocks: its work items x column tiles).
struct TcMulti {
  const TcArgs* args;        // null: one product, the kernel parameter
  const int64_t* block_end;
  int n;
};

// kMulti: a launch over many products (the batch); single launches read their arguments
// straight from the kernel parameters
template <bool kFar, bool kMulti>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc(const __grid_constant__ TcArgs a0, const TcMulti mm) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], mfull_bar[2], mempty_bar[2], cfull_bar,
      done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ volatile int issued_a, issued_b, consumed;
  // per list entry: k-chunks of its source, byte offset of its A tiles, its first X chunk
  __shared__ int32_t s_kc[kStagedEntries];
  __shared__ int64_t s_aoff[kStagedEntries], s_g0[kStagedEntries];
  __shared__ int s_nb;

  __shared__ TcArgs sa;  // multi-member launches: this block's member
  int64_t blk = blockIdx.x;
  if constexpr (kMulti) {
    int64_t first;
    const int j = member_of(mm.block_end, mm.n, blk, &first);
    copy_words(&sa, mm.args + j);
    blk -= first;
    __syncthreads();
  }
  const TcArgs& a = kMulti ? sa : a0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TcTile work = a.tc.work[blk / a.n_ct];
  const int ct = blk % a.n_ct;
  const int tgt = work.node, mt = work.mt;
  const int64_t e0 = a.tc.ptr[tgt], e1 = a.tc.ptr[tgt + 1];
  const uint32_t b_bytes = 2u * (uint32_t)a.n_t * 128u;
  const uint32_t a_bytes = 2u * kTcTileBytes;

  // The roles walk the target's list one entry at a time; its metadata (two dependent
  // global loads per entry) is loaded once, by every thread together, before they start.
  if (threadIdx.x == 0) s_nb = 0;
  __syncthreads();
  {
    int cnt = 0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int j = a.tc.idx[e];
      const int kc = a.tc.kc[j];
      cnt += kc > 0;
      const int64_t i = e - e0;
      if (i < kStagedEntries) {
        s_kc[i] = kc;
        s_aoff[i] = a.tc.a_off[e];
        s_g0[i] = a.tc.kcum[j];
      }
    }
    if (cnt) atomicAdd(&s_nb, cnt);
  }
  auto ent_kc = [&](int64_t e) -> int {
    const int64_t i = e - e0;
    return i < kStagedEntries ? s_kc[i] : a.tc.kc[a.tc.idx[e]];
  };
  auto ent_aoff = [&](int64_t e) -> int64_t {
    const int64_t i = e - e0;
    return i < kStagedEntries ? s_aoff[i] : a.tc.a_off[e];
  };
  auto ent_g0 = [&](int64_t e) -> int64_t {
    const int64_t i = e - e0;
    return i < kStagedEntries ? s_g0[i] : a.tc.kcum[a.tc.idx[e]];
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 2);  // the D and the W producer each arrive once per stage
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&mfull_bar[b]), 1);
      mbar_init(smem_u32(&mempty_bar[b]), 8);
    }
    mbar_init(smem_u32(&cfull_bar), 1);
    mbar_init(smem_u32(&done_bar), 1);
    abort_flag = 0;
    issued_a = 0;
    issued_b = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  auto fail = [&]() {
    abort_flag = 1;
    atomicCAS(a.status, 0, (int)HMAT_ETIMEOUT);
  };

  if (warp == 0 || warp == 10) {
    // ---- producers: warp 0 copies the A tile pair, warp 10 the X tile pair of every k-chunk
    if (lane == 0) {
      const bool is_d = warp == 0;
      int it = 0;
      bool ok = true;
      for (int64_t e = e0; e < e1 && ok; ++e) {
        const int kc = ent_kc(e);
        if (kc == 0) continue;
        const uint8_t* abase = a.tc.tiles + ent_aoff(e) + (int64_t)mt * kc * a_bytes;
        const int64_t g0 = ent_g0(e);
        for (int c = 0; c < kc; ++c, ++it) {
          const int s = it % kStages, r = it / kStages;
          if (r > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (r - 1) & 1, &abort_flag)) {
            fail();
            ok = false;
            break;
          }
          const uint32_t st = smem_u32(smem + s * kStageBytes);
          if (is_d) {
            mbar_expect_tx(smem_u32(&full_bar[s]), a_bytes);
            bulk_g2s(st, abase + (int64_t)c * a_bytes, a_bytes, smem_u32(&full_bar[s]));
            issued_a = it + 1;
          } else {
            mbar_expect_tx(smem_u32(&full_bar[s]), b_bytes);
            bulk_g2s(st + a_bytes, a.bsplit + ((g0 + c) * a.n_ct + ct) * (int64_t)b_bytes, b_bytes,
                     smem_u32(&full_bar[s]));
            issued_b = it + 1;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: main[b] = Ah*Xh over the blocks of a drain group, cross += Ah*Xl + Al*Xh
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(kTcRows, a.n_t);
      const uint32_t cross = tmem + 256;
      const int nb = s_nb;  // blocks with data
      int it = 0, blk = 0, grp = 0, gch = 0, gbk = 0;  // k-chunks and blocks in the current drain group
      bool ok = true;
      for (int64_t e = e0; e < e1 && ok; ++e) {
        const int kc = ent_kc(e);
        if (kc == 0) continue;
        const int b = grp & 1, rb = grp >> 1;
        const bool first_of_group = gbk == 0;
        if (first_of_group && rb > 0 && !mbar_wait(smem_u32(&mempty_bar[b]), (rb - 1) & 1, &abort_flag)) {
          fail();
          ok = false;
          break;
        }
        fence_after();
        const uint32_t main_acc = tmem + (uint32_t)b * 128;
        for (int c = 0; c < kc; ++c, ++it) {
          const int s = it % kStages, r = it / kStages;
          if (!mbar_wait(smem_u32(&full_bar[s]), r & 1, &abort_flag)) {
            fail();
            ok = false;
            break;
          }
          fence_after();
          const uint32_t st = smem_u32(smem + s * kStageBytes);
          const uint32_t a_hi = st, a_lo = st + kTcTileBytes;
          const uint32_t b_hi = st + 2 * kTcTileBytes, b_lo = b_hi + (uint32_t)a.n_t * 128;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t o = kk * 32;
            mma_f16(main_acc, desc_sw128(a_hi + o), desc_sw128(b_hi + o), idesc,
                    (first_of_group && c == 0 && kk == 0) ? 0u : 1u);
            mma_f16(cross, desc_sw128(a_hi + o), desc_sw128(b_lo + o), idesc, (it | kk) ? 1u : 0u);
            mma_f16(cross, desc_sw128(a_lo + o), desc_sw128(b_hi + o), idesc, 1u);
          }
          mma_commit(smem_u32(&empty_bar[s]));
          consumed = it + 1;
        }
        if (!ok) break;
        ++blk;
        gch += kc;
        ++gbk;
        if ((kFar ? gbk >= kDrainBlocksFar : gch >= kDrainChunks) || blk == nb) {
          mma_commit(smem_u32(&mfull_bar[b]));
          ++grp;
          gch = 0;
          gbk = 0;
        }
      }
      if (ok && blk > 0) mma_commit(smem_u32(&cfull_bar));
      mma_commit(smem_u32(&done_bar));
      uint64_t t0 = gtimer();
      while (!mbar_try(smem_u32(&done_bar), 0) && gtimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp >= 2 && warp <= 9) {
    // ---- epilogue: warp w drains TMEM lanes 32*(w%4).. of column half (w-2)/4
    const int eq = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(eq * 32) << 16;
    const uint32_t comp = tmem + lane_base + 384 + half * 64;  // this warp's compensation terms
    float hi[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) hi[j] = 0.0f;
    {
      float z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0.0f;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) tmem_st16(comp + cc * 16, z);
    }
    const int nb = s_nb;  // blocks with data
    int n_groups = 0;     // drain groups, cut as the MMA issuer cuts them
    {
      int g = 0, gb = 0, bb = 0;
      for (int64_t e = e0; e < e1; ++e) {
        const int kc = ent_kc(e);
        if (kc == 0) continue;
        g += kc;
        ++gb;
        ++bb;
        if ((kFar ? gb >= kDrainBlocksFar : g >= kDrainChunks) || bb == nb) {
          ++n_groups;
          g = 0;
          gb = 0;
        }
      }
    }
    int blk = 0;
    bool ok = true;
    for (int grp = 0; grp < n_groups; ++grp) {
      const int b = grp & 1, rb = grp >> 1;
      // every lane must agree before the warp-collective TMEM loads
      if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&mfull_bar[b]), rb & 1, &abort_flag))) {
        if (lane == 0) fail();
        ok = false;
        break;
      }
      fence_after();
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        float v[16], l[16];
        tmem_ld16x2(tmem + lane_base + (uint32_t)(b * 128 + half * 64 + cc * 16), comp + cc * 16, v, l);
#pragma unroll
        for (int j = 0; j < 16; ++j) two_sum_acc(hi[cc * 16 + j], l[j], v[j]);
        tmem_st16(comp + cc * 16, l);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&mempty_bar[b]));
      ++blk;  // drains done
    }
    bool have_cross = false;
    if (ok && blk > 0) {
      if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&cfull_bar), 0, &abort_flag))) {
        if (lane == 0) fail();
        ok = false;
      } else {
        fence_after();
        have_cross = true;
      }
    }
    const int row = mt * kTcRows + eq * 32 + lane;
    const bool write = ok && row < a.tc.size[tgt];
    const int k_a = a.tc.scale[a.tc.mt_base[tgt] + mt];
    const int k_x = scale_exponent(__longlong_as_double((long long)*a.bmax));
    const double sc = ldexp(1.0, -(k_a + k_x));
    // coupling: FP32 output, combined and scaled in FP32 (exact power-of-two scale while
    // 2^-(k_a + k_x) is a normal FP32 number); near field: FP64 output, the two small
    // terms (|l + v| ~ 2^-11 |hi|) added in FP32 first, then widened and scaled on the
    // integer units around one DADD
    const int e_sc = -(k_a + k_x);
    const bool f32_out = kFar && e_sc >= -126 && e_sc <= 127;
    const float scf = f32_out ? __int_as_float((e_sc + 127) << 23) : 0.0f;
    const int64_t out_row = write ? (kFar ? a.tc.begin[tgt] + row : a.perm[a.tc.begin[tgt] + row]) : 0;
    const int64_t c0 = (int64_t)ct * a.n_t + half * 64;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      float v[16], l[16];
      if (have_cross) {
        tmem_ld16x2(comp + cc * 16, tmem + lane_base + (uint32_t)(256 + half * 64 + cc * 16), l, v);
      } else {
        tmem_ld16(comp + cc * 16, l);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.0f;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = cc * 16 + j;
        const int64_t gc = c0 + col;
        if (write && half * 64 + col < a.n_t && gc < a.q) {
          const float t = __fadd_rn(l[j], v[j]);
          if constexpr (kFar) {
            static_cast<float*>(a.Y)[out_row * a.q + gc] =
                f32_out ? __fmul_rn(__fadd_rn(hi[col], t), scf) : far_out_hw(hi[col], t, sc);
          } else {
            const double y = scale_pow2(widen_f32(hi[col]) + widen_f32(t), e_sc, sc);
            if (a.y_f32)
              static_cast<float*>(a.Y)[out_row * a.q + gc] = narrow_f64(y);
            else
              static_cast<double*>(a.Y)[out_row * a.q + gc] = y;
          }
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) {
    // let the bulk copies this CTA issued land before its shared memory goes away (a stage
    // whose second copy was never issued cannot complete: its wait ends at the time limit)
    const int issued = issued_a > issued_b ? issued_a : issued_b;
    for (int it = consumed; it < issued; ++it) {
      const uint64_t t0 = gtimer();
      while (!mbar_try(smem_u32(&full_bar[it % kStages]), (it / kStages) & 1) && gtimer() - t0 < kWaitNs) {
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// Failure-detection self-test: one thread waits, through the routine every wait of
// k_tc uses, on a barrier that nothing arrives at; the wait gives up after
// limit_ns and the status word gets HMAT_ETIMEOUT as a stuck evaluation would set it.
// No copy or MMA is in flight, so returning is all the clean-up there is.
__global__ void k_wait_selftest(int* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x != 0) return;
  mbar_init(smem_u32(&bar), 1);
  abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(smem_u32(&bar), 0, &abort_flag, limit_ns)) atomicCAS(status, 0, (int)HMAT_ETIMEOUT);
}

}  // namespace

// ------------------------------------------------------------------ launchers

cudaError_t launch_tc_scale(const TcLists& tc, const int64_t* blk_off, const int32_t* blk_ld, const double* arena,
                            int64_t n_mtiles, const int32_t* mtile_node, const int32_t* mtile_mt, int32_t* scale_out,
                            cudaStream_t stream) {
  if (n_mtiles == 0) return cudaSuccess;
  if (n_mtiles > 2147483647LL) return cudaErrorInvalidValue;
  k_tc_scale<<<(unsigned)n_mtiles, 256, 0, stream>>>(tc, blk_off, blk_ld, arena, mtile_node, mtile_mt, scale_out);
  return cudaGetLastError();
}

cudaError_t launch_tc_pack(const TcPackJob* jobs, int64_t n_jobs, const double* arena, const int32_t* scale,
                           uint8_t* tiles, cudaStream_t stream) {
  if (n_jobs == 0) return cudaSuccess;
  if (n_jobs > 2147483647LL) return cudaErrorInvalidValue;
  k_tc_pack<<<(unsigned)n_jobs, 256, 0, stream>>>(jobs, arena, scale, tiles);
  return cudaGetLastError();
}

cudaError_t launch_relayout_f32(const double* arena, const F32Job* jobs, int64_t n_jobs, float* dst,
                                cudaStream_t stream) {
  if (n_jobs == 0) return cudaSuccess;
  if (n_jobs > 2147483647LL) return cudaErrorInvalidValue;
  k_relayout_f32<<<(unsigned)n_jobs, 256, 0, stream>>>(arena, jobs, dst);
  return cudaGetLastError();
}

namespace {

template <typename T>
cudaError_t launch_split(const TcProduct& p, const T* X, int64_t n_values, const int64_t* perm, int64_t q, int n_t,
                         int n_ct, unsigned long long* xmax, uint8_t* out, float* x32, cudaStream_t stream) {
  if (n_t <= 0 || n_t > kMaxNt || n_t % 16 != 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(xmax, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  k_absmax<T><<<(unsigned)absmax_blocks(n_values), 256, 0, stream>>>(X, n_values, xmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t grid = p.n_chunks * n_ct;
  if (grid == 0) return cudaSuccess;
  if (grid > 2147483647LL) return cudaErrorInvalidValue;
  k_split<T><<<(unsigned)grid, 256, 0, stream>>>(SplitJob{p.dev, X, perm, q, n_t, n_ct, xmax, out, x32});
  return cudaGetLastError();
}

template <bool kFar>
cudaError_t launch_tc(const TcProduct& p, const uint8_t* bsplit, const unsigned long long* bmax, const int64_t* perm,
                      void* Y, bool y_f32, int64_t q, int n_t, int n_ct, int* status, cudaStream_t stream) {
  if (p.n_work == 0) return cudaSuccess;
  if (n_t <= 0 || n_t > kMaxNt || n_t % 16 != 0) return cudaErrorInvalidValue;
  const int64_t grid = p.n_work * n_ct;
  if (grid > 2147483647LL) return cudaErrorInvalidValue;
  const int smem = kStages * kStageBytes + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_tc<kFar, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  TcArgs args{p.dev, bsplit, bmax, perm, Y, q, n_t, n_ct, status, y_f32 ? 1 : 0};
  k_tc<kFar, false><<<(unsigned)grid, kTcThreads, smem, stream>>>(args, TcMulti{nullptr, nullptr, 0});
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_absmax_multi(bool f32, const AbsJob* jobs, const int64_t* block_end, int n, int64_t blocks,
                                cudaStream_t stream) {
  if (n <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  if (f32)
    k_absmax_multi<float><<<(unsigned)blocks, 256, 0, stream>>>(jobs, block_end, n);
  else
    k_absmax_multi<double><<<(unsigned)blocks, 256, 0, stream>>>(jobs, block_end, n);
  return cudaGetLastError();
}

cudaError_t launch_split_multi(bool f32, const SplitJob* jobs, const int64_t* block_end, int n, int64_t blocks,
                               cudaStream_t stream) {
  if (n <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  if (f32)
    k_split_multi<float><<<(unsigned)blocks, 256, 0, stream>>>(jobs, block_end, n);
  else
    k_split_multi<double><<<(unsigned)blocks, 256, 0, stream>>>(jobs, block_end, n);
  return cudaGetLastError();
}

cudaError_t launch_tc_multi(bool far, const TcArgs* args, const int64_t* block_end, int n, int64_t blocks,
                            cudaStream_t stream) {
  if (n <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  const int smem = kStages * kStageBytes + 1024;
  auto kern = far ? k_tc<true, true> : k_tc<false, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, kTcThreads, smem, stream>>>(TcArgs{}, TcMulti{args, block_end, n});
  return cudaGetLastError();
}

cudaError_t launch_split_f64(const TcProduct& p, const double* X, int64_t n_values, const int64_t* perm, int64_t q,
                             int n_t, int n_ct, unsigned long long* xmax, uint8_t* out, float* x32,
                             cudaStream_t stream) {
  return launch_split<double>(p, X, n_values, perm, q, n_t, n_ct, xmax, out, x32, stream);
}

cudaError_t launch_split_f32(const TcProduct& p, const float* X, int64_t n_values, const int64_t* perm, int64_t q,
                             int n_t, int n_ct, unsigned long long* xmax, uint8_t* out, float* x32,
                             cudaStream_t stream) {
  return launch_split<float>(p, X, n_values, perm, q, n_t, n_ct, xmax, out, x32, stream);
}

cudaError_t launch_tc_near(const TcProduct& p, const uint8_t* bsplit, const unsigned long long* bmax,
                           const int64_t* perm, void* Y, bool y_f32, int64_t q, int n_t, int n_ct, int* status,
                           cudaStream_t stream) {
  return launch_tc<false>(p, bsplit, bmax, perm, Y, y_f32, q, n_t, n_ct, status, stream);
}

cudaError_t launch_tc_far(const TcProduct& p, const uint8_t* bsplit, const unsigned long long* bmax, float* U,
                          int64_t q, int n_t, int n_ct, int* status, cudaStream_t stream) {
  return launch_tc<true>(p, bsplit, bmax, nullptr, U, false, q, n_t, n_ct, status, stream);
}

namespace {

__global__ void __launch_bounds__(256) k_widen(const float* __restrict__ src, double* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = widen_f32<true>(src[i]);
}

__global__ void __launch_bounds__(256) k_narrow(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = narrow_f64<true>(src[i]);
}

}  // namespace

cudaError_t launch_widen(const float* src, double* dst, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_widen<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, stream>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_narrow(const double* src, float* dst, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_narrow<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, stream>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* status, uint64_t limit_ns, cudaStream_t stream) {
  k_wait_selftest<<<1, 32, 0, stream>>>(status, limit_ns);
  return cudaGetLastError();
}

}  // namespace hmat
