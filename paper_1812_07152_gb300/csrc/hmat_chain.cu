// The far field of the mixed mode as persistent launches (Section 2.1's upward pass,
// far-field reduction and downward pass; the GPU counterpart of the paper's
// coarsening, Algorithm 2).
//
// One launch walks a list of CTA tiles ("items") of the FP32 grouped GEMM across
// every tree level. A CTA takes the next ticket (an atomic counter), waits until the
// items its tile depends on are complete, computes the tile with the FP32 grouped-GEMM
// body of hmat_gemm_f32.cuh, and counts it complete:
//
//   CK_UP   of node a (w_a = P_a^T [w_l; w_r])  waits for CK_UP of its children;
//   CK_CPL  of node a (u_a = sum_b B_ab w_b)    waits for every CK_UP of a's level;
//   CK_DN   of node a ([u_l; u_r] += P_a u_a)   waits for CK_CPL of a and of its
//                                               children (their u must be initialised)
//                                               and for CK_DN of a's parent;
//   CK_LEAF of leaf i (Y_i += P_i u_i)          waits for CK_CPL of i, CK_DN of its parent.
//
// Tickets are handed out in list order and every dependency names an earlier item,
// so the unfinished item with the lowest ticket always has its inputs: the launch
// cannot deadlock whatever the grid size or how many of its CTAs are resident.
// Completion counters are per node and count (row tile x column tile) items; a
// producer's thread 0 publishes after a CTA barrier and a device-scope fence, a
// consumer's thread 0 reads with acquire semantics before a CTA barrier (which orders
// the other threads' operand reads after it). Every wait
// is bounded: after limit_ns it latches HMAT_ETIMEOUT in the status word and sets
// the launch's abort flag, and every CTA then stops taking tickets.
#include <algorithm>
#include <mutex>

#include "hmat_chain.cuh"
#include "hmat_gemm_f32.cuh"

namespace hmat {
namespace {

constexpr int kChainThreads = 256;

template <int BM, int BN>
constexpr int chain_smem() {
  using C = gemm::CfgF32<BM, BN>;
  return C::kSmemBytes;
}
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kChainSmem = cmax(cmax(cmax(chain_smem<16, 32>(), chain_smem<16, 64>()),
                                     cmax(chain_smem<32, 32>(), chain_smem<32, 64>())),
                                cmax(chain_smem<64, 32>(), chain_smem<64, 64>()));

// out of line: inlined, the twelve tile shapes of a launch share one register allocation
// (210 registers, one CTA per SM); as calls each keeps its own and the kernel needs the
// largest of them
template <typename TY, int BM, int BN, bool XV>
__device__ __noinline__ void chain_tile(const ChainMember& m, const ChainItem& it, int64_t q0, const float* X,
                                        const int64_t* x_map, TY* Y, const int64_t* y_map, float* smf) {
  gemm::gemm_tile_f32<TY, BM, BN, XV>(m.tiles[it.tile], m.tasks, m.entries, m.arena, X, x_map, Y, y_map, m.q, q0,
                                      smf);
}

template <typename TY, int BN, bool XV>
__device__ __forceinline__ void chain_tile_cls(const ChainMember& m, const ChainItem& it, int64_t q0, const float* X,
                                               const int64_t* x_map, TY* Y, const int64_t* y_map, float* smf) {
  switch (it.cls) {
    case 0: chain_tile<TY, 16, BN, XV>(m, it, q0, X, x_map, Y, y_map, smf); break;
    case 1: chain_tile<TY, 32, BN, XV>(m, it, q0, X, x_map, Y, y_map, smf); break;
    default: chain_tile<TY, 64, BN, XV>(m, it, q0, X, x_map, Y, y_map, smf); break;
  }
}

template <typename TY, bool XV>
__device__ __forceinline__ void chain_tile_bn(const ChainMember& m, const ChainItem& it, int64_t q0, const float* X,
                                              const int64_t* x_map, TY* Y, const int64_t* y_map, float* smf) {
  if (m.bn == 32)
    chain_tile_cls<TY, 32, XV>(m, it, q0, X, x_map, Y, y_map, smf);
  else
    chain_tile_cls<TY, 64, XV>(m, it, q0, X, x_map, Y, y_map, smf);
}

// XV: the launch copies X rows 16 bytes at a time (q a multiple of 4); a kernel of its
// own, since those shapes need far fewer registers than the 4-byte copies
template <bool XV>
__global__ void __launch_bounds__(kChainThreads) k_chain(const __grid_constant__ ChainMember m,
                                                         const __grid_constant__ ChainLaunch l) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int s_t;
  __shared__ int s_go;
  const int total = l.n_items * m.n_ct;
  // a launch with no dependencies (the downward leaf step) is a plain grid over its items
  const bool free_run = l.waits == 0 && l.extra == 0;
  for (int k = 0;; ++k) {
    if (threadIdx.x == 0 && free_run) {
      s_t = blockIdx.x + k * gridDim.x;
      s_go = s_t < total;
    } else if (threadIdx.x == 0) {
      int go = 0, t = 0;
      if (!*(volatile int32_t*)l.abort_flag) {
        t = atomicAdd(l.ticket, 1);
        // the acquire loads of the waits order this CTA's operand reads (after the barrier
        // below) after the producers' writes
        if (t < total) go = chain_deps(m.sync, m.items[l.item_begin + t / m.n_ct], l) ? 1 : 0;
      }
      s_t = t;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const int t = s_t;
    const ChainItem it = m.items[l.item_begin + t / m.n_ct];
    const int64_t q0 = (int64_t)(t % m.n_ct) * m.bn;
    switch (it.kind) {
      case CK_UP:
        // leaves read the FP32 tree-order copy of W, inner nodes their children's w
        chain_tile_bn<float, XV>(m, it, q0, it.node >= m.first_leaf ? m.w32 : m.ws32, nullptr, m.ws32, nullptr, smf);
        break;
      case CK_CPL: chain_tile_bn<float, XV>(m, it, q0, m.ws32, m.far_rows, m.us32, nullptr, smf); break;
      case CK_DN: chain_tile_bn<float, XV>(m, it, q0, m.us32, nullptr, m.us32, nullptr, smf); break;
      default:
        if (m.y_f32)
          chain_tile_bn<float, XV>(m, it, q0, m.us32, nullptr, static_cast<float*>(m.Y), m.perm, smf);
        else
          chain_tile_bn<double, XV>(m, it, q0, m.us32, nullptr, static_cast<double*>(m.Y), m.perm, smf);
        break;
    }
    __syncthreads();  // the tile's outputs are written and its shared memory is free again
    if (threadIdx.x == 0) chain_done(m.sync, it);
  }
}

}  // namespace

namespace {

std::mutex g_chain_mu;
int g_chain_occ[2][64] = {};  // resident chain CTAs per SM, per kernel and device (0: not prepared)
int g_chain_sms[64] = {};

}  // namespace

cudaError_t chain_prepare(int* grid_v, int* grid_s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_chain_mu);
  if (g_chain_occ[0][dev] == 0) {
    int s = 0;
    e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    for (int v = 0; v < 2; ++v) {
      auto kern = v ? k_chain<true> : k_chain<false>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kChainSmem);
      int o = 0;
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kChainThreads, kChainSmem);
      if (e != cudaSuccess) return e;
      g_chain_occ[v][dev] = o > 0 ? o : 1;
    }
    g_chain_sms[dev] = s;
  }
  if (grid_v) *grid_v = g_chain_sms[dev] * g_chain_occ[1][dev];
  if (grid_s) *grid_s = g_chain_sms[dev] * g_chain_occ[0][dev];
  return cudaSuccess;
}

cudaError_t launch_chain(const ChainMember& m, const ChainLaunch& l, int grid_cap, cudaStream_t stream) {
  if (l.n_items <= 0 || m.q <= 0) return cudaSuccess;
  if (m.bn != 32 && m.bn != 64) return cudaErrorInvalidValue;
  if ((int64_t)l.n_items * m.n_ct > INT32_MAX) return cudaErrorInvalidValue;
  int full_v = 0, full_s = 0;
  cudaError_t e = chain_prepare(&full_v, &full_s);  // done at load; here it only reads the cached values
  if (e != cudaSuccess) return e;
  int64_t grid = m.xv ? full_v : full_s;
  if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
  grid = std::min<int64_t>(grid, (int64_t)l.n_items * m.n_ct);
  if (m.xv)
    k_chain<true><<<(unsigned)grid, kChainThreads, kChainSmem, stream>>>(m, l);
  else
    k_chain<false><<<(unsigned)grid, kChainThreads, kChainSmem, stream>>>(m, l);
  return cudaGetLastError();
}

}  // namespace hmat
