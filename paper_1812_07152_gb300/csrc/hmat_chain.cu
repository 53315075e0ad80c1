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

// kXV = 1: one member whose items copy X rows 16 bytes at a time (q a multiple of 4),
// 0: 4 bytes at a time, 2: many members (batches), the width per member; kernels of
// their own, since the 16-byte shapes need far fewer registers than the 4-byte ones.
template <int kXV>
__global__ void __launch_bounds__(kChainThreads) k_chain(const __grid_constant__ ChainMember m1,
                                                         const __grid_constant__ ChainLaunch l,
                                                         const __grid_constant__ ChainMulti<ChainMember> mm) {
  extern __shared__ __align__(16) float smf[];
  __shared__ ChainMember sm;  // the member of the current item
  __shared__ ChainItem s_it;
  __shared__ int64_t s_q0;
  __shared__ int s_go;
  constexpr bool multi = kXV == 2;  // multi-member launches run the per-member form
  const int64_t total = multi ? mm.total : (int64_t)l.n_items * m1.n_ct;
  // a launch with no dependencies (the downward leaf step) is a plain grid over its items
  const bool free_run = multi ? mm.free_run != 0 : (l.waits == 0 && l.extra == 0);
  int cur = -1;  // warp 0: member held in sm
  for (int k = 0;; ++k) {
    if (threadIdx.x < 32) {  // warp 0: the ticket (lane 0), the member copy (all lanes)
      int go = 0, mi = 0;
      int64_t t = 0;
      if (threadIdx.x == 0) {
        if (free_run) {
          t = blockIdx.x + (int64_t)k * gridDim.x;
          go = t < total;
        } else if (!*(volatile int32_t*)l.abort_flag) {
          t = atomicAdd(l.ticket, 1);
          go = t < total;
        }
        if constexpr (multi) {
          if (go) {
            if (mm.list) {
              mi = mm.list[t].member;
            } else {
              int lo = 0, hi = mm.n_members - 1;
              while (lo < hi) {
                const int mid = (lo + hi) / 2;
                if (mm.parts[mid].ticket_end > t) hi = mid;
                else lo = mid + 1;
              }
              mi = lo;
            }
          }
        }
      }
      if constexpr (multi) {
        if (threadIdx.x == 0 && go && (mi < 0 || mi >= mm.n_members)) {  // an inconsistent ticket list
          atomicCAS(l.status, 0, (int)HMAT_EDEVICE);
          atomicExch(l.abort_flag, 1);
          go = 0;
        }
        go = __shfl_sync(0xffffffffu, go, 0);
        mi = __shfl_sync(0xffffffffu, mi, 0);
        if (go && mi != cur) {  // one 32-bit word per lane
          const uint32_t* src = reinterpret_cast<const uint32_t*>(mm.members + mi);
          uint32_t* dst = reinterpret_cast<uint32_t*>(&sm);
          for (int w = threadIdx.x; w < (int)(sizeof(ChainMember) / 4); w += 32) dst[w] = src[w];
          cur = mi;
        }
        __syncwarp();
      }
      if (threadIdx.x == 0 && go) {
        int64_t local = t;
        uint32_t waits = l.waits;
        int32_t ib = l.item_begin;
        const ChainMember& mt = multi ? sm : m1;
        int64_t ii;
        if (multi && mm.list) {
          const ChainTicket ck = mm.list[t];
          waits = ck.waits;
          ii = ck.item;
          s_q0 = (int64_t)ck.ct * mt.bn;
        } else {
          if constexpr (multi) {
            local = t - (mi > 0 ? mm.parts[mi - 1].ticket_end : 0);
            waits = mm.parts[mi].waits;
            ib = mm.parts[mi].item_begin;
          }
          ii = ib + local / mt.n_ct;
          s_q0 = (local % mt.n_ct) * mt.bn;
        }
        // every index taken from device data is checked before it is used
        go = chain_item_ok(mt.items, ii, mt.n_items, mt.n_tiles, mt.sync.n_nodes, &s_it) ? 1 : 0;
        if (!go) {
          atomicCAS(mt.sync.status, 0, (int)HMAT_EDEVICE);
          atomicExch(l.abort_flag, 1);
        }
        // the acquire loads of the waits order this CTA's operand reads (after the barrier
        // below) after the producers' writes
        if (go && !free_run) {
          ChainLaunch lw = l;
          lw.waits = waits;
          go = chain_deps(mt.sync, s_it, lw) ? 1 : 0;
        }
      }
      if (threadIdx.x == 0) s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const ChainItem it = s_it;
    const int64_t q0 = s_q0;
    const ChainMember& m = multi ? sm : m1;
    const bool xv = kXV == 2 ? m.xv != 0 : kXV == 1;
    switch (it.kind) {
      case CK_UP: {
        // leaves read the FP32 tree-order copy of W, inner nodes their children's w
        const float* X = it.node >= m.first_leaf ? m.w32 : m.ws32;
        if (xv) chain_tile_bn<float, true>(m, it, q0, X, nullptr, m.ws32, nullptr, smf);
        else chain_tile_bn<float, false>(m, it, q0, X, nullptr, m.ws32, nullptr, smf);
        break;
      }
      case CK_CPL:
        if (xv) chain_tile_bn<float, true>(m, it, q0, m.ws32, m.far_rows, m.us32, nullptr, smf);
        else chain_tile_bn<float, false>(m, it, q0, m.ws32, m.far_rows, m.us32, nullptr, smf);
        break;
      case CK_DN:
        if (xv) chain_tile_bn<float, true>(m, it, q0, m.us32, nullptr, m.us32, nullptr, smf);
        else chain_tile_bn<float, false>(m, it, q0, m.us32, nullptr, m.us32, nullptr, smf);
        break;
      default:
        if (m.y_f32) {
          float* Y = static_cast<float*>(m.Y);
          if (xv) chain_tile_bn<float, true>(m, it, q0, m.us32, nullptr, Y, m.perm, smf);
          else chain_tile_bn<float, false>(m, it, q0, m.us32, nullptr, Y, m.perm, smf);
        } else {
          double* Y = static_cast<double*>(m.Y);
          if (xv) chain_tile_bn<double, true>(m, it, q0, m.us32, nullptr, Y, m.perm, smf);
          else chain_tile_bn<double, false>(m, it, q0, m.us32, nullptr, Y, m.perm, smf);
        }
        break;
    }
    __syncthreads();  // the tile's outputs are written and its shared memory is free again
    if (threadIdx.x == 0) chain_done(m.sync, it);
  }
}

}  // namespace

namespace {

std::mutex g_chain_mu;
int g_chain_occ[3][64] = {};  // resident chain CTAs per SM, per kernel (kXV) and device (0: not prepared)
int g_chain_sms[64] = {};

template <int kXV>
cudaError_t chain_occ(int dev) {
  cudaError_t e = cudaFuncSetAttribute(k_chain<kXV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kChainSmem);
  int o = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_chain<kXV>, kChainThreads, kChainSmem);
  if (e == cudaSuccess) g_chain_occ[kXV][dev] = o > 0 ? o : 1;
  return e;
}

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
    if (e == cudaSuccess) e = chain_occ<0>(dev);
    if (e == cudaSuccess) e = chain_occ<1>(dev);
    if (e == cudaSuccess) e = chain_occ<2>(dev);
    if (e != cudaSuccess) return e;
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
  const ChainMulti<ChainMember> none{nullptr, nullptr, 0, 0, 0, nullptr};
  if (m.xv)
    k_chain<1><<<(unsigned)grid, kChainThreads, kChainSmem, stream>>>(m, l, none);
  else
    k_chain<0><<<(unsigned)grid, kChainThreads, kChainSmem, stream>>>(m, l, none);
  return cudaGetLastError();
}

cudaError_t launch_chain_multi(const ChainMulti<ChainMember>& mm, const ChainLaunch& l, int grid_cap,
                               cudaStream_t stream) {
  if (mm.total <= 0 || mm.n_members <= 0) return cudaSuccess;
  if (mm.total > INT32_MAX) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = chain_prepare(nullptr, nullptr)) != cudaSuccess) return e;
  int64_t grid;
  {
    std::lock_guard<std::mutex> lock(g_chain_mu);
    grid = (int64_t)g_chain_sms[dev] * g_chain_occ[2][dev];
  }
  if (grid_cap > 0) grid = std::min<int64_t>(grid, grid_cap);
  grid = std::min<int64_t>(grid, mm.total);
  const ChainMember none{};
  k_chain<2><<<(unsigned)grid, kChainThreads, kChainSmem, stream>>>(none, l, mm);
  return cudaGetLastError();
}

}  // namespace hmat
