// The far field of the FP64 mode as one persistent launch (Section 2.1's upward pass,
// far-field reduction and downward pass; coarsening, Algorithm 2, on the GPU).
//
// The items are 16-row tiles of the far-field tasks (each column tile of a tile is a
// ticket), so a thin top level is spread over as many CTAs as it has 16-row slices:
// an FP64 tile runs at the SM's FP64 rate (about two DFMA per clock), and a 64-row tile
// of a top-level transfer alone takes tens of microseconds on one SM. The waits, the
// ordering that makes them deadlock-free and the completion counts are those of the
// mixed mode's chain (hmat_chain.cuh); the downward leaf items also wait, since this is
// the only far-field launch of the mode (the near field before it is ordered by the
// stream).
#include <algorithm>
#include <mutex>

#include "hmat_chain.cuh"
#include "hmat_gemm.cuh"

namespace hmat {
namespace {

template <int BN, int CTM, int CTN>
using Cfg64 = gemm::Cfg<16, BN, CTM, CTN>;

template <int BN, int CTM, int CTN>
__global__ void __launch_bounds__(Cfg64<BN, CTM, CTN>::kThreads)
k_chain64(const __grid_constant__ ChainMember64 m1, const __grid_constant__ ChainLaunch l,
          const __grid_constant__ ChainMulti<ChainMember64> mm) {
  __shared__ ChainMember64 sm;  // the member of the current item
  __shared__ ChainItem s_it;
  __shared__ int64_t s_q0;
  __shared__ int s_go;
  const bool multi = mm.members != nullptr;
  const int64_t total = multi ? mm.total : (int64_t)l.n_items * m1.n_ct;
  const gemm::OtfArgs no_otf{nullptr, 0, KernelSpec{}};
  int cur = -1;  // thread 0: member held in sm
  for (;;) {
    if (threadIdx.x == 0) {
      int go = 0;
      int64_t t = 0;
      if (!*(volatile int32_t*)l.abort_flag) {
        t = atomicAdd(l.ticket, 1);
        go = t < total;
      }
      if (go) {
        int mi = 0;
        int64_t local = t;
        uint32_t waits = l.waits;
        int32_t ib = l.item_begin;
        int32_t item = -1, ct = 0;
        if (multi && mm.list) {
          const ChainTicket ck = mm.list[t];
          mi = ck.member;
          waits = ck.waits;
          item = ck.item;
          ct = ck.ct;
        } else if (multi) {
          int lo = 0, hi = mm.n_members - 1;
          while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (mm.parts[mid].ticket_end > t) hi = mid;
            else lo = mid + 1;
          }
          mi = lo;
          local = t - (mi > 0 ? mm.parts[mi - 1].ticket_end : 0);
          waits = mm.parts[mi].waits;
          ib = mm.parts[mi].item_begin;
        }
        if (multi && (mi < 0 || mi >= mm.n_members)) {  // an inconsistent ticket list
          atomicCAS(l.status, 0, (int)HMAT_EDEVICE);
          atomicExch(l.abort_flag, 1);
          go = 0;
        }
        if (go && multi && mi != cur) {  // one 32-bit word at a time: few registers live in the copy
          const uint32_t* src = reinterpret_cast<const uint32_t*>(mm.members + mi);
          uint32_t* dst = reinterpret_cast<uint32_t*>(&sm);
          for (int w = 0; w < (int)(sizeof(ChainMember64) / 4); ++w) dst[w] = src[w];
          cur = mi;
        }
        if (go) {
          const ChainMember64& mt = multi ? sm : m1;
          int64_t ii;
          if (item >= 0) {
            ii = item;
            s_q0 = (int64_t)ct * BN;
          } else {
            ii = ib + local / mt.n_ct;
            s_q0 = (local % mt.n_ct) * BN;
          }
          // every index taken from device data is checked before it is used
          go = chain_item_ok(mt.items, ii, mt.n_items, mt.n_tiles, mt.sync.n_nodes, &s_it) ? 1 : 0;
          if (!go) {
            atomicCAS(mt.sync.status, 0, (int)HMAT_EDEVICE);
            atomicExch(l.abort_flag, 1);
          } else {
            ChainLaunch lw = l;
            lw.waits = waits;
            go = chain_deps(mt.sync, s_it, lw) ? 1 : 0;
          }
        }
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const ChainItem it = s_it;
    const int64_t q0 = s_q0;
    const ChainMember64& m = multi ? sm : m1;
    const GemmTile tile = m.tiles[it.tile];
    const double* X;
    const int64_t* x_map = nullptr;
    double* Y;
    const int64_t* y_map = nullptr;
    switch (it.kind) {
      case CK_UP:  // leaves read W in the caller's order, inner nodes their children's w
        if (it.node >= m.first_leaf) {
          X = m.W;
          x_map = m.perm;
        } else {
          X = m.ws;
        }
        Y = m.ws;
        break;
      case CK_CPL:
        X = m.ws;
        x_map = m.far_rows;
        Y = m.us;
        break;
      case CK_DN:
        X = m.us;
        Y = m.us;
        break;
      default:
        X = m.us;
        Y = m.Y;
        y_map = m.perm;
        break;
    }
    gemm::gemm_tile<double, double, double, double, 16, BN, CTM, CTN, false>(
        tile, m.tasks, m.entries, m.arena, 0, X, x_map, Y, y_map, m.q, q0, no_otf);
    __syncthreads();  // the tile's outputs are written and its shared memory is free again
    if (threadIdx.x == 0) chain_done(m.sync, it);
  }
}

std::mutex g_mu;
int g_grid[64][gemm::kColShapes] = {};  // default grid, per device and shape
int g_full[64][gemm::kColShapes] = {};  // resident CTAs on the whole device (the largest useful grid)

template <int BN, int CTM, int CTN>
cudaError_t prepare_shape(int dev, int shape) {
  constexpr int NT = Cfg64<BN, CTM, CTN>::kThreads;
  if (g_grid[dev][shape] != 0) return cudaSuccess;
  int occ = 0, sms = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chain64<BN, CTM, CTN>, NT, 0);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // about eight warps per SM: the FP64 pipe (two DFMA per clock per SM) is kept busy by a
  // few warps, and CTAs beyond what a level can use would only wait
  g_grid[dev][shape] = std::max(1, std::min(occ, 256 / NT)) * sms;
  g_full[dev][shape] = std::max(occ, 1) * sms;
  return cudaSuccess;
}

cudaError_t prepare_all(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  cudaError_t e = prepare_shape<1, 1, 1>(dev, 0);
  if (e == cudaSuccess) e = prepare_shape<2, 1, 1>(dev, 1);
  if (e == cudaSuccess) e = prepare_shape<4, 2, 1>(dev, 2);
  if (e == cudaSuccess) e = prepare_shape<8, 2, 2>(dev, 3);
  if (e == cudaSuccess) e = prepare_shape<16, 4, 4>(dev, 4);
  if (e == cudaSuccess) e = prepare_shape<32, 4, 4>(dev, 5);
  if (e == cudaSuccess) e = prepare_shape<64, 4, 4>(dev, 6);
  return e;
}

template <int BN, int CTM, int CTN>
cudaError_t launch_shape(const ChainMember64& m, const ChainLaunch& l, const ChainMulti<ChainMember64>& mm, int shape,
                         int grid_cap, cudaStream_t s) {
  constexpr int NT = Cfg64<BN, CTM, CTN>::kThreads;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int def, full;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    def = g_grid[dev][shape];
    full = g_full[dev][shape];
  }
  if (def == 0) {  // prepared at load; only a device that loaded nothing gets here
    if ((e = prepare_all(dev)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    def = g_grid[dev][shape];
    full = g_full[dev][shape];
  }
  int64_t grid = grid_cap > 0 ? std::min<int64_t>(full, grid_cap) : def;
  grid = std::min<int64_t>(grid, mm.members ? mm.total : (int64_t)l.n_items * m.n_ct);
  k_chain64<BN, CTM, CTN><<<(unsigned)grid, NT, 0, s>>>(m, l, mm);
  return cudaGetLastError();
}

}  // namespace

cudaError_t chain64_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  return prepare_all(dev);
}

namespace {

cudaError_t launch_any(const ChainMember64& m, const ChainLaunch& l, const ChainMulti<ChainMember64>& mm, int shape,
                       int grid_cap, cudaStream_t stream) {
  // the per-thread register tiles of hmat_gemm.cuh's column shapes
  switch (shape) {
    case 0: return launch_shape<1, 1, 1>(m, l, mm, shape, grid_cap, stream);
    case 1: return launch_shape<2, 1, 1>(m, l, mm, shape, grid_cap, stream);
    case 2: return launch_shape<4, 2, 1>(m, l, mm, shape, grid_cap, stream);
    case 3: return launch_shape<8, 2, 2>(m, l, mm, shape, grid_cap, stream);
    case 4: return launch_shape<16, 4, 4>(m, l, mm, shape, grid_cap, stream);
    case 5: return launch_shape<32, 4, 4>(m, l, mm, shape, grid_cap, stream);
    case 6: return launch_shape<64, 4, 4>(m, l, mm, shape, grid_cap, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_chain64(const ChainMember64& m, const ChainLaunch& l, int shape, int grid_cap,
                           cudaStream_t stream) {
  if (l.n_items <= 0 || m.q <= 0) return cudaSuccess;
  if ((int64_t)l.n_items * m.n_ct > INT32_MAX) return cudaErrorInvalidValue;
  return launch_any(m, l, ChainMulti<ChainMember64>{nullptr, nullptr, 0, 0, 0, nullptr}, shape, grid_cap, stream);
}

cudaError_t launch_chain64_multi(const ChainMulti<ChainMember64>& mm, const ChainLaunch& l, int shape, int grid_cap,
                                 cudaStream_t stream) {
  if (mm.total <= 0 || mm.n_members <= 0) return cudaSuccess;
  if (mm.total > INT32_MAX) return cudaErrorInvalidValue;
  return launch_any(ChainMember64{}, l, mm, shape, grid_cap, stream);
}

}  // namespace hmat
