// Internal structures of libhmat: the packed device layout of one HMatrix and
// the per-phase work lists that the evaluation kernels walk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hmat.h"

namespace hmat {

// One output block of a grouped GEMM: rows [out_row, out_row + m) of the output
// matrix receive sum over entries e of op(A_e) * X[x_row_e : x_row_e + k_e, :].
struct GemmTask {
  int64_t out_row;
  int32_t m;
  int32_t e_begin;
  int32_t e_end;
  int32_t accumulate;  // 0: overwrite the output rows, 1: add to them
};

// One term of a task. A is stored row-major in the arena at a_off with row stride
// lda: trans = 0 -> stored m x k (A itself); trans = 1 -> stored k x m (A = S^T).
struct GemmEntry {
  int64_t a_off;
  int64_t x_row;
  int32_t k;
  int32_t lda;
  int32_t trans;
  int32_t pad;
};

// A CTA's share of a task: output rows [m0, m0 + tile_rows) of task `task`.
struct GemmTile {
  int32_t task;
  int32_t m0;
};

// Which matrix a phase reads (X) and writes (Y).
enum MatrixKind : int32_t { MAT_USER = 0, MAT_SKEL_W = 1, MAT_SKEL_U = 2 };

// The steps of the evaluation, in execution order.
enum PhaseKind : int32_t {
  PH_NEAR = 0,       // Y_i = sum_j D_ij W_j                    (near-field reduction)
  PH_UP_LEAF = 1,    // w_i = P_i^T W_i                          (upward pass, leaves)
  PH_UP_TRANS = 2,   // w_a = P_a^T [w_l; w_r]                   (upward pass, one level)
  PH_COUPLING = 3,   // u_a = sum_b B_ab w_b                     (far-field reduction)
  PH_DOWN_TRANS = 4, // [u_l; u_r] += P_a u_a                    (downward pass, one level)
  PH_DOWN_LEAF = 5   // Y_i += P_i u_i                           (downward pass, leaves)
};

struct Phase {
  PhaseKind kind;
  int32_t level;
  MatrixKind x;
  MatrixKind y;
  int64_t tile_begin;  // into the tile array (one array for all phases)
  int64_t n_tiles;
  int32_t max_m;       // largest task height of the launch
  int32_t tile_rows;   // rows per CTA tile of this launch (16, 32 or 64)
};

struct Handle {
  int device = -1;
  int64_t n_points = 0;
  int32_t levels = 0;
  int64_t n_nodes = 0;
  int64_t n_leaves = 0;
  int64_t n_near = 0;
  int64_t n_far = 0;
  int64_t near_values = 0, basis_values = 0, coupling_values = 0;
  int64_t sum_rank = 0;

  std::vector<int64_t> begin, size, skel_off, perm_host, near_ptr, far_ptr;
  std::vector<int32_t> rank, near_idx, far_idx;
  std::vector<Phase> phases;

  // device
  double* arena = nullptr;       // packed FP64 blocks (near, basis, coupling)
  int64_t arena_values = 0;
  int64_t* perm = nullptr;       // tree order -> caller order
  GemmTask* tasks = nullptr;
  GemmEntry* entries = nullptr;
  GemmTile* tiles = nullptr;
  int* status = nullptr;         // device status word (hmat_status of the first error)
  double* ws = nullptr;          // skeleton weights w (sum_rank x q_cap)
  double* us = nullptr;          // skeleton potentials u (sum_rank x q_cap)
  int64_t q_cap = 0;
  int64_t ws_bytes = 0;
  double* host_w = nullptr;      // device copies of W / Y for hmat_eval_host
  double* host_y = nullptr;
  int64_t host_cap = 0;          // capacity of host_w / host_y in values

  // per-launch event timing (hmat_profile / hmat_phase_times)
  struct ProfRecord {
    int32_t kind;
    cudaEvent_t start, stop;
  };
  bool profiling = false;
  std::vector<ProfRecord> prof;
  std::vector<cudaEvent_t> event_pool;
  int64_t device_bytes = 0;
};

// A dense kernel block evaluated on the device: arena[a_off + r * cols + c] =
// k(x[row point r], x[col point c]); a point index list is either the range
// row_off .. row_off + rows - 1 of tree-order points (skel = 0) or the entries
// row_off .. of the skeleton point list (skel = 1).
struct BlockJob {
  int64_t a_off;
  int64_t row_off;
  int64_t col_off;
  int32_t rows;
  int32_t cols;
  int32_t row_skel;
  int32_t col_skel;
};

// Source of the near and coupling blocks when they are evaluated on the device.
struct DeviceBlockSource {
  const double* points_tree;   // host, n_points x dim, tree order
  int32_t dim;
  const int64_t* skel_points;  // host, sum of ranks entries in node order (tree-order point ids)
  int32_t kernel;
  double kernel_param;
};

// Shared body of hmat_load (src == nullptr: every block from the host arrays of d)
// and hmat_build (src != nullptr: d->near and d->coupling are ignored and the
// blocks are evaluated on the device from the points).
hmat_status load_impl(const hmat_desc* d, const DeviceBlockSource* src, hmat_handle** out);

cudaError_t launch_eval_blocks(const BlockJob* jobs, int64_t n_jobs, const double* pts, int dim,
                               const int64_t* skel_pts, int kernel, double param, double* arena,
                               cudaStream_t stream);

// Launch the FP64 grouped GEMM of one phase on `stream`.
cudaError_t launch_fp64_phase(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map,
                              double* Y, const int64_t* y_map, int64_t q, cudaStream_t stream);

}  // namespace hmat

// The opaque handle of the C ABI is the internal Handle.
struct hmat_handle : public hmat::Handle {};
