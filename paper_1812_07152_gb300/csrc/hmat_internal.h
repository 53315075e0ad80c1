// Internal structures of libhmat: the packed device layout of one HMatrix and
// the per-phase work lists that the evaluation kernels walk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hmat.h"

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

// How the rows of a phase's X operand are found: directly, through the point
// permutation (W in the caller's order) or through the coupling row map (the
// skeleton rows of a target's far partners, concatenated).
enum XMap : int32_t { XMAP_NONE = 0, XMAP_PERM = 1, XMAP_FAR = 2 };

struct Phase {
  PhaseKind kind;
  int32_t level;
  MatrixKind x;
  MatrixKind y;
  XMap xmap;
  int64_t tile_begin;  // into the tile array (one array for all phases)
  int64_t n_tiles;
  int32_t max_m;       // largest task height of the launch
  int32_t tile_rows;   // rows per CTA tile of this launch (16, 32 or 64)
};

// Mixed-precision products on the tensor cores: the near field (targets = leaves,
// blocks D_ij) and the coupling reduction (targets = tree nodes, blocks B_ab). A
// target's blocks are cut into m-tiles of 128 rows and k-chunks of 64 columns; each
// (m-tile, k-chunk) is stored as an FP16 hi tile and an FP16 lo tile (hi = fp16(x),
// lo = fp16(x - hi), x = the value times 2^scale of its m-tile), 128 rows x 128
// bytes each in the canonical K-major 128-byte-swizzled layout of a tcgen05 operand,
// so one bulk copy lands a tile in shared memory ready for the MMA. The right-hand
// operand (W for the near field, the skeleton weights w for the coupling) is split
// the same way per evaluation, per (source k-chunk, column tile).
constexpr int kTcRows = 128;        // rows per m-tile (MMA M)
constexpr int kTcK = 64;            // FP16 values per k-chunk row (128 bytes)
constexpr int kTcTileBytes = kTcRows * kTcK * 2;   // one FP16 tile: 16 KB
// The mixed mode puts the coupling on the tensor cores when the stored coupling values
// fill at least this fraction of the padded 128 x 64 tiles they occupy.
constexpr double kTcCouplingFill = 0.25;

struct TcTile {
  int32_t node;  // target (leaf-local id for the near field, tree node for the coupling)
  int32_t mt;    // m-tile of the target
};

// One (entry, m-tile, k-chunk) tile pair to pack from the FP64 arena.
struct TcPackJob {
  int64_t dst;        // byte offset of the hi tile (the lo tile follows)
  int64_t src;        // FP64 arena offset of the block's (row 0, column 0)
  int32_t rows, cols; // block shape
  int32_t r0, k0;     // first row / column of the tile inside the block
  int32_t scale_idx;  // index of the m-tile's scale exponent
  int32_t ld;         // row stride of the block in the arena
};

// Device-side description of one tensor-core product family, passed by value to its
// kernels. Targets and sources share one index space ("nodes"): rows of node n are
// begin[n] .. begin[n] + size[n] - 1 of the output (as a target) and of the
// right-hand side (as a source).
struct TcLists {
  const uint8_t* tiles;        // packed hi/lo tiles
  const int64_t* a_off;        // per entry: byte offset of its (m-tile 0, chunk 0) pair
  const int64_t* ptr;          // per target: CSR into the entries
  const int32_t* idx;          // per entry: its source node
  const int32_t* kc;           // per node: k-chunks = ceil(size / 64)
  const int64_t* kcum;         // per node: k-chunks of the preceding nodes
  const int64_t* begin;        // per node: first row
  const int32_t* size;         // per node: rows
  const int32_t* mt_base;      // per node: index of its first m-tile scale
  const int32_t* scale;        // per m-tile: scale exponent of the blocks
  const TcTile* work;          // (target, m-tile) work items, longest lists first
  const int32_t* chunk_node;   // per global k-chunk: its node
  const int32_t* chunk_c;      // per global k-chunk: its chunk index within the node
};

// Host-side owner of one product family.
struct TcProduct {
  TcLists dev{};
  uint8_t* tiles = nullptr;
  int64_t tile_bytes = 0;
  void* meta = nullptr;        // one allocation for the TcLists arrays
  int64_t n_work = 0;          // (target, m-tile) work items
  int64_t n_chunks = 0;        // source k-chunks
};

// ---- the far chain of the mixed mode (hmat_chain.cu)
//
// The upward pass, the FP32 coupling reduction, the downward transfers and the
// downward leaf step run as persistent launches over one list of CTA tiles ("items")
// instead of one launch per phase and tree level (the role of coarsening,
// Algorithm 2: no SM idles at a level boundary while the thin top levels run). A CTA
// takes the next item with an atomic ticket, waits (bounded) until the items it
// depends on are complete, computes its tile and counts it complete. Tickets are
// taken in list order and every dependency points to an earlier item, so the item
// with the lowest unfinished ticket can always run: no deadlock at any grid size.
enum ChainKind : uint8_t {
  CK_UP = 0,    // w_a = P_a^T W_a (leaf) or P_a^T [w_l; w_r]: needs the children's CK_UP
  CK_CPL = 1,   // u_a = sum_b B_ab w_b: needs every CK_UP item of a's level
  CK_DN = 2,    // [u_l; u_r] += P_a u_a: needs CK_CPL of a and of its children, CK_DN of its parent
  CK_LEAF = 3   // Y_i += P_i u_i (FP64 Y through perm): needs CK_CPL of i, CK_DN of its parent
};
struct ChainItem {
  int32_t tile;    // into Handle::tiles
  int32_t node;    // the task's tree node (whose counter the item advances)
  uint8_t kind;    // ChainKind
  uint8_t cls;     // row tile: 0 -> 16 rows, 1 -> 32, 2 -> 64
  uint8_t level;   // tree level of node
  uint8_t xmap;    // 1: X rows through the coupling row map
};
// Which dependencies a launch waits for (the others are ordered by the stream).
constexpr uint32_t kWaitUp = 1, kWaitLevel = 2, kWaitCpl = 4, kWaitDn = 8;

// The dependency state of one evaluation's chain (per member of a launch).
struct ChainSync {
  const int32_t* expect;      // items per node of CK_UP, CK_CPL, CK_DN, then CK_UP items per level
  int32_t* ctr;               // completed items (x column tiles), same layout as expect
  int* status;                // the handle's status word
  int32_t n_nodes;
  int32_t first_leaf;
  int32_t n_ct;               // column tiles of each item
  int32_t pad;
};

// Everything an item needs of one evaluation of one HMatrix.
struct ChainMember {
  const GemmTile* tiles;
  const GemmTask* tasks;
  const GemmEntry* entries;   // FP32 entries (arena32 offsets)
  const float* arena;         // arena32
  const float* w32;           // W in tree order, FP32 (upward leaf input)
  float* ws32;                // skeleton weights w
  float* us32;                // skeleton potentials u
  void* Y;                    // caller's output (CK_LEAF adds into it through perm): FP64, or FP32 when y_f32
  const int64_t* perm;
  const int64_t* far_rows;
  const ChainItem* items;
  ChainSync sync;
  int64_t q;
  int32_t n_ct;               // column tiles of bn columns
  int32_t bn;                 // 32 or 64
  int32_t first_leaf;
  int32_t xv;                 // q % 4 == 0: X rows copied 16 bytes at a time
  int32_t y_f32;              // Y holds FP32 values
  int32_t n_items;            // size of items (every item index is checked against it)
  int32_t n_tiles;            // size of tiles
  int32_t pad;
};

// The FP64 far chain (hmat_chain64.cu): one launch over the upward pass, the coupling,
// the downward transfers and the downward leaf step of the FP64 mode, after the near
// field (which the stream orders before it). Items are 16-row tiles of the tasks.
struct ChainMember64 {
  const GemmTile* tiles;
  const GemmTask* tasks;
  const GemmEntry* entries;   // FP64 entries
  const double* arena;
  const double* W;            // caller's right-hand side (rows through perm)
  double* ws;
  double* us;
  double* Y;                  // caller's output (rows through perm)
  const int64_t* perm;
  const int64_t* far_rows;
  const ChainItem* items;
  ChainSync sync;
  int64_t q;
  int32_t n_ct;
  int32_t first_leaf;
  int32_t n_items;            // size of items (every item index is checked against it)
  int32_t n_tiles;            // size of tiles
};

// One persistent launch: tickets item_begin .. item_begin + n_items - 1 of member m,
// each times m.n_ct column tiles.
struct ChainLaunch {
  int32_t item_begin;
  int32_t n_items;
  int32_t* ticket;            // this launch's ticket counter (zeroed before the evaluation)
  int32_t* abort_flag;        // set by the first wait that gives up (zeroed likewise)
  uint32_t waits;             // kWait* mask
  int32_t extra;              // self-test: added to every requirement, so that every wait runs out
  uint64_t limit_ns;          // a wait gives up after this long and latches HMAT_ETIMEOUT
  int* status;                // status word for an inconsistent ticket list (no member to report to)
};

// Ranges of a handle's chain items per launch: A (upward pass; with the FP32 coupling
// also the coupling and the downward transfers), B (downward transfers after the
// tensor-core coupling), C (downward leaf step).
struct ChainPlan {
  std::vector<ChainItem> host;    // the items (host copy, for the batches' ticket lists)
  ChainItem* items = nullptr;     // device
  int32_t* expect = nullptr;      // device, 3 * n_nodes + levels + 1
  int32_t begin[3] = {0, 0, 0};
  int32_t count[3] = {0, 0, 0};
  uint32_t waits[3] = {0, 0, 0};
  int64_t n_ctr = 0;              // counters: 4 (tickets A, B, C, abort) + the expect layout
};
constexpr int kChainCtrHead = 4;

// Many members in one launch (batches): member k's tickets are parts[k-1].ticket_end ..
// parts[k].ticket_end - 1 of the launch (items item_begin .. item_begin + n_items - 1 of
// members[k], each times its column tiles), waiting as `waits` says. One ticket counter
// and one abort flag for the launch (ChainLaunch); members keep their own counters.
struct ChainPart {
  int64_t ticket_end;
  int32_t item_begin;
  int32_t n_items;
  uint32_t waits;
  int32_t pad;
};
// A ticket of a multi-member launch whose tickets follow an explicit order (list != null):
// member index, item index in that member's item array, column tile, the waits.
struct ChainTicket {
  int32_t member;
  int32_t item;
  int32_t ct;
  uint32_t waits;
};
template <typename M>
struct ChainMulti {
  const M* members;           // device; null: the launch has one member, the kernel parameter
  const ChainPart* parts;     // device; per-member ticket ranges (when list is null)
  int32_t n_members;
  int32_t free_run;           // no member waits: a plain grid over the tickets
  int64_t total;              // tickets of the launch
  const ChainTicket* list;    // device, or null: the tickets in this order, one entry each
};
// A batch orders the tickets of its chain launches across members by stage (an item's
// stage is below that of every item it waits for, so the order stays deadlock-free):
// every member's leaf items, then every member's next level, and so on.
int chain_stage(const ChainItem& it, int levels, int max_levels);

cudaError_t launch_chain(const ChainMember& m, const ChainLaunch& l, int grid_cap, cudaStream_t stream);
cudaError_t launch_chain_multi(const ChainMulti<ChainMember>& mm, const ChainLaunch& l, int grid_cap,
                               cudaStream_t stream);
// FP64 chain with column tiles of kColBN[shape] columns; chain64_prepare caches the
// kernels' occupancy on the current device (at load, outside any graph capture).
cudaError_t launch_chain64(const ChainMember64& m, const ChainLaunch& l, int shape, int grid_cap, cudaStream_t stream);
cudaError_t launch_chain64_multi(const ChainMulti<ChainMember64>& mm, const ChainLaunch& l, int shape, int grid_cap,
                                 cudaStream_t stream);
cudaError_t chain64_prepare();
// Sets the chain kernels' attributes on the current device (once) and returns the CTAs
// that fit on it at once (16-byte X copies, 4-byte X copies; either may be null);
// called at load, so that no launch (or graph capture) does it.
cudaError_t chain_prepare(int* grid_v, int* grid_s);
constexpr uint64_t kChainWaitNs = 2000000000ull;  // a chain wait gives up after 2 s
// columns per chain tile for q
inline int chain_bn(int64_t q) { return q <= 32 ? 32 : 64; }

// The state one evaluation needs besides the read-only HMatrix: the workspaces
// (carved from one device block for a given q and mode) and, for the mixed mode, a
// side stream with its fork/join events. A handle owns a default context; a batch
// or a server owns one per evaluation it keeps in flight.
struct EvalContext {
  uint8_t* block = nullptr;      // own workspace block (cudaMalloc); nullptr when bound to external memory
  int64_t block_bytes = 0;
  double* ws = nullptr;          // FP64: skeleton weights w and potentials u (sum of ranks x q)
  double* us = nullptr;
  unsigned long long* wmax = nullptr;  // mixed: max |W| (FP64 bits)
  uint8_t* wsplit = nullptr;     // mixed: W as FP16 hi/lo operand tiles
  unsigned long long* smax = nullptr;  // mixed: max |w| of the skeleton weights (FP64 bits)
  uint8_t* ssplit = nullptr;     // mixed: skeleton weights as FP16 hi/lo operand tiles
  float* w32 = nullptr;          // mixed: FP32 copy of W in tree order
  float* ws32 = nullptr;         // mixed: FP32 skeleton workspaces
  float* us32 = nullptr;
  int32_t* chain_ctr = nullptr;  // tickets and completion counters of the far chain (either mode)
  double* w64 = nullptr;         // FP64 mode with FP32 W and Y: W widened, Y before rounding (n x q each)
  double* y64 = nullptr;
  void* host_w = nullptr;        // device copies of W / Y for hmat_eval_host
  void* host_y = nullptr;
  int64_t host_cap = 0;          // bytes of each
  cudaStream_t copy = nullptr;   // hmat_eval_host: host <-> device copies beside the evaluation
  cudaEvent_t ev_copy[5] = {};
  cudaStream_t aux = nullptr;    // mixed: the far chain runs here, beside the near field
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// Tile shapes chosen by hmat_autotune for one (q, mode) of a handle. Every choice
// gives bitwise the same result as the default; only the time differs.
struct TuneEntry {
  int64_t q = 0;
  int mode = 0;
  std::vector<int8_t> shape;   // FP64: column shape (index into kColBN) per entry of Handle::phases
  int n_t = 0;                 // mixed: columns per tensor-core CTA
  int chain_grid = 0;          // CTAs of the persistent far chain (0: every resident CTA)
  int chain_shape = -1;        // FP64: column shape of the far chain (index into kColBN; -1: default)
  double default_ms = 0, tuned_ms = 0;
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
  int64_t n_tiles = 0;            // entries of the tile array (both modes' launches and chains)

  std::vector<int64_t> begin, size, skel_off, perm_host, near_ptr, far_ptr;
  std::vector<int32_t> rank, near_idx, far_idx;
  std::vector<Phase> phases;      // FP64 mode: one launch per row-tile size of every phase
  std::vector<Phase> phases32;    // mixed mode: the upward and downward passes in FP32

  // device
  double* arena = nullptr;       // packed FP64 blocks (near, basis, coupling)
  int64_t arena_values = 0;
  int64_t* perm = nullptr;       // tree order -> caller order
  int64_t* far_rows = nullptr;   // coupling row map: per target, its far partners' skeleton rows
  GemmTask* tasks = nullptr;
  GemmEntry* entries = nullptr;
  GemmTile* tiles = nullptr;
  int* status = nullptr;         // device status word (hmat_status of the first error)

  // mixed precision (HMAT_LOAD_MIXED); without the FP64 blocks (HMAT_LOAD_MIXED_ONLY)
  bool has_mixed = false;
  bool has_fp64 = true;
  TcProduct tc_near;             // near field D_ij on the tensor cores
  TcProduct tc_far;              // coupling B_ab on the tensor cores (when tc_coupling)
  bool tc_coupling = false;      // mixed coupling engine: tensor cores, else FP32 CUDA cores
  float* arena32 = nullptr;      // FP32 operands of the upward and downward passes (and of
                                 // the coupling when it runs in FP32), one block per entry,
                                 // k-major: A(m, k) at [a_off + k * lda + m], lda a multiple
                                 // of 4 (rows m..lda-1 zero), a_off a multiple of 4
  GemmEntry* entries32 = nullptr;  // the entries with a_off/lda into arena32 (trans = 1)
  ChainPlan chain;                 // the far field of the mixed mode as persistent launches
  ChainPlan chain64;               // the far field of the FP64 mode as one persistent launch (range A)

  // near blocks evaluated on the fly (HMAT_BUILD_NEAR_OTF): the arena holds no near
  // blocks; the near phase computes K(x_i, x_j) from the tree-ordered points
  bool near_otf = false;
  double* pts_tree = nullptr;  // device, n_points x dim, tree order
  int32_t dim = 0;
  int32_t kernel = 0;
  double kernel_param = 0.0;

  double* noalloc_scratch = nullptr;  // device address of hmat_eval_noalloc's static array
  struct EvalContext* ctx = nullptr;  // the handle's own evaluation state (hmat_eval)
  std::vector<TuneEntry> tuned;       // hmat_autotune results, one per (q, mode)

  // per-launch event timing (hmat_profile / hmat_phase_times)
  struct ProfRecord {
    int32_t kind;
    cudaEvent_t start, stop;
  };
  int profiling = 0;               // 1: events around every launch; 2: the same, far chain serialised
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
  int64_t ld;        // row stride of the block in the arena
  int64_t row_off;
  int64_t col_off;
  int32_t rows;
  int32_t cols;
  int32_t row_skel;
  int32_t col_skel;
};

// One node's row ID on the device (hmat_id.cu): rows and columns are point indices
// (tree order) at ids[rows_off ..] and ids[cols_off ..]; A (n_cols x n_rows,
// column-major) at work[a_off ..]; pivots at piv[piv_off ..].
struct IdJob {
  int64_t a_off;
  int64_t rows_off;
  int64_t cols_off;
  int64_t piv_off;
  int32_t n_rows;
  int32_t n_cols;
};
cudaError_t launch_row_id(const IdJob* jobs, int64_t n_jobs, int64_t max_rows, const double* pts, int d,
                          const int64_t* ids, int kernel, double param, double tol, int max_rank, double* work,
                          int32_t* piv, int32_t* rank, cudaStream_t stream);

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
hmat_status load_impl(const hmat_desc* d, const DeviceBlockSource* src, int flags, hmat_handle** out);

cudaError_t launch_eval_blocks(const BlockJob* jobs, int64_t n_jobs, const double* pts, int dim,
                               const int64_t* skel_pts, int kernel, double param, double* arena,
                               cudaStream_t stream);

// Mixed mode: load-time packing and per-evaluation kernels (hmat_mixed.cu).
cudaError_t launch_tc_scale(const TcLists& tc, const int64_t* blk_off, const int32_t* blk_ld, const double* arena,
                            int64_t n_mtiles, const int32_t* mtile_node, const int32_t* mtile_mt, int32_t* scale_out,
                            cudaStream_t stream);
cudaError_t launch_tc_pack(const TcPackJob* jobs, int64_t n_jobs, const double* arena, const int32_t* scale,
                           uint8_t* tiles, cudaStream_t stream);
// One block of the FP64 arena copied to FP32 in the k-major padded layout of arena32:
// dst[dst_off + k * ld + m] = A(m, k) for m < m_rows, 0 for m_rows <= m < ld, where
// A(m, k) = src[src_off + k * lda + m] (trans) or src[src_off + m * lda + k].
struct F32Job {
  int64_t src_off;
  int64_t dst_off;
  int32_t m_rows;
  int32_t k;
  int32_t lda;
  int32_t ld;
  int32_t trans;
  int32_t pad;
};
cudaError_t launch_relayout_f32(const double* arena, const F32Job* jobs, int64_t n_jobs, float* dst,
                                cudaStream_t stream);
// Right-hand operand split: X (n_values values, row-major with q columns; FP64 rows
// through perm for the near field, FP32 rows in node order for the coupling) ->
// hi/lo tiles per (source k-chunk, column tile); x32 (may be null) gets the FP32
// tree-order copy of an FP64 X.
cudaError_t launch_split_f64(const TcProduct& p, const double* X, int64_t n_values, const int64_t* perm, int64_t q,
                             int n_t, int n_ct, unsigned long long* xmax, uint8_t* out, float* x32,
                             cudaStream_t stream);
cudaError_t launch_split_f32(const TcProduct& p, const float* X, int64_t n_values, const int64_t* perm, int64_t q,
                             int n_t, int n_ct, unsigned long long* xmax, uint8_t* out, float* x32,
                             cudaStream_t stream);
// The arguments of one tensor-core product (near field or coupling) of one evaluation.
struct TcArgs {
  TcLists tc;
  const uint8_t* bsplit;            // right-hand operand tiles (k_split)
  const unsigned long long* bmax;   // max |X| of the right-hand side (FP64 bits)
  const int64_t* perm;              // near field: tree order -> caller order of Y's rows
  void* Y;                          // near field: double or float (caller order); coupling: float (node rows)
  int64_t q;
  int n_t;
  int n_ct;
  int* status;
  int y_f32;                        // near field: Y holds FP32 values
};
// One right-hand-side split of one evaluation (multi-member launches carry one per member).
struct SplitJob {
  TcLists tc;
  const void* X;                    // FP64 or FP32 by the launch
  const int64_t* perm;              // rows of X through perm (the near field's W), or null
  int64_t q;
  int n_t;
  int n_ct;
  const unsigned long long* xmax;
  uint8_t* out;
  float* x32;                       // FP32 tree-order copy of X, or null
};
// max |X| over n values of one member.
struct AbsJob {
  const void* X;
  int64_t n;
  unsigned long long* out;
};
// Blocks of one max |X| pass over n values.
inline int64_t absmax_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b);
}
// Multi-member launches (batches); the tables and block prefixes are device arrays.
cudaError_t launch_absmax_multi(bool f32, const AbsJob* jobs, const int64_t* block_end, int n, int64_t blocks,
                                cudaStream_t stream);
cudaError_t launch_split_multi(bool f32, const SplitJob* jobs, const int64_t* block_end, int n, int64_t blocks,
                               cudaStream_t stream);
cudaError_t launch_tc_multi(bool far, const TcArgs* args, const int64_t* block_end, int n, int64_t blocks,
                            cudaStream_t stream);

// Y (FP64, or FP32 when y_f32; rows through perm) = near field; or U (FP32, node rows) = coupling.
cudaError_t launch_tc_near(const TcProduct& p, const uint8_t* bsplit, const unsigned long long* bmax,
                           const int64_t* perm, void* Y, bool y_f32, int64_t q, int n_t, int n_ct, int* status,
                           cudaStream_t stream);
cudaError_t launch_tc_far(const TcProduct& p, const uint8_t* bsplit, const unsigned long long* bmax, float* U,
                          int64_t q, int n_t, int n_ct, int* status, cudaStream_t stream);
// One bounded wait that nothing completes: sets HMAT_ETIMEOUT in *status after limit_ns.
cudaError_t launch_wait_selftest(int* status, uint64_t limit_ns, cudaStream_t stream);

// Device address of hmat_eval_noalloc's static workspace array on the current device
// (hmat_noalloc.cu); looked up by every load, never by the evaluation itself.
cudaError_t noalloc_scratch_address(double** out);

// Evaluation contexts (hmat_eval.cpp). dtype: HMAT_DTYPE_F64 or HMAT_DTYPE_F32 (W and Y).
hmat_status ctx_create(const Handle& h, EvalContext** out);
void ctx_destroy(EvalContext* c);
int64_t ctx_bytes(const Handle& h, int64_t q, int mode, int dtype = HMAT_DTYPE_F64);  // workspace bytes
void ctx_bind(const Handle& h, EvalContext* c, int64_t q, int mode, uint8_t* base,
              int dtype = HMAT_DTYPE_F64);                                             // carve the workspaces
hmat_status ctx_reserve(const Handle& h, EvalContext* c, int64_t q, int mode,
                        int dtype = HMAT_DTYPE_F64);                                   // grow the own block
// Enqueue Y = K~ W on `s` with the workspaces of `c` (bound for q, mode and dtype by the caller).
hmat_status eval_impl(Handle* h, EvalContext* c, const void* W, void* Y, int64_t q, int mode, int dtype,
                      cudaStream_t s);
inline int64_t dtype_bytes(int dtype) { return dtype == HMAT_DTYPE_F32 ? 4 : 8; }
// FP32 <-> FP64 copies of n values (hmat_mixed.cu): widening exact, narrowing to nearest even.
cudaError_t launch_widen(const float* src, double* dst, int64_t n, cudaStream_t stream);
cudaError_t launch_narrow(const double* src, float* dst, int64_t n, cudaStream_t stream);
// The far chain of one mixed evaluation with the workspaces of c (bound for q): the
// member description, launch `part` (0, 1, 2 = ChainPlan ranges A, B, C) and the grid cap
// chosen by the autotuner.
ChainMember chain_member(const Handle& h, const EvalContext* c, void* Y, bool y_f32, int64_t q);
ChainLaunch chain_launch(const Handle& h, const EvalContext* c, int part, int32_t extra, uint64_t limit_ns);
// The same for the FP64 mode's single far-chain launch (the column shape from the tuned entry).
ChainMember64 chain_member64(const Handle& h, const EvalContext* c, const double* W, double* Y, int64_t q);
ChainLaunch chain_launch64(const Handle& h, const EvalContext* c, int32_t extra, uint64_t limit_ns);
int chain_grid_cap(const Handle& h, int64_t q);
hmat_status cuda_status(cudaError_t e);

// Launch the FP64 grouped GEMM of one phase on `stream`: column shape `shape` (-1:
// the default for q), the first `n_tiles` tiles of the phase (-1: all).
cudaError_t launch_fp64_phase(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map,
                              double* Y, const int64_t* y_map, int64_t q, int shape, int64_t n_tiles,
                              cudaStream_t stream);
// the near phase of a handle built with HMAT_BUILD_NEAR_OTF (hmat_fp64_otf.cu)
cudaError_t launch_fp64_near_otf(const Handle& h, const Phase& ph, const double* X, const int64_t* x_map, double* Y,
                                 const int64_t* y_map, int64_t q, int shape, int64_t n_tiles, cudaStream_t stream);
int fp64_default_shape(int64_t q);
int fp64_shape_columns(int shape);

// Tensor-core column tiling of the mixed mode (hmat_eval.cpp): the candidate widths
// for q (multiples of 16, at most 128; the first is the default), the widest
// workspace any of them needs (columns = n_ct * n_t), and the width an evaluation
// uses (the tuned one when there is one).
std::vector<int> mixed_nt_candidates(int64_t q);
int64_t mixed_cols_bound(int64_t q);
void mixed_tiles(const Handle& h, int64_t q, int* n_t, int64_t* n_ct);
const TuneEntry* find_tuned(const Handle& h, int64_t q, int mode);

}  // namespace hmat

namespace hmat {
inline const int64_t* phase_x_map(const Handle& h, const Phase& ph) {
  return ph.xmap == XMAP_PERM ? h.perm : (ph.xmap == XMAP_FAR ? h.far_rows : nullptr);
}
}  // namespace hmat

// The opaque handle of the C ABI is the internal Handle.
struct hmat_handle : public hmat::Handle {};
