/*
 * hmat.h - C ABI of the GB300 HMatrix-matrix evaluation library (libhmat.so).
 *
 * The library evaluates Y = K~ W, the product of a compressed kernel matrix
 * (an HMatrix: H2 or HSS, nested bases) with a dense N x Q block W, on one
 * GPU. This is the evaluation phase of MatRox (arXiv 1812.07152, Section 2.1,
 * "Evaluation"): a near-field reduction over the dense blocks D, a bottom-up
 * pass over the cluster tree applying the bases V^T, a far-field reduction
 * over the coupling blocks B and a top-down pass applying the bases U (U = V
 * because the kernel matrix is symmetric, Section 1).
 *
 * Conventions shared by every entry point
 *  - Every call returns an hmat_status; no C++ exception crosses the ABI.
 *  - Host pointers are read during the call only and may be freed afterwards.
 *  - Device pointers (W, Y) are CUDA global memory on the device that was
 *    current when the handle was created; that device must be current again.
 *  - All matrices are row-major and contiguous.
 *  - Asynchronous errors found by a kernel (a wait that ran out, an index out
 *    of range) are latched in a device status word read by hmat_status_poll.
 */
#ifndef HMAT_H_
#define HMAT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hmat_handle* hmat_t;

typedef enum {
  HMAT_OK = 0,
  HMAT_EINVAL = -1,          /* an argument or the HMatrix description is invalid */
  HMAT_ENOMEM = -2,          /* host or device allocation failed */
  HMAT_ECUDA = -3,           /* a CUDA runtime call failed */
  HMAT_ETIMEOUT = -4,        /* a bounded device-side wait gave up */
  HMAT_EUNSUPPORTED = -5,    /* valid request that this build does not support */
  HMAT_EDEVICE = -6,         /* a kernel detected an inconsistent index or size */
  HMAT_EBUSY = -7            /* the server's queue is full: the request was not accepted */
} hmat_status;

/*
 * hmat_desc - one compressed kernel matrix (Section 3.1: the CTree, the HTree
 * near/far lists, the sranks and the submatrices D, V = U and B), FP64.
 *
 * Tree: a perfect binary cluster tree of depth `levels` in heap numbering:
 * node a has children 2a+1 and 2a+2, level l holds nodes 2^l - 1 .. 2^(l+1) - 2,
 * n_nodes = 2^(levels+1) - 1, the n_leaves = 2^levels leaves are the last level.
 * Node a owns the tree-order points node_begin[a] .. node_begin[a] + node_size[a] - 1;
 * the root owns all n_points and each inner node is split into its children
 * in order (left child first).
 *
 * perm[k] is the index, in the caller's point order, of the k-th point in tree
 * order (a bijection of 0..n_points-1). W and Y are in the caller's order.
 *
 * rank[a] = s_a, the skeleton size of node a (0 = no basis). basis[a] is the
 * interpolation matrix P_a, row-major: n_a x s_a for a leaf, (s_l + s_r) x s_a
 * for an inner node with children l, r (the nested transfer matrix). It may be
 * NULL when s_a = 0. The upward pass forms w_a = P_a^T W_a (leaf) or
 * P_a^T [w_l; w_r] (inner), the downward pass applies P_a (Section 2.1).
 *
 * Near list (CSR over leaves, leaf-local ids 0..n_leaves-1): for target leaf i
 * the entries near_ptr[i] .. near_ptr[i+1]-1 name source leaves near_idx[e];
 * near[e] is the dense block D_ij (n_i x n_j, row-major).
 *
 * Far list (CSR over all nodes, node ids): for target node a the entries
 * far_ptr[a] .. far_ptr[a+1]-1 name source nodes far_idx[e] on the same level;
 * coupling[e] is B_ab (s_a x s_b, row-major), may be NULL when it is empty.
 */
typedef struct {
  int64_t n_points;
  int32_t levels;
  const int64_t* node_begin;        /* [n_nodes] */
  const int64_t* node_size;         /* [n_nodes] */
  const int32_t* rank;              /* [n_nodes] */
  const int64_t* near_ptr;          /* [n_leaves + 1] */
  const int32_t* near_idx;          /* [near_ptr[n_leaves]] */
  const int64_t* far_ptr;           /* [n_nodes + 1] */
  const int32_t* far_idx;           /* [far_ptr[n_nodes]] */
  const double* const* basis;       /* [n_nodes] */
  const double* const* coupling;    /* [far_ptr[n_nodes]] */
  const double* const* near;        /* [near_ptr[n_leaves]] */
  const int64_t* perm;              /* [n_points] */
} hmat_desc;

/*
 * Inspector (Section 3.1, "Modularizing compression"): tree construction,
 * interaction computation and low-rank approximation in one native call.
 *
 * Kernel functions (Section 1): HMAT_KERNEL_GAUSSIAN exp(-r^2 / (2 h^2)) with
 * kernel_param = h > 0; HMAT_KERNEL_IMQ 1 / sqrt(r^2 + c^2) with kernel_param =
 * c > 0; HMAT_KERNEL_INVDIST 1 / r (the kernel of the comparison with SMASH,
 * Section 4.1), 0 for coincident points including the diagonal (the paper leaves
 * k(x, x) undefined), kernel_param ignored.
 *
 * Admissibility (Section 2.1, "Compression"; Section 4.1 for HSS):
 * HMAT_ADM_HSS - every pair of distinct siblings is far (weak admissibility);
 * HMAT_ADM_GEOMETRIC - nodes a, b are far when the distance of their centroids
 *   exceeds eta * max(r_a, r_b), r the largest distance of a point of the node
 *   to its centroid (the paper's tau * dist > diam_a + diam_b with tau = 2/eta);
 * HMAT_ADM_NONE - nothing is far: every block is kept dense;
 * HMAT_ADM_TAU - the paper's tau * dist(a, b) > diam(a) + diam(b) with tau = eta,
 *   on bounding boxes: dist = the Euclidean gap between the boxes of a and b, diam
 *   = a box's diagonal;
 * HMAT_ADM_BUDGET - GOFMM's budget (the paper's H2-b, Section 4.1), budget = eta in
 *   [0, 1]: the 32 nearest neighbours of every point vote for their leaves, a leaf
 *   is near itself and the floor(budget * leaves) most-voted leaves (ties by leaf
 *   index), symmetrised, and a node pair is far when no near leaf pair lies below it
 *   (budget 0 gives HSS). The neighbours are found by brute force (n^2 distances).
 *
 * Cluster trees (Section 3.1, tree construction): HMAT_TREE_KD splits a node at the
 * median of its widest bounding-box dimension; HMAT_TREE_TWO_MEANS (the paper's
 * choice for d > 3) at the median of the projection onto q - p, p the point farthest
 * from the node's point of smallest input index and q the point farthest from p
 * (ties by input index). Both give a perfect tree of depth ceil(log2(n / leaf)).
 */
#define HMAT_KERNEL_GAUSSIAN 0
#define HMAT_KERNEL_IMQ 1
#define HMAT_KERNEL_INVDIST 2
#define HMAT_ADM_HSS 0
#define HMAT_ADM_GEOMETRIC 1
#define HMAT_ADM_NONE 2
#define HMAT_ADM_TAU 3
#define HMAT_ADM_BUDGET 4
#define HMAT_TREE_KD 0
#define HMAT_TREE_TWO_MEANS 1

typedef struct {
  int64_t n_points;
  int32_t dim;
  const double* points;      /* host, n_points x dim, row-major, caller order */
  int32_t kernel;            /* HMAT_KERNEL_* */
  double kernel_param;
  int32_t admissibility;     /* HMAT_ADM_* */
  double eta;
  int32_t leaf_size;         /* >= 2 */
  double tol;                /* ID tolerance (bacc): rank = #{|R_jj| > tol |R_11|} */
  int32_t max_rank;          /* rank cap (>= 1) */
  int32_t exact_columns;     /* 1: every far point as ID column, 0: a sample, -1: exact iff n_points <= 4096 */
  uint64_t sample_seed;      /* seed of the column sample */
  int32_t threads;           /* host threads of the inspector (0: all cores) */
  int32_t tree;              /* HMAT_TREE_KD or HMAT_TREE_TWO_MEANS */
} hmat_build_params;

/*
 * hmat_build - compress the kernel matrix of a point set and load it.
 *
 * The cluster tree is a perfect binary tree of depth L = ceil(log2(n / leaf_size)):
 * every node above the leaves is split at a median (HMAT_TREE_KD: of its widest
 * bounding-box dimension, lowest dimension on ties, points ordered by that
 * coordinate, then by input index; HMAT_TREE_TWO_MEANS: see above; the left child
 * takes floor(n/2)). Near/far pairs come from a
 * dual-tree traversal from (root, root). Each node that is, or has an ancestor
 * that is, in a far pair gets a nested row interpolative decomposition (column-
 * pivoted Householder QR of K(R, C)^T; R = the node's points for a leaf and the
 * children's skeletons otherwise; C = the points whose interaction with the node
 * is approximated, or a seeded uniform sample of max(4 max_rank, 512) of them).
 * The near blocks D and coupling blocks B are evaluated on the GPU directly into
 * the packed device arena (with HMAT_BUILD_NEAR_OTF the near blocks are not stored
 * but evaluated inside every FP64 evaluation). `flags`: any of HMAT_LOAD_MIXED,
 * HMAT_LOAD_MIXED_ONLY, HMAT_BUILD_ID_GPU, HMAT_BUILD_NEAR_OTF (not with either
 * mixed flag); other bits:
 * HMAT_EUNSUPPORTED. Synchronous; host threads as requested.
 */
hmat_status hmat_build(const hmat_build_params* params, int flags, hmat_t* out);

/*
 * Inspector reuse (Section 3.2, "Reusing inspection"): the tree and the near/far
 * lists depend only on the points and the admissibility (inspector-p1); the bases
 * and blocks depend on the kernel and the accuracy too (inspector-p2). A plan holds
 * the first part, so a new kernel, kernel parameter or tolerance recompresses
 * without rebuilding it.
 *
 * hmat_plan_create - build the cluster tree and the interaction lists of a point
 * set (the tree, admissibility and threads of hmat_build; copies the points).
 * hmat_plan_build - nested row IDs for one kernel and accuracy on the host, near
 * and coupling blocks evaluated on the GPU, then the load; returns a new handle
 * that owns its memory (the plan may be freed or reused afterwards). hmat_build is
 * hmat_plan_create + hmat_plan_build + hmat_plan_free, so both give bitwise the
 * same HMatrix.
 * hmat_plan_free - release the plan (NULL is a no-op).
 */
typedef struct hmat_plan* hmat_plan_t;
typedef struct {
  int64_t n_points;
  int32_t dim;
  const double* points;      /* host, n_points x dim, row-major, caller order */
  int32_t admissibility;     /* HMAT_ADM_* */
  double eta;
  int32_t leaf_size;         /* >= 2 */
  int32_t threads;           /* host threads (0: all cores) */
  int32_t tree;              /* HMAT_TREE_KD or HMAT_TREE_TWO_MEANS */
} hmat_plan_params;
typedef struct {
  int32_t kernel;            /* HMAT_KERNEL_* */
  double kernel_param;
  double tol;                /* ID tolerance (bacc) */
  int32_t max_rank;          /* rank cap (>= 1) */
  int32_t exact_columns;     /* as in hmat_build_params */
  uint64_t sample_seed;
} hmat_compress_params;
hmat_status hmat_plan_create(const hmat_plan_params* params, hmat_plan_t* out);
hmat_status hmat_plan_build(hmat_plan_t plan, const hmat_compress_params* params, int flags, hmat_t* out);
hmat_status hmat_plan_free(hmat_plan_t plan);

/*
 * hmat_structure - copy out the structure of a loaded HMatrix (each pointer may
 * be NULL to skip it): perm [n_points], rank [n_nodes], near_ptr [n_leaves + 1],
 * near_idx [near entries], far_ptr [n_nodes + 1], far_idx [far entries], in the
 * layout of hmat_desc.
 */
hmat_status hmat_structure(hmat_t h, int64_t* perm, int32_t* rank, int64_t* near_ptr, int32_t* near_idx,
                           int64_t* far_ptr, int32_t* far_idx);

/* Evaluation modes for hmat_eval. */
#define HMAT_MODE_FP64 0            /* every block and every sum in FP64 (DFMA) */
#define HMAT_MODE_MIXED 1           /* near field (and high-rank coupling) on the tensor cores (FP16
                                       hi+lo splits of the blocks and of W, FP32 accumulation drained
                                       every few blocks into compensated sums), far field in FP32;
                                       needs a handle loaded with HMAT_LOAD_MIXED */

/* Build flag (hmat_build, hmat_plan_build): the nested row IDs run on the GPU, one CTA
   per node of a tree level (same algorithm as on the host; sums in another order, so a
   pivot may differ where two candidates are within rounding of each other). */
#define HMAT_BUILD_ID_GPU 2

/* Build flag (hmat_build, hmat_plan_build): the near blocks D_ij are not stored. The
   FP64 near field evaluates each entry K(x_i, x_j) from the points inside its kernel,
   with the formula the build uses to store them, so the result is bitwise that of a
   handle built without the flag; the handle keeps the points (8 B x dim per point)
   instead of the near blocks (8 B per near value), and pays the kernel evaluations in
   time, once per column tile of the product. FP64 mode only: with HMAT_LOAD_MIXED the
   build returns HMAT_EUNSUPPORTED, and so does hmat_load (it has no points). */
#define HMAT_BUILD_NEAR_OTF 4

/* Load flags (hmat_load, hmat_build). */
#define HMAT_LOAD_MIXED 1           /* also keep the tensor-core copy of the near blocks (FP16 hi/lo,
                                       4 bytes per value) and an FP32 copy of the bases and coupling
                                       blocks, for HMAT_MODE_MIXED */
#define HMAT_LOAD_MIXED_ONLY 8      /* HMAT_LOAD_MIXED, then drop the FP64 blocks (8 bytes per stored
                                       value): the handle serves HMAT_MODE_MIXED only (HMAT_MODE_FP64,
                                       its autotuning and hmat_eval_noalloc return HMAT_EUNSUPPORTED), in
                                       a third of the device memory; for memory-bound serving of many
                                       resident matrices */

/*
 * hmat_load - validate an HMatrix description, pack its blocks per tree level
 * into one device arena and return a handle that owns it.
 *
 * Synchronous. Validation (HMAT_EINVAL, nothing allocated on failure): tree
 * shape and index ranges, CSR pointers non-decreasing, list ids in range, far
 * partners on the same level and distinct, perm a bijection, every non-empty
 * block pointer non-NULL and every stored value finite. `flags` is 0,
 * HMAT_LOAD_MIXED or HMAT_LOAD_MIXED_ONLY (any other bit: HMAT_EUNSUPPORTED).
 * The device is the one current at the call. Returns HMAT_ENOMEM when the
 * arena does not fit.
 */
hmat_status hmat_load(const hmat_desc* desc, int flags, hmat_t* out);

/*
 * hmat_eval - Y = K~ W for the HMatrix of `h`.
 *
 * W (n_points x q, FP64) and Y (n_points x q, FP64) are device pointers in the
 * caller's point order; Y is overwritten, not accumulated; W and Y must not
 * overlap. q = 0 is a no-op. `stream` is a cudaStream_t (NULL = legacy default
 * stream); the call only enqueues work and returns. Calls on one handle must
 * be ordered (one stream, or synchronised by the caller): they share the
 * handle's workspace. The workspace grows to q on demand with cudaMalloc,
 * which synchronises the device; hmat_reserve avoids that inside a timed or
 * captured region. `mode` is HMAT_MODE_FP64 or HMAT_MODE_MIXED (the latter on a
 * handle loaded with HMAT_LOAD_MIXED, else HMAT_EUNSUPPORTED).
 */
hmat_status hmat_eval(hmat_t h, const double* W, double* Y, int64_t q, int mode, void* stream);

/*
 * Element types of W and Y for the *_typed entry points (the evaluation mode is
 * independent of them).
 * HMAT_DTYPE_F64 - double.
 * HMAT_DTYPE_F32 - float. In HMAT_MODE_FP64 the evaluation is the FP64 one of the
 *   widened W (every sum in FP64) and Y is its value rounded to nearest once. In
 *   HMAT_MODE_MIXED W is read as it is (the split and the far field start from FP32
 *   anyway) and Y is written as the FP32 rounding of the mode's result. The
 *   workspace of an FP64-mode evaluation with FP32 W and Y holds FP64 copies of both
 *   (2 x n_points x q doubles more).
 */
#define HMAT_DTYPE_F64 0
#define HMAT_DTYPE_F32 1

/*
 * hmat_eval_typed - hmat_eval for W and Y of element type `dtype` (n_points x q,
 * device pointers, caller order); HMAT_EINVAL for another dtype. hmat_eval(h, W, Y,
 * q, mode, stream) is hmat_eval_typed(h, W, Y, q, mode, HMAT_DTYPE_F64, stream).
 */
hmat_status hmat_eval_typed(hmat_t h, const void* W, void* Y, int64_t q, int mode, int dtype, void* stream);

/* hmat_reserve - size the workspace for right-hand sides of up to q_max columns. */
hmat_status hmat_reserve(hmat_t h, int64_t q_max);

/*
 * hmat_eval_host - Y = K~ W with W and Y in HOST memory (n_points x q, FP64,
 * caller order): copies W to a device buffer owned by the handle, evaluates as
 * hmat_eval does, copies Y back, all on `stream`, and synchronises the stream
 * before returning. Pinned host buffers give full copy bandwidth. The device
 * buffers grow on demand (cudaMalloc, which synchronises the device). In the mixed
 * mode with q >= 128 the columns are evaluated in two groups whose copies overlap the
 * other group's evaluation (on a copy stream of the handle); the groups' W scales
 * differ from one whole-q evaluation, so results can differ from hmat_eval's by
 * rounding (within the mixed mode's accuracy).
 */
hmat_status hmat_eval_host(hmat_t h, const double* W, double* Y, int64_t q, int mode, void* stream);
/* hmat_eval_host_typed - hmat_eval_host for host W and Y of element type `dtype`. */
hmat_status hmat_eval_host_typed(hmat_t h, const void* W, void* Y, int64_t q, int mode, int dtype, void* stream);

/*
 * hmat_profile - enable (1) or disable (0) CUDA-event timing of every kernel
 * launch of later evaluations on this handle; enabling clears earlier records.
 * enable = 2 times the same launches with the mixed mode's far chain moved from its
 * side stream onto the caller's stream, so that every launch's time is its own
 * and not shared with a launch running beside it (the evaluation is otherwise
 * unchanged; its result is bitwise the same).
 * hmat_phase_times - synchronise on the recorded events and return, for phase
 * kind k < n, the summed device time in ms[k] and the number of launches in
 * launches[k] since profiling was enabled; then clear the records. Phase kinds:
 * HMAT_PHASE_NEAR (near-field reduction over D), HMAT_PHASE_UP_LEAF (w = P^T W
 * at the leaves), HMAT_PHASE_UP_TRANSFER (w = P^T [w_l; w_r], one launch per
 * level), HMAT_PHASE_COUPLING (u = sum B w), HMAT_PHASE_DOWN_TRANSFER
 * ([u_l; u_r] += P u, one launch per level), HMAT_PHASE_DOWN_LEAF (Y += P u),
 * HMAT_PHASE_SPLIT (mixed mode only: scale and split W into FP16 hi/lo tiles),
 * HMAT_PHASE_FAR_UP (one persistent launch over every tree level: in the FP64 mode
 * the whole far field, from the upward pass to the downward leaf step; in the mixed
 * mode the upward pass, and, when the coupling runs in FP32, the coupling and the
 * downward transfers), HMAT_PHASE_FAR_DOWN (mixed mode: one persistent launch of the
 * downward transfers after the tensor-core coupling). In the mixed mode the downward
 * leaf step is one persistent launch too (HMAT_PHASE_DOWN_LEAF). The FP64 mode's
 * other phase kinds are hmat_eval_noalloc's, which keeps one launch per level.
 */
#define HMAT_PHASE_NEAR 0
#define HMAT_PHASE_UP_LEAF 1
#define HMAT_PHASE_UP_TRANSFER 2
#define HMAT_PHASE_COUPLING 3
#define HMAT_PHASE_DOWN_TRANSFER 4
#define HMAT_PHASE_DOWN_LEAF 5
#define HMAT_PHASE_SPLIT 6          /* mixed mode: max |W| and the FP16 hi/lo split of W */
#define HMAT_PHASE_FAR_UP 7         /* persistent far-chain launch (FP64: the whole far field) */
#define HMAT_PHASE_FAR_DOWN 8       /* mixed mode: persistent far-chain launch, downward transfers */
#define HMAT_PHASE_COUNT 9
hmat_status hmat_profile(hmat_t h, int enable);
hmat_status hmat_phase_times(hmat_t h, double* ms, int64_t* launches, int n);

/*
 * hmat_measure_fp64_peak - FP64 FMA throughput of the current device, measured
 * with a register-resident DFMA loop on every SM (about 0.1 s); *gflops receives
 * GFLOP/s (2 flops per FMA). This is the ceiling of the FP64 evaluation mode.
 */
hmat_status hmat_measure_fp64_peak(double* gflops);

/*
 * hmat_selftest_conversions - checks, on the current device, the integer-unit
 * conversions the mixed mode uses (binary32 -> binary64 widening, round-to-nearest-
 * even binary64 -> binary32 narrowing, scaling a binary64 value by 2^e) bitwise
 * against the hardware conversion and multiply, on n samples: the first 144 pair
 * special values (signed zeros, infinities, NaN, ends of the normal and subnormal
 * ranges), the rest are drawn from `seed` (random bit patterns of every exponent
 * class, a quarter of the doubles at a rounding tie, scale exponents in [-300, 300]).
 * Each conversion is checked in both of its forms (hardware fallback inline and out
 * of line); mismatches[0..2] receive the number of differing widenings, narrowings
 * and scalings over both forms (NaN matches any NaN).
 * Synchronous; HMAT_EINVAL for n < 0 or a null mismatches.
 */
hmat_status hmat_selftest_conversions(int64_t n, uint64_t seed, int64_t* mismatches);

/*
 * hmat_eval_noalloc - the FP64 evaluation of hmat_eval (mode HMAT_MODE_FP64)
 * for callers that must not allocate device memory during the call. The paper
 * has no counterpart; this exists for callers such as a latency-critical
 * serving loop, where a cudaMalloc would synchronise the whole device and stall
 * the work of other streams, or a process whose device memory is entirely
 * owned by another allocator (for example a framework's caching allocator), in
 * which a foreign cudaMalloc can fail or fragment the pool.
 *
 * The skeleton workspaces (the upward weights w and the downward potentials u,
 * sum of ranks x q values each) live in one static device array of
 * HMAT_NOALLOC_SCRATCH_VALUES doubles (16 MiB) compiled into libhmat.so. The
 * first hmat_load or hmat_build on a device loads that array onto the device
 * (both allocate anyway) and every load stores its device address in the handle;
 * the device then holds the array until the process exits. The call returns
 * HMAT_EINVAL when 2 x (sum of ranks) x q exceeds that size (the sum of ranks is
 * out[7] of hmat_info). It calls no cudaMalloc or cudaFree and no allocating
 * library routine, and looks nothing up: the handle must already exist, and its
 * own workspace (hmat_info out[8]) is neither used nor grown.
 *
 * Every call shares the one array and leaves its last contents behind; every
 * workspace row is written before it is read, so nothing needs clearing. Calls
 * whose work overlaps on the GPU (other streams, other handles, other host
 * threads) race on the array: order them.
 * Arguments and results are those of hmat_eval.
 */
#define HMAT_NOALLOC_SCRATCH_VALUES 2097152
hmat_status hmat_eval_noalloc(hmat_t h, const double* W, double* Y, int64_t q, void* stream);

/*
 * hmat_autotune - choose the tile shapes of h's evaluations with q columns in
 * `mode` by timing candidates on the device (CUDA events on `stream`); later
 * hmat_eval, hmat_eval_host, batch and server evaluations of h with that q and mode
 * use them. FP64 mode: per near-field launch (one per row-tile size), the column
 * tile of the grouped GEMM (1 to 64 columns) among those that pad less than half a
 * tile (a long launch is timed on its longest tiles), then the column tile of the
 * persistent far chain, timed on whole chain launches (narrower tiles too when the
 * chain is short: they spread thin levels over more SMs). Mixed mode: the column width of the
 * tensor-core near-field CTAs (fewer, wider tiles copy each near block fewer
 * times; more, narrower ones fill more SMs on a matrix with few leaves). Every
 * candidate sums each output in the same order, so results are bitwise those of
 * an untuned evaluation.
 *
 * Synchronous: allocates private W, Y and workspaces (cudaMalloc), runs the
 * candidates on `stream`, frees them and returns. Must not run while another
 * thread evaluates h (the choice table is not locked). A call for a (q, mode)
 * already tuned replaces the earlier choice. `report` (may be NULL) receives the
 * number of launches tuned, the summed time of those launches with the default and
 * with the chosen shapes (ms; a long launch timed on a prefix counts at full
 * length, scaled by its tile count; in the mixed mode, when it has a far field, the
 * time of a whole evaluation), the chosen near-field width in columns and the
 * chosen far-chain grid.
 */
typedef struct {
  int64_t q;
  int32_t mode;
  int32_t launches_tuned;
  double default_ms;
  double tuned_ms;
  int32_t near_cols;
  int32_t chain_grid;        /* mixed mode: CTAs of the persistent far chain, 0 = every resident CTA */
} hmat_tune_report;
hmat_status hmat_autotune(hmat_t h, int64_t q, int mode, void* stream, hmat_tune_report* report);

/*
 * hmat_tune_apply - install a mixed-mode choice without timing (for example one that
 * hmat_autotune reported in an earlier process): for evaluations of h with
 * choice->q columns, choice->near_cols columns per tensor-core CTA (0: the default;
 * else one of the widths hmat_autotune tries for that q, else HMAT_EINVAL) and
 * choice->chain_grid CTAs for the persistent far chain (0: every resident CTA; any
 * positive count is valid: the chain completes with any number of CTAs, even one).
 * Results are bitwise the same for every choice. choice->mode must be
 * HMAT_MODE_MIXED (else HMAT_EUNSUPPORTED); the other fields are ignored.
 */
hmat_status hmat_tune_apply(hmat_t h, const hmat_tune_report* choice);

/*
 * Batches: many HMatrices (uneven sizes, ranks and q) evaluated together. The first
 * hmat_batch_eval with a given set of W, Y pointers and q values captures one CUDA
 * graph in which every step of the evaluation is one launch over all members (a
 * flattened work list with a member table): in the mixed mode the W splits, the
 * persistent far chains, the tensor-core couplings, the tensor-core near fields and
 * the downward leaf steps of all members, about ten kernels in all; in the FP64 mode
 * each member's near-field launches on parallel graph branches, then the far fields
 * of all members in one persistent chain launch per column tile width. Later calls
 * with the same arguments replay that graph with a single launch (a call with other
 * arguments captures a new graph). Each member's result is bitwise what it gets
 * alone, with the handle's tuned tile shapes. The same handle may appear more than
 * once. Handles must outlive the batch and must not be evaluated elsewhere while one
 * of the batch's graphs runs. The batch owns one device block for every member's
 * workspaces and the launch tables.
 *
 * hmat_batch_create - `count` handles (all on the current device), `mode` is
 * HMAT_MODE_FP64 or HMAT_MODE_MIXED (every handle loaded with HMAT_LOAD_MIXED).
 * hmat_batch_eval - Y[i] = K~_i W[i] (device pointers, n_i x q[i], caller order)
 * for every member, enqueued on `stream`; the first call for a new argument set
 * allocates workspaces (cudaMalloc, which synchronises the device).
 * hmat_batch_info - out[0] members, out[1] kernel launches in the graph of the last
 * argument set (0 before the first call), out[2] device bytes held by the batch, out[3]
 * the CTAs of its chain launches (0: every resident CTA), out[4] 1 when the batch runs
 * the branched schedule, out[5] 1 when its mixed members run at their default
 * tensor-core column widths instead of their own tuned ones.
 * hmat_batch_autotune - time whole replays of the batch for these arguments with the
 * chain launches capped at several CTA counts (the chains run beside the tensor-core
 * near field, which needs whole SMs), and with the branched schedule (every member's
 * own evaluation as a branch of the graph: more, smaller launches that overlap one
 * another), in the mixed mode also with every member at its default tensor-core column
 * width (a width tuned for a member alone need not suit it in the batch), and keep the
 * fastest for later calls; the members' other tile shapes are those of hmat_autotune.
 * Results are bitwise the same for every choice. ms_default /
 * ms_tuned (may be NULL) receive the replay time of the flattened schedule with every
 * resident CTA and of the choice. Synchronous.
 */
typedef struct hmat_batch* hmat_batch_t;
hmat_status hmat_batch_create(const hmat_t* handles, int count, int mode, hmat_batch_t* out);
hmat_status hmat_batch_eval(hmat_batch_t b, const double* const* W, double* const* Y, const int64_t* q,
                            void* stream);
/* hmat_batch_eval_typed - hmat_batch_eval with every member's W and Y of element type
 * `dtype` (a call with another dtype than the captured graph's captures a new one). */
hmat_status hmat_batch_eval_typed(hmat_batch_t b, const void* const* W, void* const* Y, const int64_t* q, int dtype,
                                  void* stream);
hmat_status hmat_batch_info(hmat_batch_t b, int64_t* out, int n);
hmat_status hmat_batch_autotune(hmat_batch_t b, const void* const* W, void* const* Y, const int64_t* q, int dtype,
                                void* stream, double* ms_default, double* ms_tuned);
/* hmat_batch_schedule - pin the schedule without timing: branched 0 (flattened, the
 * default) or 1, the chain launches' CTAs (0: every resident CTA) and default_widths 0
 * (the members' tuned tensor-core column widths, the default) or 1 (their default
 * widths); the next call recaptures. HMAT_EINVAL for other values. */
hmat_status hmat_batch_schedule(hmat_batch_t b, int branched, int chain_grid, int default_widths);
hmat_status hmat_batch_free(hmat_batch_t b);

/*
 * Serving: a request loop over HMatrices kept resident on the device. Requests
 * (a matrix, a host W of n x q, a host Y) are queued by hmat_server_submit and
 * dispatched by a host thread: a request is admitted when one of `slots` CUDA
 * streams is free and the device memory it needs (its workspaces and the device
 * copies of W and Y) fits, with the memory of the requests in flight, within
 * `memory_budget` bytes. Requests on the same matrix that wait together are run
 * as one evaluation with their W columns side by side (up to `max_q` columns),
 * which reads each stored block once for all of them (continuous batching);
 * requests in different slots overlap on the device. Results are those of
 * hmat_eval on each request alone: bitwise in FP64 mode (every column of Y
 * depends only on the same column of W, summed in the same order), within the
 * mode's accuracy in the mixed mode (W's power-of-two scale is taken over the
 * merged columns). Workspace comes from a stream-ordered memory pool. Served
 * handles must not be evaluated or profiled elsewhere while the server runs.
 *
 * hmat_server_submit - W and Y are pinned host buffers (cudaHostAlloc,
 * cudaHostRegister) or device buffers, n x q row-major with row strides ldw and
 * ldy (>= q, in values), valid until the request completes (pageable host memory: HMAT_EINVAL, as its copies would stall the
 * dispatcher); *id identifies the request. Returns HMAT_ENOMEM when the request
 * alone exceeds the memory budget, HMAT_EINVAL when q > max_q.
 * hmat_server_wait - wait for request `id` (timeout_ms < 0: no limit); returns
 * its status, HMAT_ETIMEOUT if it has not completed in time. A completed request
 * is forgotten once waited on (waiting again: HMAT_EINVAL).
 * hmat_server_stats - out[0] completed requests, out[1] p50 and out[2] p99
 * latency in ms (submit to result in host memory), out[3] mean requests per
 * evaluation, out[4] evaluations, out[5] peak device bytes in flight, out[6]
 * requests refused with HMAT_EBUSY.
 * hmat_server_matrix_stats - for one matrix: out[0] completed requests, out[1] p50
 * and out[2] p99 latency in ms.
 *
 * Load shedding: with max_pending > 0, hmat_server_submit returns HMAT_EBUSY (and
 * queues nothing) while max_pending requests wait for admission; a request stream
 * beyond the device's rate is then served at that rate with bounded queueing delay
 * instead of an unbounded queue.
 */
typedef struct hmat_server* hmat_server_t;
typedef struct {
  int slots;                /* evaluations in flight at once (>= 1) */
  int64_t memory_budget;    /* device bytes of the requests in flight (> 0) */
  int64_t max_q;            /* columns of one merged evaluation (>= 1) */
  int mode;                 /* HMAT_MODE_FP64 or HMAT_MODE_MIXED */
  int64_t max_pending;      /* requests waiting for admission at most (0: no limit) */
} hmat_server_params;
hmat_status hmat_server_create(const hmat_t* handles, int count, const hmat_server_params* params,
                               hmat_server_t* out);
hmat_status hmat_server_submit(hmat_server_t s, int matrix, const double* W, int64_t ldw, double* Y, int64_t ldy,
                               int64_t q, int64_t* id);
/* hmat_server_submit_typed - hmat_server_submit for W and Y of element type `dtype`
 * (strides in values of that type). Requests merge only with requests of the same
 * matrix and dtype. */
hmat_status hmat_server_submit_typed(hmat_server_t s, int matrix, const void* W, int64_t ldw, void* Y, int64_t ldy,
                                     int64_t q, int dtype, int64_t* id);
hmat_status hmat_server_wait(hmat_server_t s, int64_t id, int timeout_ms);
hmat_status hmat_server_stats(hmat_server_t s, double* out, int n);
hmat_status hmat_server_matrix_stats(hmat_server_t s, int matrix, double* out, int n);
hmat_status hmat_server_free(hmat_server_t s);

/*
 * hmat_status_poll - synchronise `stream` and return the device status word
 * latched by the kernels since the last poll (HMAT_OK when nothing happened),
 * then clear it.
 */
hmat_status hmat_status_poll(hmat_t h, void* stream);

/*
 * hmat_selftest_timeout - failure-detection self-test (no counterpart in the
 * paper). Enqueues on `stream` one device wait, through the bounded-wait routine
 * of the tensor-core near-field kernel, on a barrier that nothing completes; after
 * limit_ns nanoseconds (0 < limit_ns <= 10 s, else HMAT_EINVAL) the wait gives up
 * and latches HMAT_ETIMEOUT in h's status word, as a stuck evaluation would, so the
 * next hmat_status_poll returns HMAT_ETIMEOUT. The wait holds no copy, MMA or
 * tensor memory, so the CUDA context stays usable afterwards.
 */
hmat_status hmat_selftest_timeout(hmat_t h, int64_t limit_ns, void* stream);

/*
 * hmat_selftest_chain_timeout - failure-detection self-test of the persistent far
 * chain of `mode` (no counterpart in the paper). Enqueues on `stream` the chain's
 * first launch for q columns (on the handle's own workspace, which it reserves like
 * hmat_eval) with every dependency requirement raised by one, so that no wait can be
 * met: each wait gives up after limit_ns nanoseconds (0 < limit_ns <= 10 s, else
 * HMAT_EINVAL), latches HMAT_ETIMEOUT in h's status word and stops the launch, which
 * reads and writes no workspace before its waits. The next hmat_status_poll returns
 * HMAT_ETIMEOUT; the context stays usable. HMAT_EUNSUPPORTED when the handle has no
 * copy for `mode`, HMAT_EINVAL when the HMatrix has no far field.
 */
hmat_status hmat_selftest_chain_timeout(hmat_t h, int64_t q, int mode, int64_t limit_ns, void* stream);

/*
 * hmat_selftest_row_id - runs the GPU row interpolative decomposition of the inspector
 * (HMAT_BUILD_ID_GPU; Section 3.1, low-rank approximation) on a given matrix instead
 * of one formed from points, to check it against a reference (no counterpart in the
 * paper). M: host, n_rows x n_cols row-major, the rows are the candidates. The ID is
 * the column-pivoted QR of M^T stopped at the first |R_kk| <= tol |R_11| or at max_rank:
 * *rank = k, piv[0..n_rows-1] the row order after the pivoting (piv[0..k-1] the
 * skeleton), T (k x (n_rows - k), row-major) = R_11^{-1} R_12, so that row piv[k + c]
 * of M ~= sum_i T[i][c] M[piv[i]]. Synchronous; n_rows <= 8192 and n_rows x n_cols <=
 * 2^26 (else HMAT_EINVAL).
 */
hmat_status hmat_selftest_row_id(const double* M, int64_t n_rows, int64_t n_cols, double tol, int32_t max_rank,
                                 int32_t* piv, int32_t* rank, double* T);

/*
 * hmat_selftest_device_check - failure-detection self-test of the persistent far
 * chain's index checks (no counterpart in the paper): every item, tile and node index
 * a chain launch takes from device memory is checked against the size of the array it
 * indexes before anything is read through it, and an inconsistent one latches
 * HMAT_EDEVICE in the status word and stops the launch. This enqueues one chain launch
 * of `mode` for q columns whose only ticket names the item just past the handle's item
 * array; the check catches it before any read, so the next hmat_status_poll returns
 * HMAT_EDEVICE and the context stays usable. HMAT_EUNSUPPORTED when the handle has no
 * copy for `mode`, HMAT_EINVAL when it has no far field.
 */
hmat_status hmat_selftest_device_check(hmat_t h, int64_t q, int mode, void* stream);

/* hmat_info - sizes of the loaded HMatrix: out[0] = n_points, out[1] = levels,
 * out[2] = near entries, out[3] = far entries, out[4] = near values (stored, or
 * evaluated on the fly under HMAT_BUILD_NEAR_OTF, see out[10]),
 * out[5] = stored basis values, out[6] = stored coupling values,
 * out[7] = sum of ranks, out[8] = device bytes held by the handle,
 * out[9] = engine of the mixed mode's coupling reduction: 0 no mixed copy, 1 FP32
 * CUDA cores, 2 tensor cores (chosen at load: tensor cores when the stored coupling
 * values fill at least a quarter of the padded 128 x 64 tiles they would occupy),
 * out[10] = 1 when the near blocks are evaluated on the fly, else 0. */
hmat_status hmat_info(hmat_t h, int64_t* out, int n_out);

/* hmat_free - release every device and host resource of the handle (synchronises the device). */
hmat_status hmat_free(hmat_t h);

/* hmat_strerror - static text for a status code. */
const char* hmat_strerror(hmat_status s);

#ifdef __cplusplus
}
#endif

#endif  /* HMAT_H_ */
