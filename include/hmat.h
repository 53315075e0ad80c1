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
  HMAT_EDEVICE = -6          /* a kernel detected an inconsistent index or size */
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

/* Evaluation modes for hmat_eval. */
#define HMAT_MODE_FP64 0            /* every block and every sum in FP64 (DFMA) */

/*
 * hmat_load - validate an HMatrix description, pack its blocks per tree level
 * into one device arena and return a handle that owns it.
 *
 * Synchronous. Validation (HMAT_EINVAL, nothing allocated on failure): tree
 * shape and index ranges, CSR pointers non-decreasing, list ids in range, far
 * partners on the same level and distinct, perm a bijection, every non-empty
 * block pointer non-NULL and every stored value finite. `flags` must be 0.
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
 * captured region. `mode` is HMAT_MODE_FP64.
 */
hmat_status hmat_eval(hmat_t h, const double* W, double* Y, int64_t q, int mode, void* stream);

/* hmat_reserve - size the workspace for right-hand sides of up to q_max columns. */
hmat_status hmat_reserve(hmat_t h, int64_t q_max);

/*
 * hmat_status_poll - synchronise `stream` and return the device status word
 * latched by the kernels since the last poll (HMAT_OK when nothing happened),
 * then clear it.
 */
hmat_status hmat_status_poll(hmat_t h, void* stream);

/* hmat_info - sizes of the loaded HMatrix: out[0] = n_points, out[1] = levels,
 * out[2] = near entries, out[3] = far entries, out[4] = stored near values,
 * out[5] = stored basis values, out[6] = stored coupling values,
 * out[7] = sum of ranks, out[8] = device bytes held by the handle. */
hmat_status hmat_info(hmat_t h, int64_t* out, int n_out);

/* hmat_free - release every device and host resource of the handle (synchronises the device). */
hmat_status hmat_free(hmat_t h);

/* hmat_strerror - static text for a status code. */
const char* hmat_strerror(hmat_status s);

#ifdef __cplusplus
}
#endif

#endif  /* HMAT_H_ */
