"""Plain FP64 CPU oracle for the HMatrix-matrix product Y = K~ W (MatRox, arXiv 1812.07152).

TEST INFRASTRUCTURE ONLY. This module is the slow, obviously correct reference
that the GPU path is checked against. Only the tests, the smoke check and the
bench's CPU-baseline leg may import it; the product path never does. It shares
no code with the CUDA path: the only common dependency is the seeded input
generator package ``workloads``, which holds none of the method's arithmetic.

What it builds and computes, with the passage each part follows:

* kernel matrix K(i, j) = k(x_i, x_j)                       (Section 1; 1/r: Section 4.1)
* cluster tree by recursive kd or two-means median splits   (Section 3.1, "Tree construction")
* near / far interactions from an admissibility condition   (Section 2.1, "Compression"; Section 4.1 for HSS)
* nested interpolative decomposition of the far field       (Section 2.1 footnote; Section 3.1, "Low-rank approximation")
* full-rank near blocks D and coupling blocks B             (Section 3.1)
* the evaluation: near-field reduction loop over D, bottom-up tree loop over
  the V bases, the B reduction loop, top-down tree loop over the U bases
                                                            (Section 2.1, "Evaluation")
* overall accuracy eps_f = ||K~W - KW||_F / ||KW||_F         (Section 5)

Readings where the paper is silent (kept identical in the GPU-side fixture
builder only through the fixture itself, never through shared code):

* the tree is perfect: every node above depth L = ceil(log2(N/m)) is split, the
  split dimension is the widest bounding-box extent (lowest index on ties),
  points are ordered by that coordinate (ties by input index) and the left child
  takes the first floor(n/2);
* geometric admissibility: far iff ||c_a - c_b|| > eta * max(r_a, r_b), c the
  centroid and r the largest distance of a point to it; found by a dual-tree
  traversal from (root, root);
* two-means (Section 3.1 names it for d > 3 without an algorithm): p farthest
  from the node's point of smallest input index, q farthest from p, points
  ordered by their projection onto q - p, split at the median;
* the paper's tau * dist(a, b) > diam(a) + diam(b) (Section 2.1) on bounding
  boxes: dist = the gap between the boxes, diam = the box diagonal;
* GOFMM's budget (the paper's H2-b, Section 4.1): 32 nearest neighbours per point
  vote for leaves; a leaf keeps floor(budget * leaves) most-voted leaves as near;
  a pair is far when no near leaf pair lies below it;
* HSS: every pair of distinct siblings is far, every leaf is near itself only;
* ID: column-pivoted QR of K(R, C)^T, rank = #{j : |R_jj| > tol * |R_11|}
  capped at max_rank, columns C = every point whose interaction with the node
  is approximated (exact when N <= 4096, else a seeded uniform sample of
  min(|C|, max(4 * max_rank, 512)) of them);
* U = V = P (K is symmetric); a node has a basis iff it or an ancestor has a
  far interaction; the root never has one;
* the singular kernel 1/r is 0 for coincident points (its diagonal included).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg as sla

EXACT_COLUMNS_MAX_N = 4096


# --------------------------------------------------------------------------------------
# Kernel function (Section 1: K(i, j) = k(x_i, x_j); Gaussian exp(-||x - y||^2 / 2h^2))
# --------------------------------------------------------------------------------------

def kernel_matrix(kind: str, param: float, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Dense kernel block K(X, Y) in FP64, from explicit coordinate differences."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    r2 = np.zeros((X.shape[0], Y.shape[0]))
    for k in range(X.shape[1]):
        diff = X[:, k][:, None] - Y[:, k][None, :]
        r2 += diff * diff
    if kind == "gaussian":
        return np.exp(-r2 / (2.0 * param * param))
    if kind == "imq":
        return 1.0 / np.sqrt(r2 + param * param)
    if kind == "invdist":
        # 1 / ||x - y||, the kernel of the comparison with SMASH (Section 4.1); the paper
        # does not define k(x, x): coincident points interact with 0
        out = np.zeros_like(r2)
        nz = r2 > 0.0
        out[nz] = 1.0 / np.sqrt(r2[nz])
        return out
    raise ValueError(f"unknown kernel {kind!r}")


# --------------------------------------------------------------------------------------
# Cluster tree (Section 3.1, "Tree construction": recursive kd partitioning, leaf size m)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class ClusterTree:
    """Perfect binary tree in heap numbering: node a has children 2a+1 and 2a+2,
    level l holds nodes 2^l - 1 .. 2^(l+1) - 2, the leaves are level ``levels``.

    ``perm[k]`` is the input index of the k-th point in tree order; node a owns the
    tree-order points ``begin[a] .. begin[a] + size[a] - 1``."""
    levels: int
    perm: np.ndarray
    begin: np.ndarray
    size: np.ndarray

    @property
    def n_nodes(self) -> int:
        return 2 ** (self.levels + 1) - 1

    @property
    def first_leaf(self) -> int:
        return 2 ** self.levels - 1

    @property
    def n_leaves(self) -> int:
        return 2 ** self.levels

    def level_of(self, a: int) -> int:
        return int(math.floor(math.log2(a + 1)))

    def nodes_at(self, level: int) -> range:
        return range(2 ** level - 1, 2 ** (level + 1) - 1)

    def index_set(self, a: int) -> np.ndarray:
        return np.arange(self.begin[a], self.begin[a] + self.size[a])


def tree_depth(n: int, leaf_size: int) -> int:
    """Smallest L with ceil(n / 2^L) <= leaf_size (0 when n <= leaf_size)."""
    L = 0
    while -(-n // (2 ** L)) > leaf_size:
        L += 1
    return L


def _sq_dist_seq(A: np.ndarray, y: np.ndarray) -> np.ndarray:
    """||a - y||^2 for every row a of A, summed over the coordinates in order."""
    out = np.zeros(A.shape[0])
    for k in range(A.shape[1]):
        diff = A[:, k] - y[k]
        out = out + diff * diff
    return out


def _first_argmax(values: np.ndarray, idx: np.ndarray) -> int:
    """Position of the largest value, the smallest input index among equal ones."""
    best = values.max()
    cand = np.flatnonzero(values == best)
    return int(cand[np.argmin(idx[cand])])


def two_means_order(pts: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Balanced two-means split of one node (Section 3.1: two-means partitioning for
    d > 3; the paper gives no algorithm). Two mutually far centres: p is the point
    farthest from the point of smallest input index, q the point farthest from p
    (ties by input index); each point is ordered by its projection onto q - p (ties
    by input index) and the first floor(n/2) form the left child, so the tree stays
    balanced."""
    a0 = int(np.argmin(idx))
    p = pts[_first_argmax(_sq_dist_seq(pts, pts[a0]), idx)]
    q = pts[_first_argmax(_sq_dist_seq(pts, p), idx)]
    proj = np.zeros(pts.shape[0])
    for k in range(pts.shape[1]):
        proj = proj + (pts[:, k] - p[k]) * (q[k] - p[k])
    return np.lexsort((idx, proj))


def build_cluster_tree(X: np.ndarray, leaf_size: int, tree: str = "kd") -> ClusterTree:
    """Perfect binary cluster tree with median splits down to a common depth (Section
    3.1): ``tree`` is ``"kd"`` (split the widest bounding-box dimension) or
    ``"two_means"`` (split along the axis of two mutually far points)."""
    if tree not in ("kd", "two_means"):
        raise ValueError(f"unknown tree {tree!r}")
    n = X.shape[0]
    if leaf_size < 2:
        raise ValueError("leaf size must be at least 2 (so that no leaf is empty)")
    L = tree_depth(n, leaf_size)
    n_nodes = 2 ** (L + 1) - 1
    begin = np.zeros(n_nodes, dtype=np.int64)
    size = np.zeros(n_nodes, dtype=np.int64)
    perm = np.arange(n, dtype=np.int64)
    size[0] = n
    for level in range(L):
        for a in range(2 ** level - 1, 2 ** (level + 1) - 1):
            b0, nb = begin[a], size[a]
            idx = perm[b0:b0 + nb]
            pts = X[idx]
            if nb == 0:
                order = np.zeros(0, dtype=np.int64)
            elif tree == "two_means":
                order = two_means_order(pts, idx)
            else:
                extent = pts.max(axis=0) - pts.min(axis=0)
                dim = int(np.argmax(extent))           # first maximum: lowest index on ties
                order = np.lexsort((idx, pts[:, dim]))  # by coordinate, then by input index
            perm[b0:b0 + nb] = idx[order]
            half = nb // 2
            begin[2 * a + 1], size[2 * a + 1] = b0, half
            begin[2 * a + 2], size[2 * a + 2] = b0 + half, nb - half
    return ClusterTree(L, perm, begin, size)


# --------------------------------------------------------------------------------------
# Interactions (Section 2.1: near pairs are kept dense, far pairs are approximated)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Interactions:
    near: List[Tuple[int, int]]   # (leaf i, leaf j), node ids
    far: List[Tuple[int, int]]    # (node a, node b) on the same level


def node_geometry(tree: ClusterTree, Xt: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Centroid and radius (largest distance of a point to the centroid) per node."""
    d = Xt.shape[1]
    cent = np.zeros((tree.n_nodes, d))
    rad = np.zeros(tree.n_nodes)
    for a in range(tree.n_nodes):
        pts = Xt[tree.begin[a]:tree.begin[a] + tree.size[a]]
        if len(pts) == 0:
            continue
        cent[a] = pts.mean(axis=0)
        rad[a] = np.sqrt(((pts - cent[a]) ** 2).sum(axis=1)).max()
    return cent, rad


def node_boxes(tree: ClusterTree, Xt: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Bounding box (lowest and highest coordinate per dimension) of every node."""
    d = Xt.shape[1]
    lo = np.zeros((tree.n_nodes, d))
    hi = np.zeros((tree.n_nodes, d))
    for a in range(tree.n_nodes):
        pts = Xt[tree.begin[a]:tree.begin[a] + tree.size[a]]
        if len(pts):
            lo[a], hi[a] = pts.min(axis=0), pts.max(axis=0)
    return lo, hi


BUDGET_NEIGHBOURS = 32


def knn_tree_order(Xt: np.ndarray, k: int) -> np.ndarray:
    """Indices (tree order) of the k nearest other points of every point, by brute force:
    squared distances summed over the coordinates in order, ties by index."""
    n = Xt.shape[0]
    k = min(k, n - 1)
    out = np.zeros((n, max(k, 0)), dtype=np.int64)
    if k <= 0:
        return out
    for i in range(n):
        d2 = _sq_dist_seq(Xt, Xt[i])
        d2[i] = np.inf
        order = np.lexsort((np.arange(n), d2))
        out[i] = order[:k]
    return out


def budget_near_leaves(tree: ClusterTree, Xt: np.ndarray, budget: float) -> set:
    """Near leaf pairs of GOFMM's budget admissibility (used by the paper for its H2-b
    structure, Section 4.1; the paper gives no algorithm): every point votes for the leaves
    of its BUDGET_NEIGHBOURS nearest neighbours; a leaf is near itself and the
    floor(budget * leaves) leaves with the most votes from its points (ties by leaf index);
    the relation is made symmetric."""
    nl, fl = tree.n_leaves, tree.first_leaf
    leaf_of = np.zeros(Xt.shape[0], dtype=np.int64)
    for i in range(nl):
        leaf_of[tree.begin[fl + i]:tree.begin[fl + i] + tree.size[fl + i]] = i
    nbr = knn_tree_order(Xt, BUDGET_NEIGHBOURS)
    keep = int(math.floor(budget * nl))
    near = set()
    for i in range(nl):
        near.add((i, i))
        pts = range(tree.begin[fl + i], tree.begin[fl + i] + tree.size[fl + i])
        votes = np.zeros(nl, dtype=np.int64)
        for p_ in pts:
            for q_ in nbr[p_]:
                votes[leaf_of[q_]] += 1
        votes[i] = 0
        cand = [j for j in np.lexsort((np.arange(nl), -votes)) if votes[j] > 0][:keep]
        for j in cand:
            near.add((i, int(j)))
            near.add((int(j), i))
    return near


def compute_interactions(tree: ClusterTree, Xt: np.ndarray, mode: str, eta: float = 2.0) -> Interactions:
    """Dual-tree traversal from (root, root). A pair of distinct nodes that is
    admissible is far; a pair of leaves that is not is near; otherwise the four
    child pairs are visited. ``mode`` is ``"hss"`` (distinct siblings are always
    admissible), ``"geometric"`` (centroid distance > eta * max radius), ``"tau"``
    (the paper's tau * dist(a, b) > diam(a) + diam(b) of Section 2.1, with tau =
    ``eta``, read on bounding boxes: dist = the Euclidean gap between the two boxes,
    diam = a box's diagonal; sums over the coordinates in order), ``"budget"``
    (GOFMM's budget, ``eta`` = the budget: a pair is far when no leaf pair below it is
    in ``budget_near_leaves``) or ``"none"`` (nothing is admissible: every leaf pair
    is near)."""
    if mode == "geometric":
        cent, rad = node_geometry(tree, Xt)
    if mode == "budget":
        fl = tree.first_leaf
        near_below = set()          # (a, b) with a near leaf pair below, on every level
        for i, j in budget_near_leaves(tree, Xt, eta):
            a, b = fl + i, fl + j
            while True:
                near_below.add((a, b))
                if a == 0:
                    break
                a, b = (a - 1) // 2, (b - 1) // 2
    if mode == "tau":
        lo, hi = node_boxes(tree, Xt)
        diam = np.zeros(tree.n_nodes)
        for k in range(Xt.shape[1]):
            ext = hi[:, k] - lo[:, k]
            diam = diam + ext * ext
        diam = np.sqrt(diam)

    def admissible(a: int, b: int) -> bool:
        if a == b:
            return False
        if mode == "hss":
            return True
        if mode == "none":
            return False
        if mode == "geometric":
            dist = float(np.sqrt(((cent[a] - cent[b]) ** 2).sum()))
            return dist > eta * max(rad[a], rad[b])
        if mode == "budget":
            return (a, b) not in near_below
        if mode == "tau":
            g2 = 0.0
            for k in range(Xt.shape[1]):
                gap = max(0.0, float(lo[b, k] - hi[a, k]), float(lo[a, k] - hi[b, k]))
                g2 = g2 + gap * gap
            return eta * math.sqrt(g2) > float(diam[a] + diam[b])
        raise ValueError(f"unknown admissibility {mode!r}")

    near, far = [], []
    frontier = [(0, 0)]
    for level in range(tree.levels + 1):
        nxt = []
        for a, b in frontier:
            if admissible(a, b):
                far.append((a, b))
            elif level == tree.levels:
                near.append((a, b))
            else:
                for ca in (2 * a + 1, 2 * a + 2):
                    for cb in (2 * b + 1, 2 * b + 2):
                        nxt.append((ca, cb))
        frontier = nxt
    near.sort()
    far.sort()
    return Interactions(near, far)


# --------------------------------------------------------------------------------------
# Interpolative decomposition (Section 2.1 footnote; Section 3.1 "Low-rank approximation")
# --------------------------------------------------------------------------------------

def row_id(A_rows_by_cols: np.ndarray, tol: float, max_rank: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Row interpolative decomposition of M (|R| x |C|): M ~= P M[skel, :].

    Column-pivoted QR of M^T: M^T[:, piv] = Q R. The rank k is the number of
    |R_jj| above tol * |R_11| (capped at max_rank); the skeleton rows are piv[:k]
    and the remaining rows are T^T times the skeleton rows, T = R_11^{-1} R_12.
    Returns (skel, P, diag) with P of shape |R| x k and diag = |R_jj|."""
    nr = A_rows_by_cols.shape[0]
    if nr == 0 or A_rows_by_cols.shape[1] == 0:
        return np.zeros(0, dtype=np.int64), np.zeros((nr, 0)), np.zeros(0)
    R, piv = sla.qr(A_rows_by_cols.T, mode="r", pivoting=True)
    diag = np.abs(np.diag(R))
    k = 0
    if diag.size and diag[0] > 0:
        k = int(np.count_nonzero(diag > tol * diag[0]))
    k = min(k, max_rank, nr)
    P = np.zeros((nr, k))
    if k > 0:
        T = sla.solve_triangular(R[:k, :k], R[:k, k:nr]) if k < nr else np.zeros((k, 0))
        P[piv[:k], :] = np.eye(k)
        P[piv[k:], :] = T.T
    return piv[:k].astype(np.int64), P, diag


# --------------------------------------------------------------------------------------
# Compression: the HMatrix (Section 3.1: CTree, HTree, sranks, submatrices D, V=U, B)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class HMatrix:
    """A compressed kernel matrix. Index sets and skeletons are tree-order point ids."""
    tree: ClusterTree
    inter: Interactions
    rank: np.ndarray                    # s_a per node (0: no basis or empty)
    skel: List[np.ndarray]              # S_a per node
    basis: List[Optional[np.ndarray]]   # P_a: leaf n_a x s_a, inner (s_l + s_r) x s_a
    near_blocks: List[np.ndarray]       # D_ij for inter.near, same order
    far_blocks: List[np.ndarray]        # B_ab for inter.far, same order
    kernel: str
    kernel_param: float

    # CSR views (leaf-local near lists, node-indexed far lists), sorted as in inter.*
    def near_csr(self) -> Tuple[np.ndarray, np.ndarray]:
        fl = self.tree.first_leaf
        ptr = np.zeros(self.tree.n_leaves + 1, dtype=np.int64)
        for i, _ in self.inter.near:
            ptr[i - fl + 1] += 1
        ptr = np.cumsum(ptr)
        idx = np.array([j - fl for _, j in self.inter.near], dtype=np.int32)
        return ptr, idx

    def far_csr(self) -> Tuple[np.ndarray, np.ndarray]:
        ptr = np.zeros(self.tree.n_nodes + 1, dtype=np.int64)
        for a, _ in self.inter.far:
            ptr[a + 1] += 1
        ptr = np.cumsum(ptr)
        idx = np.array([b for _, b in self.inter.far], dtype=np.int32)
        return ptr, idx


def far_columns(tree: ClusterTree, far_of: Dict[int, List[int]], a: int) -> np.ndarray:
    """Every tree-order point whose interaction with node a is approximated:
    the index sets of the far partners of a and of each of its ancestors."""
    parts = []
    g = a
    while True:
        for b in far_of.get(g, ()):
            parts.append(tree.index_set(b))
        if g == 0:
            break
        g = (g - 1) // 2
    if not parts:
        return np.zeros(0, dtype=np.int64)
    return np.unique(np.concatenate(parts))


def compress(X: np.ndarray, leaf_size: int, admissibility: str, kernel: str, kernel_param: float,
             tol: float, max_rank: int, sample_seed: int = 2, eta: float = 2.0,
             exact_columns: Optional[bool] = None, tree: str = "kd") -> HMatrix:
    """Build the HMatrix of K = k(X, X): tree, interactions, nested row IDs bottom-up,
    then the dense near blocks and the coupling blocks on the skeletons."""
    tree = build_cluster_tree(X, leaf_size, tree)
    Xt = X[tree.perm]
    inter = compute_interactions(tree, Xt, admissibility, eta)
    far_of: Dict[int, List[int]] = {}
    for a, b in inter.far:
        far_of.setdefault(a, []).append(b)

    # A node needs a basis iff it or an ancestor has a far partner.
    needs = np.zeros(tree.n_nodes, dtype=bool)
    for a in range(1, tree.n_nodes):
        needs[a] = (a in far_of) or needs[(a - 1) // 2]

    n = X.shape[0]
    if exact_columns is None:
        exact_columns = n <= EXACT_COLUMNS_MAX_N
    n_sample = max(4 * max_rank, 512)

    rank = np.zeros(tree.n_nodes, dtype=np.int32)
    skel: List[np.ndarray] = [np.zeros(0, dtype=np.int64) for _ in range(tree.n_nodes)]
    basis: List[Optional[np.ndarray]] = [None] * tree.n_nodes
    for level in range(tree.levels, 0, -1):
        for a in tree.nodes_at(level):
            if not needs[a]:
                continue
            if level == tree.levels:
                rows = tree.index_set(a)
            else:
                rows = np.concatenate([skel[2 * a + 1], skel[2 * a + 2]])
            cols = far_columns(tree, far_of, a)
            if not exact_columns and cols.size > n_sample:
                rng = np.random.default_rng([sample_seed, a])
                cols = np.sort(rng.choice(cols, size=n_sample, replace=False))
            M = kernel_matrix(kernel, kernel_param, Xt[rows], Xt[cols])
            sk, P, _ = row_id(M, tol, max_rank)
            skel[a] = rows[sk]
            basis[a] = P
            rank[a] = P.shape[1]

    near_blocks = [kernel_matrix(kernel, kernel_param, Xt[tree.index_set(i)], Xt[tree.index_set(j)])
                   for i, j in inter.near]
    far_blocks = [kernel_matrix(kernel, kernel_param, Xt[skel[a]], Xt[skel[b]]) for a, b in inter.far]
    return HMatrix(tree, inter, rank, skel, basis, near_blocks, far_blocks, kernel, kernel_param)


def compress_workload(w, **overrides) -> Tuple[HMatrix, np.ndarray]:
    """Compress the kernel matrix of a ``workloads.Workload``; returns (HMatrix, points)."""
    from workloads import make_points
    X = make_points(w)
    kw = dict(leaf_size=w.leaf_size, admissibility=w.admissibility, kernel=w.kernel,
              kernel_param=w.kernel_param, tol=w.tol, max_rank=w.max_rank,
              sample_seed=w.sample_seed, eta=w.eta, tree=w.tree)
    kw.update(overrides)
    return compress(X, **kw), X


# --------------------------------------------------------------------------------------
# Evaluation Y = K~ W (Section 2.1, "Evaluation")
# --------------------------------------------------------------------------------------

def evaluate(H: HMatrix, W: np.ndarray, leaves: Optional[Sequence[int]] = None) -> np.ndarray:
    """Y = K~ W in FP64, input point order, Y overwritten.

    Steps: gather W into tree order; near-field reduction over D; upward pass
    (leaf w_a = P_a^T W_a, inner w_a = P_a^T [w_l; w_r]); far-field reduction
    u_a = sum_b B_ab w_b; downward pass ([u_l; u_r] += P_a u_a, leaf Y_a += P_a u_a);
    scatter back to input order.

    With ``leaves`` (leaf node ids) only those leaves' rows are formed (the rest of Y
    is left at zero); the upward pass still runs over the whole tree."""
    tree = H.tree
    W = np.asarray(W, dtype=np.float64)
    if W.ndim != 2 or W.shape[0] != tree.perm.shape[0]:
        raise ValueError("W must be N x Q")
    q = W.shape[1]
    Wt = W[tree.perm]
    Yt = np.zeros_like(Wt)
    want = set(range(tree.first_leaf, tree.n_nodes)) if leaves is None else set(int(x) for x in leaves)

    # near field
    for (i, j), D in zip(H.inter.near, H.near_blocks):
        if i in want:
            Yt[tree.begin[i]:tree.begin[i] + tree.size[i]] += D @ Wt[tree.begin[j]:tree.begin[j] + tree.size[j]]

    # upward pass
    wt: List[Optional[np.ndarray]] = [None] * tree.n_nodes
    for level in range(tree.levels, 0, -1):
        for a in tree.nodes_at(level):
            if H.basis[a] is None:
                continue
            if level == tree.levels:
                src = Wt[tree.begin[a]:tree.begin[a] + tree.size[a]]
            else:
                src = np.vstack([_or_empty(wt[2 * a + 1], q), _or_empty(wt[2 * a + 2], q)])
            wt[a] = H.basis[a].T @ src

    # far field
    ut: List[Optional[np.ndarray]] = [None] * tree.n_nodes
    for a in range(tree.n_nodes):
        if H.basis[a] is not None:
            ut[a] = np.zeros((int(H.rank[a]), q))
    for (a, b), B in zip(H.inter.far, H.far_blocks):
        if B.size:
            ut[a] += B @ wt[b]

    # downward pass
    for level in range(1, tree.levels):
        for a in tree.nodes_at(level):
            if H.basis[a] is None:
                continue
            z = H.basis[a] @ ut[a]
            sl = int(H.rank[2 * a + 1])
            if sl:
                ut[2 * a + 1] += z[:sl]
            if z.shape[0] - sl:
                ut[2 * a + 2] += z[sl:]
    for a in tree.nodes_at(tree.levels):
        if H.basis[a] is not None and a in want:
            Yt[tree.begin[a]:tree.begin[a] + tree.size[a]] += H.basis[a] @ ut[a]

    Y = np.empty_like(Yt)
    Y[tree.perm] = Yt
    return Y


def _or_empty(x: Optional[np.ndarray], q: int) -> np.ndarray:
    return np.zeros((0, q)) if x is None else x


def assemble_dense(H: HMatrix) -> np.ndarray:
    """K~ as a dense N x N matrix in input order, assembled block by block from the
    factors: D_ij on near leaf pairs and Pbar_a B_ab Pbar_b^T on far pairs, where
    Pbar_a maps the skeleton of a to all of a's points through the nested bases."""
    tree = H.tree
    n = tree.perm.shape[0]
    pbar: List[Optional[np.ndarray]] = [None] * tree.n_nodes
    for level in range(tree.levels, 0, -1):
        for a in tree.nodes_at(level):
            if H.basis[a] is None:
                continue
            if level == tree.levels:
                pbar[a] = H.basis[a]
            else:
                l, r = 2 * a + 1, 2 * a + 2
                blk = sla.block_diag(_or_cols(pbar[l], tree.size[l], H.rank[l]),
                                     _or_cols(pbar[r], tree.size[r], H.rank[r]))
                pbar[a] = blk @ H.basis[a]
    Kt = np.zeros((n, n))
    for (i, j), D in zip(H.inter.near, H.near_blocks):
        Kt[tree.begin[i]:tree.begin[i] + tree.size[i], tree.begin[j]:tree.begin[j] + tree.size[j]] = D
    for (a, b), B in zip(H.inter.far, H.far_blocks):
        blk = pbar[a] @ B @ pbar[b].T
        Kt[tree.begin[a]:tree.begin[a] + tree.size[a], tree.begin[b]:tree.begin[b] + tree.size[b]] = blk
    out = np.empty_like(Kt)
    out[np.ix_(tree.perm, tree.perm)] = Kt
    return out


def _or_cols(p: Optional[np.ndarray], n: int, k: int) -> np.ndarray:
    return np.zeros((int(n), int(k))) if p is None else p


def overall_error(Y_approx: np.ndarray, Y_exact: np.ndarray) -> float:
    """eps_f = ||K~W - KW||_F / ||KW||_F (Section 5)."""
    return float(np.linalg.norm(Y_approx - Y_exact) / np.linalg.norm(Y_exact))


def dense_product(X: np.ndarray, kernel: str, kernel_param: float, W: np.ndarray, chunk: int = 2048) -> np.ndarray:
    """K W with the unapproximated kernel matrix, row chunk by row chunk."""
    out = np.empty((X.shape[0], W.shape[1]))
    for s in range(0, X.shape[0], chunk):
        out[s:s + chunk] = kernel_matrix(kernel, kernel_param, X[s:s + chunk], X) @ W
    return out


# --------------------------------------------------------------------------------------
# Sizes of the work (used by the bench's CPU baseline and by the roofline figures)
# --------------------------------------------------------------------------------------

def stored_entries(H: HMatrix) -> Dict[str, int]:
    """Number of stored FP64 entries per block family."""
    return {
        "near": int(sum(D.size for D in H.near_blocks)),
        "basis": int(sum(P.size for P in H.basis if P is not None)),
        "coupling": int(sum(B.size for B in H.far_blocks)),
    }
