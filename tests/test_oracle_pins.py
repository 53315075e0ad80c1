"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-worked
golden fixtures (tests/golden/), closed forms, the dense unapproximated product
K W (a textbook GEMM), invariants of the method (linearity, symmetry, column
independence, covering of every leaf pair), and error bounds of the
interpolative decomposition. A dropped term, a wrong sign or index or a
transposed operand anywhere in the evaluator makes eps_f against K W or the
symmetry check fail.
"""
import json
import os

import math

import numpy as np
import pytest

from oracle import hmatrix as hm
from workloads import WORKLOADS, make_points, normal_rhs, reduced, uniform_points, gmm_points

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- kernel (Section 1)

def test_kernel_closed_forms():
    x = np.zeros((1, 3))
    y = np.array([[0.5, 0.0, 0.0]])
    # Gaussian with h = 0.5 at distance h: exp(-1/2)
    assert hm.kernel_matrix("gaussian", 0.5, x, y)[0, 0] == pytest.approx(np.exp(-0.5), rel=1e-15)
    assert hm.kernel_matrix("gaussian", 0.5, x, x)[0, 0] == 1.0
    # inverse multiquadric 1/sqrt(r^2 + c^2): at r = 0 -> 1/c; at r = 0.5, c = 0.1 -> 1/sqrt(0.26)
    assert hm.kernel_matrix("imq", 0.1, x, x)[0, 0] == pytest.approx(10.0, rel=1e-15)
    assert hm.kernel_matrix("imq", 0.1, x, y)[0, 0] == pytest.approx(1 / np.sqrt(0.26), rel=1e-15)
    # 1/r (Section 4.1): 2 at r = 0.5, 0 for coincident points (the paper leaves k(x, x) open)
    assert hm.kernel_matrix("invdist", 0.0, x, y)[0, 0] == 2.0
    assert hm.kernel_matrix("invdist", 0.0, x, x)[0, 0] == 0.0


def test_invdist_block_matches_pairwise_loop():
    rng = np.random.default_rng(12)
    X = rng.random((7, 3))
    X[4] = X[1]                                              # a duplicated point: its pair is 0 too
    K = hm.kernel_matrix("invdist", 0.0, X, X)
    for i in range(7):
        for j in range(7):
            r = math.sqrt(sum((X[i, k] - X[j, k]) ** 2 for k in range(3)))
            assert K[i, j] == (0.0 if r == 0.0 else pytest.approx(1.0 / r, rel=1e-15))


# ---------------------------------------------------------------- cluster tree (Section 3.1)

@pytest.mark.parametrize("name", ["kdtree_2d_8pts.json", "kdtree_ties_4pts.json"])
def test_kdtree_golden(name):
    g = _golden(name)
    t = hm.build_cluster_tree(np.array(g["points"], dtype=float), g["leaf_size"])
    assert t.levels == g["levels"]
    assert t.perm.tolist() == g["perm"]
    assert t.begin.tolist() == g["begin"]
    assert t.size.tolist() == g["size"]


@pytest.mark.parametrize("n,d,m", [(2048, 3, 64), (1000, 2, 64), (777, 8, 33), (130, 3, 128), (64, 3, 64)])
def test_kdtree_invariants(n, d, m):
    X = uniform_points(n, d, 7)
    t = hm.build_cluster_tree(X, m)
    assert sorted(t.perm.tolist()) == list(range(n))             # bijection
    assert t.levels == hm.tree_depth(n, m)
    assert (t.size[t.first_leaf:] <= m).all() and (t.size[t.first_leaf:] >= 1).all()
    for level in range(t.levels + 1):
        s = t.size[list(t.nodes_at(level))]
        assert s.max() - s.min() <= 1                               # balanced per level
    Xt = X[t.perm]
    for a in range(t.first_leaf):
        l, r = 2 * a + 1, 2 * a + 2
        assert t.begin[l] == t.begin[a] and t.begin[r] == t.begin[a] + t.size[l]
        assert t.size[l] == t.size[a] // 2 and t.size[l] + t.size[r] == t.size[a]
        pts = Xt[t.begin[a]:t.begin[a] + t.size[a]]
        dim = int(np.argmax(pts.max(0) - pts.min(0)))
        assert Xt[t.index_set(l), dim].max() <= Xt[t.index_set(r), dim].min()   # median split


# ---------------------------------------------------------------- interactions (Section 2.1)

def test_admissibility_golden_line():
    g = _golden("admissibility_line_16pts.json")
    X = np.array(g["points"], dtype=float)
    t = hm.build_cluster_tree(X, g["leaf_size"])
    assert t.perm.tolist() == list(range(16))
    geo = hm.compute_interactions(t, X[t.perm], "geometric", g["eta"])
    assert sorted(map(tuple, g["geometric_near"])) == geo.near
    assert sorted(map(tuple, g["geometric_far"])) == geo.far
    hss = hm.compute_interactions(t, X[t.perm], "hss")
    assert sorted(map(tuple, g["hss_near"])) == hss.near
    assert sorted(map(tuple, g["hss_far"])) == hss.far


def test_tau_admissibility_golden_line():
    g = _golden("admissibility_tau_line_16pts.json")
    X = np.array(g["points"], dtype=float)
    t = hm.build_cluster_tree(X, g["leaf_size"])
    inter = hm.compute_interactions(t, X[t.perm], "tau", g["tau"])
    assert sorted(map(tuple, g["near"])) == inter.near
    assert sorted(map(tuple, g["far"])) == inter.far


def test_budget_admissibility_golden_line():
    g = _golden("admissibility_budget_line_16pts.json")
    X = np.array(g["points"], dtype=float)
    t = hm.build_cluster_tree(X, g["leaf_size"])
    inter = hm.compute_interactions(t, X[t.perm], "budget", g["budget"])
    assert sorted(map(tuple, g["near"])) == inter.near
    assert sorted(map(tuple, g["far"])) == inter.far


def test_budget_zero_is_hss():
    """Section 4.1: budget 0 gives the HSS structure."""
    X = uniform_points(1000, 3, 13)
    t = hm.build_cluster_tree(X, 32)
    b = hm.compute_interactions(t, X[t.perm], "budget", 0.0)
    h = hm.compute_interactions(t, X[t.perm], "hss")
    assert b.near == h.near and b.far == h.far


def test_knn_brute_force_small():
    X = np.array([[0.0], [1.0], [3.0], [3.5], [10.0]])
    nbr = hm.knn_tree_order(X, 2)
    assert nbr.tolist() == [[1, 2], [0, 2], [3, 1], [2, 1], [3, 2]]


def test_two_means_golden_splits():
    for case in _golden("two_means_splits.json")["cases"]:
        X = np.array(case["points"], dtype=float)
        t = hm.build_cluster_tree(X, case["leaf_size"], tree="two_means")
        assert t.perm.tolist() == case["perm"], case["derivation"]
        if "sizes" in case:
            assert t.size.tolist() == case["sizes"]
        if "kd_perm" in case:
            assert hm.build_cluster_tree(X, case["leaf_size"]).perm.tolist() == case["kd_perm"]


def _box_gap_and_diams(t, Xt, a, b):
    """Bounding-box gap and diagonals of two nodes, by plain loops over points and coordinates."""
    def box(x):
        pts = [Xt[i] for i in range(t.begin[x], t.begin[x] + t.size[x])]
        return ([min(p[k] for p in pts) for k in range(Xt.shape[1])], [max(p[k] for p in pts) for k in range(Xt.shape[1])])
    (la, ha), (lb, hb) = box(a), box(b)
    gap = math.sqrt(sum(max(0.0, lb[k] - ha[k], la[k] - hb[k]) ** 2 for k in range(Xt.shape[1])))
    da = math.sqrt(sum((ha[k] - la[k]) ** 2 for k in range(Xt.shape[1])))
    db = math.sqrt(sum((hb[k] - lb[k]) ** 2 for k in range(Xt.shape[1])))
    return gap, da, db


@pytest.mark.parametrize("tau", [3.0, 5.0, 10.0])
def test_tau_far_pairs_admissible_and_minimal(tau):
    """Every far pair meets tau * gap > diam_a + diam_b and its parent pair does not (the traversal
    stops at the first admissible level), checked with plain loops."""
    w = reduced(WORKLOADS["h2_invdist3d_n262144"], 700, q=1)
    X = make_points(w)
    t = hm.build_cluster_tree(X, 40)
    Xt = X[t.perm]
    inter = hm.compute_interactions(t, Xt, "tau", tau)
    assert inter.far
    for a, b in inter.far:
        gap, da, db = _box_gap_and_diams(t, Xt, a, b)
        assert tau * gap > da + db
        pa, pb = (a - 1) // 2, (b - 1) // 2
        if a > 0 and pa != pb:
            gap, da, db = _box_gap_and_diams(t, Xt, pa, pb)
            assert not tau * gap > da + db


def _covering_counts(t, inter):
    """How many times each leaf pair is covered by a near pair or a far pair of ancestors."""
    fl, nl = t.first_leaf, t.n_leaves
    cover = np.zeros((nl, nl), dtype=int)
    for i, j in inter.near:
        cover[i - fl, j - fl] += 1
    for a, b in inter.far:
        la = [x - fl for x in range(t.n_nodes) if _is_desc(x, a, t)]
        lb = [x - fl for x in range(t.n_nodes) if _is_desc(x, b, t)]
        cover[np.ix_(la, lb)] += 1
    return cover


def _is_desc(x, a, t):
    if x < t.first_leaf:
        return False
    while x > a:
        x = (x - 1) // 2
    return x == a


@pytest.mark.parametrize("mode,X,tree,eta", [
    ("hss", uniform_points(1000, 3, 3), "kd", 2.0),
    ("geometric", uniform_points(2048, 3, 4), "kd", 2.0),
    ("geometric", uniform_points(1500, 2, 5), "kd", 2.0),
    ("geometric", gmm_points(2048, 8, 10, 6), "kd", 2.0),
    ("geometric", gmm_points(2048, 8, 10, 6), "two_means", 2.0),
    ("tau", uniform_points(2048, 3, 4), "kd", 3.0),
    ("tau", gmm_points(1500, 8, 10, 7), "two_means", 5.0),
    ("budget", uniform_points(1024, 3, 8), "kd", 0.1),
    ("budget", gmm_points(1024, 8, 10, 9), "two_means", 0.05),
])
def test_interactions_symmetric_and_covering(mode, X, tree, eta):
    t = hm.build_cluster_tree(X, 32, tree=tree)
    if tree == "two_means":                                   # a perfect, balanced tree of every point
        assert sorted(t.perm.tolist()) == list(range(X.shape[0]))
        for a in range(t.first_leaf):
            assert t.size[2 * a + 1] == t.size[a] // 2 and t.begin[2 * a + 2] == t.begin[a] + t.size[a] // 2
    inter = hm.compute_interactions(t, X[t.perm], mode, eta)
    assert set(inter.near) == {(j, i) for i, j in inter.near}
    assert set(inter.far) == {(b, a) for a, b in inter.far}
    for a, b in inter.far:
        assert t.level_of(a) == t.level_of(b) and a != b
    cover = _covering_counts(t, inter)
    assert (cover == 1).all()


# ---------------------------------------------------------------- interpolative decomposition

def test_row_id_exact_low_rank():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((40, 7)) @ rng.standard_normal((7, 90))
    sk, P, diag = hm.row_id(A, 1e-12, 1000)
    assert len(sk) == 7
    assert np.linalg.norm(A - P @ A[sk]) <= 1e-12 * np.linalg.norm(A)
    assert np.allclose(P[sk], np.eye(7))                    # skeleton rows interpolate themselves


def test_row_id_full_rank_is_permutation():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((20, 50))
    sk, P, _ = hm.row_id(A, 0.0, 1000)
    assert sorted(sk.tolist()) == list(range(20))
    assert np.array_equal(np.sort(P, axis=1)[:, -1], np.ones(20)) and np.count_nonzero(P) == 20
    assert np.linalg.norm(A - P @ A[sk]) == 0.0


def test_row_id_truncation_bound():
    # ||A - P A(S,:)||_2 <= |R_{k+1,k+1}| * sqrt(1 + ||T||^2) * sqrt(k (n - k) + 1) (pivoted-QR ID bound)
    rng = np.random.default_rng(13)
    U, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    V, _ = np.linalg.qr(rng.standard_normal((200, 60)))
    A = U @ np.diag(10.0 ** -np.arange(60) * 0.25) @ V.T
    sk, P, diag = hm.row_id(A, 1e-6, 1000)
    k = len(sk)
    assert 0 < k < 60 and diag[k] <= 1e-6 * diag[0] < diag[k - 1]
    err = np.linalg.norm(A - P @ A[sk], 2)
    T_norm = np.linalg.norm(P, 2)
    assert err <= diag[k] * np.sqrt(1 + T_norm ** 2) * np.sqrt(k * (60 - k) + 1)
    sk2, P2, _ = hm.row_id(A, 1e-6, 5)
    assert len(sk2) == 5                                     # the cap binds


# ---------------------------------------------------------------- evaluation (Section 2.1)

def _small(w, **kw):
    H, X = hm.compress_workload(w, **kw)
    return H, X


@pytest.mark.parametrize("base", ["h2_gmm8d_n65536", "h2_invdist3d_n262144"])
def test_all_near_equals_dense_product(base):
    w = reduced(WORKLOADS[base], 1200, q=5)
    H, X = _small(w, admissibility="none")
    assert len(H.inter.far) == 0
    W = normal_rhs(w.n, w.q, 3)
    KW = hm.dense_product(X, w.kernel, w.kernel_param, W)
    assert hm.overall_error(hm.evaluate(H, W), KW) <= 1e-13


def test_hss_full_rank_reproduces_K():
    w = reduced(WORKLOADS["hss_uniform3d_n2048"], 1024, q=4)
    H, X = _small(w, tol=0.0, max_rank=10 ** 6)
    W = normal_rhs(w.n, w.q, 4)
    KW = hm.dense_product(X, w.kernel, w.kernel_param, W)
    assert hm.overall_error(hm.evaluate(H, W), KW) <= 1e-13


@pytest.mark.parametrize("base,n,ov", [("hss_uniform3d_n2048", 2048, {}), ("h2_imq3d_n262144", 4096, {}),
                                       ("h2_gmm8d_n65536", 4096, {}), ("h2_invdist3d_n262144", 4096, {}),
                                       ("h2_gmm8d_n65536", 4096, {"tree": "two_means"}),
                                       ("h2_imq3d_n262144", 4096, {"admissibility": "tau", "eta": 3.0}),
                                       ("h2_gmm8d_n65536", 2048, {"admissibility": "budget", "eta": 0.03})])
def test_error_is_order_tol(base, n, ov):
    w = reduced(WORKLOADS[base], n, q=8, **ov)
    X = make_points(w)
    W = normal_rhs(w.n, w.q, 5)
    KW = hm.dense_product(X, w.kernel, w.kernel_param, W)
    errs = []
    for tol in (1e-3, 1e-5, 1e-7):
        H = hm.compress(X, w.leaf_size, w.admissibility, w.kernel, w.kernel_param, tol, 10 ** 6, eta=w.eta,
                        tree=w.tree)
        e = hm.overall_error(hm.evaluate(H, W), KW)
        assert e <= 100 * tol, (tol, e)
        errs.append(e)
    assert errs[0] >= errs[1] >= errs[2]


def test_linearity_and_column_independence():
    w = reduced(WORKLOADS["h2_imq3d_n262144"], 3000, q=6)
    H, _ = _small(w)
    W1 = normal_rhs(w.n, w.q, 6)
    W2 = normal_rhs(w.n, w.q, 7)
    Y1, Y2 = hm.evaluate(H, W1), hm.evaluate(H, W2)
    Y12 = hm.evaluate(H, 2.5 * W1 - 0.75 * W2)
    assert np.linalg.norm(Y12 - (2.5 * Y1 - 0.75 * Y2)) <= 1e-14 * np.linalg.norm(Y12)
    for q in (0, 3, 5):
        yq = hm.evaluate(H, W1[:, q:q + 1])
        assert np.linalg.norm(yq[:, 0] - Y1[:, q]) <= 1e-15 * np.linalg.norm(Y1[:, q])


@pytest.mark.parametrize("base", ["hss_uniform3d_n2048", "h2_imq3d_n262144", "h2_invdist3d_n262144"])
def test_symmetry(base):
    # U = V and B_ba = B_ab^T, D_ji = D_ij^T, so K~ is symmetric: W1^T (K~ W2) = W2^T (K~ W1)
    w = reduced(WORKLOADS[base], 2048, q=3)
    H, _ = _small(w)
    W1 = normal_rhs(w.n, 3, 8)
    W2 = normal_rhs(w.n, 3, 9)
    G12 = W1.T @ hm.evaluate(H, W2)
    G21 = W2.T @ hm.evaluate(H, W1)
    assert np.linalg.norm(G12 - G21.T) <= 1e-13 * np.linalg.norm(G12)


def test_dense_assembly_matches_nested_evaluation():
    w = reduced(WORKLOADS["h2_imq3d_n262144"], 2500, q=4)
    H, _ = _small(w)
    W = normal_rhs(w.n, w.q, 10)
    Kt = hm.assemble_dense(H)
    assert np.linalg.norm(Kt - Kt.T) <= 1e-13 * np.linalg.norm(Kt)
    Y = hm.evaluate(H, W)
    assert np.linalg.norm(Kt @ W - Y) <= 1e-13 * np.linalg.norm(Y)


def test_leaf_subset_rows_match_full():
    w = reduced(WORKLOADS["h2_imq3d_n262144"], 2100, q=3)
    H, _ = _small(w)
    W = normal_rhs(w.n, w.q, 11)
    Y = hm.evaluate(H, W)
    t = H.tree
    pick = [t.first_leaf, t.first_leaf + 3, t.n_nodes - 1]
    Ys = hm.evaluate(H, W, leaves=pick)
    rows = np.concatenate([t.perm[t.index_set(a)] for a in pick])
    assert np.array_equal(Ys[rows], Y[rows])


def test_rank_cap_and_basis_shapes():
    w = WORKLOADS["hss_uniform3d_n2048"]
    H, _ = _small(w)
    t = H.tree
    assert H.rank[0] == 0 and H.basis[0] is None
    for a in range(1, t.n_nodes):
        P = H.basis[a]
        assert P is not None and P.shape[1] == H.rank[a] <= w.max_rank
        rows = t.size[a] if a >= t.first_leaf else H.rank[2 * a + 1] + H.rank[2 * a + 2]
        assert P.shape[0] == rows
