"""The library's inspector (hmat_build: kd-tree, admissibility, nested ID on the
host; D and B evaluated on the GPU) against the oracle's compression.

The tree and the near/far lists are index work and must be identical to the
oracle's; the ranks come from a different pivoted QR and may differ by a pivot
or two, so the bases are checked by what they must achieve: eps_f against the
dense product K W (the oracle's unapproximated GEMM) of the same order as the
oracle's own compression, <= 100 tol with the rank cap lifted, and exact
(<= 1e-13) with tol = 0 and no cap.
"""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _params(w, **ov):
    p = dict(kernel=w.kernel, kernel_param=w.kernel_param, admissibility=w.admissibility, leaf_size=w.leaf_size,
             tol=w.tol, max_rank=w.max_rank, eta=w.eta, sample_seed=w.sample_seed)
    p.update(ov)
    return p


def _eval(h, W):
    Wd = torch.from_numpy(W).cuda()
    Yd = torch.empty_like(Wd)
    hp.hmat_eval(h, Wd, Yd, W.shape[1])
    assert hp.hmat_status_poll(h) == hp.HMAT_OK
    return Yd.cpu().numpy()


@pytest.mark.parametrize("base,n,ov", [
    ("hss_uniform3d_n2048", 2048, ()),
    ("h2_imq3d_n262144", 3000, ()),
    ("h2_gmm8d_n65536", 4096, ()),
    ("h2_imq3d_n262144", 4000, (("leaf_size", 40),)),
    ("h2_invdist3d_n262144", 3000, ()),
    ("h2_gmm8d_n65536", 4096, (("tree", "two_means"),)),                      # the paper's tree for d > 3
    ("h2_imq3d_n262144", 3000, (("admissibility", "tau"), ("eta", 3.0))),     # the paper's tau condition
    ("h2_gmm8d_n65536", 3000, (("tree", "two_means"), ("admissibility", "tau"), ("eta", 5.0))),
    ("h2_gmm8d_n65536", 2048, (("admissibility", "budget"), ("eta", 0.03))),     # the paper's H2-b
    ("h2_imq3d_n262144", 3000, (("admissibility", "budget"), ("eta", 0.1))),
])
def test_structure_identical_and_accuracy_comparable(base, n, ov):
    w, H, X = oracle_case(base, n, 8, **dict(ov))
    h = hp.hmat_build(X, **_params(w, **dict(ov)))
    try:
        st = hp.hmat_structure(h)
        near_ptr, near_idx = H.near_csr()
        far_ptr, far_idx = H.far_csr()
        assert np.array_equal(st["perm"], H.tree.perm)
        assert np.array_equal(st["near_ptr"], near_ptr) and np.array_equal(st["near_idx"], near_idx)
        assert np.array_equal(st["far_ptr"], far_ptr) and np.array_equal(st["far_idx"], far_idx)
        assert np.array_equal(st["rank"] > 0, H.rank > 0)
        assert np.abs(st["rank"].astype(int) - H.rank).max() <= 3
        W = rhs(w.n, 8, 21)
        KW = hm.dense_product(X, w.kernel, w.kernel_param, W)
        e_lib = hm.overall_error(_eval(h, W), KW)
        e_orc = hm.overall_error(hm.evaluate(H, W), KW)
        assert e_lib <= 3 * e_orc + 1e-12, (e_lib, e_orc)
    finally:
        hp.hmat_free(h)


@pytest.mark.parametrize("base,n", [("hss_uniform3d_n2048", 2048), ("h2_imq3d_n262144", 4096),
                                    ("h2_invdist3d_n262144", 4096)])
def test_error_order_tol_uncapped(base, n):
    w, _, X = oracle_case(base, n, 8)
    W = rhs(w.n, 8, 22)
    KW = hm.dense_product(X, w.kernel, w.kernel_param, W)
    for tol in (1e-4, 1e-7):
        h = hp.hmat_build(X, **_params(w, tol=tol, max_rank=10 ** 6))
        try:
            assert hm.overall_error(_eval(h, W), KW) <= 100 * tol
        finally:
            hp.hmat_free(h)


def test_full_rank_hss_is_exact():
    w, _, X = oracle_case("hss_uniform3d_n2048", 1024, 4)
    h = hp.hmat_build(X, **_params(w, tol=0.0, max_rank=10 ** 6))
    try:
        W = rhs(w.n, 4, 23)
        KW = hm.dense_product(X, w.kernel, w.kernel_param, W)
        assert hm.overall_error(_eval(h, W), KW) <= 1e-13
    finally:
        hp.hmat_free(h)


def test_build_rejects_bad_parameters():
    X = np.random.default_rng(0).random((100, 3))
    base = dict(kernel="gaussian", kernel_param=0.5, admissibility="hss", leaf_size=16, tol=1e-6, max_rank=32)
    for bad in (dict(leaf_size=1), dict(max_rank=0), dict(kernel_param=0.0), dict(tol=-1.0)):
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_build(X, **{**base, **bad})
        assert ei.value.status == hp.HMAT_EINVAL
    Xn = X.copy()
    Xn[3, 1] = np.nan
    with pytest.raises(hp.HmatError):
        hp.hmat_build(Xn, **base)


def test_invdist_blocks_zero_for_coincident_points():
    """The 1/r kernel's diagonal convention on the device: duplicated points interact with 0,
    so with nothing far the library reproduces the oracle's dense product exactly."""
    rng = np.random.default_rng(31)
    X = rng.random((700, 3))
    X[350:360] = X[10:20]                                   # ten duplicated points
    W = rhs(700, 3, 32)
    h = hp.hmat_build(X, kernel="invdist", kernel_param=0.0, admissibility="none", leaf_size=64, tol=1e-6,
                      max_rank=64, eta=2.0)
    try:
        KW = hm.dense_product(X, "invdist", 0.0, W)
        assert np.isfinite(KW).all()
        assert hm.overall_error(_eval(h, W), KW) <= 1e-13
    finally:
        hp.hmat_free(h)


def test_plan_reuse_equals_fresh_builds():
    """Inspector reuse (Section 3.2): one plan (tree + lists) recompressed for other kernels and
    tolerances gives bitwise the HMatrix of a fresh hmat_build with the same parameters."""
    w, _, X = oracle_case("h2_imq3d_n262144", 3000, 8)
    plan = hp.hmat_plan_create(X, admissibility=w.admissibility, leaf_size=w.leaf_size, eta=w.eta)
    try:
        W = rhs(w.n, 5, 41)
        for kernel, param, tol in (("imq", 0.1, 1e-7), ("gaussian", 0.3, 1e-5), ("invdist", 0.0, 1e-6)):
            h1 = hp.hmat_plan_build(plan, kernel, param, tol, 256, sample_seed=w.sample_seed)
            h2 = hp.hmat_build(X, **_params(w, kernel=kernel, kernel_param=param, tol=tol, max_rank=256))
            try:
                s1, s2 = hp.hmat_structure(h1), hp.hmat_structure(h2)
                for k in s1:
                    assert np.array_equal(s1[k], s2[k]), (kernel, k)
                assert np.array_equal(_eval(h1, W), _eval(h2, W)), kernel
                KW = hm.dense_product(X, kernel, param, W)
                assert hm.overall_error(_eval(h1, W), KW) <= max(100 * tol, 1e-12)
            finally:
                hp.hmat_free(h1)
                hp.hmat_free(h2)
    finally:
        hp.hmat_plan_free(plan)


def test_plan_rejects_bad_parameters():
    w, _, X = oracle_case("hss_uniform3d_n2048", 1000, 1)
    with pytest.raises(hp.HmatError):
        hp.hmat_plan_create(X, admissibility=w.admissibility, leaf_size=1)
    plan = hp.hmat_plan_create(X, admissibility=w.admissibility, leaf_size=w.leaf_size)
    try:
        for kernel, param, tol, rank in (("gaussian", 0.0, 1e-6, 64), ("imq", 0.1, -1.0, 64), ("imq", 0.1, 1e-6, 0)):
            with pytest.raises(hp.HmatError) as ei:
                hp.hmat_plan_build(plan, kernel, param, tol, rank)
            assert ei.value.status == hp.HMAT_EINVAL
    finally:
        hp.hmat_plan_free(plan)


@pytest.mark.parametrize("base,n,ov", [
    ("hss_uniform3d_n2048", 2048, ()),
    ("h2_imq3d_n262144", 3000, ()),
    ("h2_gmm8d_n65536", 4096, ()),
    ("h2_invdist3d_n262144", 3000, ()),
    ("h2_imq3d_n262144", 5000, (("leaf_size", 256),)),
])
def test_gpu_row_ids_match_host_row_ids(base, n, ov):
    """HMAT_BUILD_ID_GPU runs the same pivoted QR per node on the GPU (sums in another order):
    the same ranks and skeletons except where two pivot candidates tie within rounding, and
    the same accuracy against the dense product."""
    w, H, X = oracle_case(base, n, 8, **dict(ov))
    plan = hp.hmat_plan_create(X, admissibility=w.admissibility, leaf_size=w.leaf_size, eta=w.eta)
    try:
        args = (w.kernel, w.kernel_param, w.tol, w.max_rank)
        h_host = hp.hmat_plan_build(plan, *args, sample_seed=w.sample_seed)
        h_gpu = hp.hmat_plan_build(plan, *args, sample_seed=w.sample_seed, flags=hp.HMAT_BUILD_ID_GPU)
        try:
            r_host = hp.hmat_structure(h_host)["rank"].astype(int)
            r_gpu = hp.hmat_structure(h_gpu)["rank"].astype(int)
            assert np.abs(r_host - r_gpu).max() <= 1
            assert np.mean(r_host == r_gpu) >= 0.95
            W = rhs(w.n, 8, 51)
            KW = hm.dense_product(X, w.kernel, w.kernel_param, W)
            e_host = hm.overall_error(_eval(h_host, W), KW)
            e_gpu = hm.overall_error(_eval(h_gpu, W), KW)
            assert e_gpu <= 1.5 * e_host + 1e-13, (e_gpu, e_host)
            e_orc = hm.overall_error(hm.evaluate(H, W), KW)
            assert e_gpu <= 3 * e_orc + 1e-12, (e_gpu, e_orc)
        finally:
            hp.hmat_free(h_host)
            hp.hmat_free(h_gpu)
    finally:
        hp.hmat_plan_free(plan)


def test_gpu_row_ids_full_rank_is_exact():
    w, _, X = oracle_case("hss_uniform3d_n2048", 1024, 4)
    h = hp.hmat_build(X, **_params(w, tol=0.0, max_rank=10 ** 6), flags=hp.HMAT_BUILD_ID_GPU)
    try:
        W = rhs(w.n, 4, 52)
        KW = hm.dense_product(X, w.kernel, w.kernel_param, W)
        assert hm.overall_error(_eval(h, W), KW) <= 1e-13
    finally:
        hp.hmat_free(h)


@pytest.mark.gpu
@pytest.mark.parametrize("n_rows,n_cols,tol,rank_expected", [(40, 60, 10 ** -7.5, 8), (64, 200, 10 ** -11.5, 12),
                                                             (30, 30, 0.0, 30)])
def test_gpu_row_id_returns_the_oracle_skeleton_on_a_separated_spectrum(n_rows, n_cols, tol, rank_expected):
    """A matrix whose rows have geometrically decaying scales (a factor 10 apart, in a
    shuffled order) over a generic Gaussian matrix has unambiguous pivots: each step of the
    column-pivoted QR picks the row of the next scale. The GPU row ID must return exactly
    the oracle's skeleton (in pivot order) and rank, and its interpolation matrix P within
    1e-9 of the oracle's."""
    rng = np.random.default_rng(n_rows)
    order = rng.permutation(n_rows)
    scales = 10.0 ** -np.arange(n_rows, dtype=np.float64)
    M = (scales[np.argsort(order)][:, None]) * rng.standard_normal((n_rows, n_cols))
    skel, P, diag = hm.row_id(M, tol, 10 ** 6)
    assert len(skel) == rank_expected
    # the pivots follow the scales: the oracle's skeleton is the rows in decreasing scale
    assert list(skel) == list(np.argsort(-scales[np.argsort(order)])[:rank_expected])
    k, piv, T = hp.hmat_selftest_row_id(M, tol, 10 ** 6)
    assert k == rank_expected
    assert list(piv[:k]) == list(skel)
    Pg = np.zeros((n_rows, k))
    Pg[piv[:k], :] = np.eye(k)
    Pg[piv[k:], :] = T.T
    assert np.abs(Pg - P).max() <= 1e-9 * max(1.0, np.abs(P).max())
    # the rank cap stops both at the same pivot
    skel_c, _, _ = hm.row_id(M, tol, 5)
    kc, piv_c, _ = hp.hmat_selftest_row_id(M, tol, 5)
    assert kc == len(skel_c) == min(5, rank_expected) and list(piv_c[:kc]) == list(skel_c)
