"""Near blocks evaluated on the fly (HMAT_BUILD_NEAR_OTF): the FP64 near field computes
D_ij = K(x_i, x_j) from the points inside its kernel instead of reading stored blocks.

* GPU: bitwise the result of the same build with stored blocks (same entry formula, same
  products and sums), over tile shapes of every row class, the three kernels and q = 1;
  with every block near (no admissible pair) the product is the dense K W to 1e-13 (the
  fixed point that pins the path to the oracle's dense definition, 1/r with duplicated
  points included); autotuned shapes give bitwise the untuned result; the handle holds no
  near blocks.
* CPU: the flag is refused where it cannot hold (with the mixed copy, or on hmat_load,
  which has no points) before any device work.
"""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import desc_from_oracle, oracle_case, rhs
from workloads import WORKLOADS, make_points, reduced

torch = pytest.importorskip("torch")


def _params(w, **ov):
    p = dict(kernel=w.kernel, kernel_param=w.kernel_param, admissibility=w.admissibility, leaf_size=w.leaf_size,
             tol=w.tol, max_rank=w.max_rank, eta=w.eta, sample_seed=w.sample_seed)
    p.update(ov)
    return p


def _eval(h, W, mode=None):
    Wd = torch.from_numpy(W).cuda()
    Yd = torch.empty_like(Wd)
    hp.hmat_eval(h, Wd, Yd, W.shape[1], hp.HMAT_MODE_FP64 if mode is None else mode)
    assert hp.hmat_status_poll(h) == hp.HMAT_OK
    return Yd.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("base,n,q,ov", [
    ("hss_uniform3d_n2048", 2048, 16, ()),
    ("h2_gmm8d_n65536", 4096, 37, ()),
    ("h2_imq3d_n262144", 4000, 64, (("leaf_size", 40),)),      # 64- and 32-row near tiles
    ("h2_imq3d_n262144", 3000, 130, (("leaf_size", 20),)),     # 32- and 16-row near tiles
    ("h2_invdist3d_n262144", 3000, 1, ()),
])
def test_on_the_fly_is_bitwise_the_stored_result(base, n, q, ov):
    w = reduced(WORKLOADS[base], n)
    X = make_points(w)
    p = _params(w, **dict(ov))
    W = rhs(n, q, 41)
    h_s = hp.hmat_build(X, **p)
    h_o = hp.hmat_build(X, **p, flags=hp.HMAT_BUILD_NEAR_OTF)
    try:
        i_s, i_o = hp.hmat_info(h_s), hp.hmat_info(h_o)
        assert i_s["near_on_the_fly"] == 0 and i_o["near_on_the_fly"] == 1
        assert i_o["near_values"] == i_s["near_values"] and i_o["sum_rank"] == i_s["sum_rank"]
        # the handle holds the points (n x d doubles) instead of the near blocks
        saved = i_s["device_bytes"] - i_o["device_bytes"]
        assert saved >= 8 * i_s["near_values"] - 8 * n * X.shape[1], (saved, i_s["near_values"])
        Y_s, Y_o = _eval(h_s, W), _eval(h_o, W)
        assert np.array_equal(Y_s, Y_o)
    finally:
        hp.hmat_free(h_s)
        hp.hmat_free(h_o)


@pytest.mark.gpu
@pytest.mark.parametrize("kernel,param", [("gaussian", 0.5), ("imq", 0.1), ("invdist", 0.0)])
def test_on_the_fly_all_near_is_the_dense_product(kernel, param):
    rng = np.random.default_rng(52)
    X = rng.random((900, 3))
    X[450:460] = X[10:20]                      # duplicated points (1/r: K(x, x) = 0)
    W = rhs(900, 5, 53)
    h = hp.hmat_build(X, kernel=kernel, kernel_param=param, admissibility="none", leaf_size=64, tol=1e-6,
                      max_rank=64, flags=hp.HMAT_BUILD_NEAR_OTF)
    try:
        KW = hm.dense_product(X, kernel, param, W)
        err = hm.overall_error(_eval(h, W), KW)
        print(f"on-the-fly near field, every block near, {kernel}: relative error vs dense K W {err:.2e}")
        assert err <= 1e-13
    finally:
        hp.hmat_free(h)


@pytest.mark.gpu
def test_on_the_fly_autotuned_is_bitwise_untuned_and_mixed_is_refused():
    w = reduced(WORKLOADS["h2_gmm8d_n65536"], 4096)
    X = make_points(w)
    h = hp.hmat_build(X, **_params(w), flags=hp.HMAT_BUILD_NEAR_OTF)
    try:
        W = rhs(4096, 96, 61)
        Y0 = _eval(h, W)
        rep = hp.hmat_autotune(h, 96, hp.HMAT_MODE_FP64)
        assert rep["launches_tuned"] > 0
        assert np.array_equal(_eval(h, W), Y0)
        Wd = torch.from_numpy(W).cuda()
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_eval(h, Wd, torch.empty_like(Wd), 96, hp.HMAT_MODE_MIXED)
        assert ei.value.status == hp.HMAT_EUNSUPPORTED
    finally:
        hp.hmat_free(h)


def test_on_the_fly_flag_refused_with_mixed_and_on_load():
    X = np.random.default_rng(3).random((300, 3))
    with pytest.raises(hp.HmatError) as ei:
        hp.hmat_build(X, kernel="gaussian", kernel_param=0.5, admissibility="hss", leaf_size=32, tol=1e-6,
                      max_rank=32, flags=hp.HMAT_BUILD_NEAR_OTF | hp.HMAT_LOAD_MIXED)
    assert ei.value.status == hp.HMAT_EUNSUPPORTED
    _, H, _ = oracle_case("hss_uniform3d_n2048", 300, 3)
    with pytest.raises(hp.HmatError) as ei:
        hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_BUILD_NEAR_OTF)
    assert ei.value.status == hp.HMAT_EUNSUPPORTED
