"""hmat_autotune: tuned tile shapes give bitwise the untuned result (GPU).

Every candidate shape sums each output over the same depth order, so an evaluation
after tuning must equal the one before it bit for bit, in both modes; the FP64
result is also held to the oracle (relative Frobenius error <= 1e-12).
"""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _eval(h, W, mode):
    Wd = torch.from_numpy(W).cuda()
    Yd = torch.full_like(Wd, float("nan"))
    hp.hmat_eval(h, Wd, Yd, W.shape[1], mode)
    assert hp.hmat_status_poll(h) == hp.HMAT_OK
    return Yd.cpu().numpy()


@pytest.mark.parametrize("q", [1, 2, 6, 17, 130])
def test_fp64_autotune_is_bitwise_neutral(q):
    w, H, _ = oracle_case("h2_imq3d_n262144", 3000, 64)
    W = rhs(w.n, q, 40 + q)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        Y0 = _eval(h, W, hp.HMAT_MODE_FP64)
        rep = hp.hmat_autotune(h, q, hp.HMAT_MODE_FP64)
        assert rep["q"] == q and rep["launches_tuned"] > 0
        assert 0 < rep["tuned_ms"] <= rep["default_ms"]
        assert rep["near_cols"] in (1, 2, 4, 8, 16, 32, 64)
        Y1 = _eval(h, W, hp.HMAT_MODE_FP64)
        assert np.array_equal(Y0, Y1)
        Yref = hm.evaluate(H, W)
        assert np.linalg.norm(Y1 - Yref) <= 1e-12 * np.linalg.norm(Yref)
        # tuning another q leaves this one's choice (and result) alone
        hp.hmat_autotune(h, q + 3, hp.HMAT_MODE_FP64)
        assert np.array_equal(Y0, _eval(h, W, hp.HMAT_MODE_FP64))
    finally:
        hp.hmat_free(h)


@pytest.mark.parametrize("base,n,q", [("h2_imq3d_n262144", 3000, 17), ("h2_gmm8d_n65536", 4096, 130),
                                      ("hss_uniform3d_n2048", 2048, 256)])
def test_mixed_autotune_is_bitwise_neutral(base, n, q):
    w, H, _ = oracle_case(base, n, 64)
    W = rhs(w.n, q, 70 + q)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        Y0 = _eval(h, W, hp.HMAT_MODE_MIXED)
        rep = hp.hmat_autotune(h, q, hp.HMAT_MODE_MIXED)
        # the near-field width, then (with a far field) the persistent far chain's grid on whole evaluations
        assert rep["launches_tuned"] in (1, 2) and rep["near_cols"] % 16 == 0 and 16 <= rep["near_cols"] <= 128
        assert rep["chain_grid"] >= 0
        assert 0 < rep["tuned_ms"] <= rep["default_ms"]
        Y1 = _eval(h, W, hp.HMAT_MODE_MIXED)
        assert np.array_equal(Y0, Y1)
        Yref = hm.evaluate(H, W)
        assert np.linalg.norm(Y1 - Yref) <= 1e-6 * np.linalg.norm(Yref)
    finally:
        hp.hmat_free(h)


def test_autotune_rejects_bad_calls():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        for q, mode, status in ((0, hp.HMAT_MODE_FP64, hp.HMAT_EINVAL), (4, 7, hp.HMAT_EUNSUPPORTED),
                                (4, hp.HMAT_MODE_MIXED, hp.HMAT_EUNSUPPORTED)):
            with pytest.raises(hp.HmatError) as ei:
                hp.hmat_autotune(h, q, mode)
            assert ei.value.status == status
    finally:
        hp.hmat_free(h)
