"""GPU parity of the FP64 path (HMAT_MODE_FP64) against the FP64 oracle.

Every case loads the oracle's HMatrix through the C ABI, evaluates on the GPU
and compares element by element with the oracle's evaluator on the same seeded
W: the bar is the FP64 target, relative Frobenius error <= 1e-12 and every
element within 1e-12 of the largest |Y| (reordered FP64 sums differ from the
oracle's only by rounding).
"""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _gpu_eval(H, W, mode=hp.HMAT_MODE_FP64, handle=None):
    own = handle is None
    if own:
        handle = hp.hmat_load(**desc_from_oracle(H))
    try:
        Wd = torch.from_numpy(W).cuda()
        Yd = torch.full_like(Wd, float("nan"))
        hp.hmat_eval(handle, Wd, Yd, W.shape[1], mode)
        assert hp.hmat_status_poll(handle) == hp.HMAT_OK
        return Yd.cpu().numpy()
    finally:
        if own:
            hp.hmat_free(handle)


def _assert_parity(Y, Yref, tol=TOL):
    assert np.isfinite(Y).all()
    scale = np.abs(Yref).max()
    err = np.linalg.norm(Y - Yref) / np.linalg.norm(Yref)
    assert err <= tol, err
    assert np.abs(Y - Yref).max() <= tol * scale


CASES = [
    # (base workload, n, q, compression overrides)
    ("hss_uniform3d_n2048", 2048, 16, ()),                      # HSS, N=2048 at the workload's own size
    ("h2_gmm8d_n65536", 4096, 37, ()),                          # H2 d=8 mixture, ragged q
    ("h2_imq3d_n262144", 3000, 64, ()),                         # IMQ, N not a power of two (ragged leaves)
    ("h2_imq3d_n262144", 5000, 65, (("leaf_size", 40),)),       # deeper tree, q one past a tile
    ("hss_uniform3d_n2048", 1000, 1, ()),                       # q = 1
    ("hss_uniform3d_n2048", 777, 3, (("leaf_size", 50),)),      # q = 3, odd sizes
    ("h2_gmm8d_n65536", 4096, 2, ()),                           # q = 2 (2-column tiles)
    ("h2_invdist3d_n262144", 3000, 1, ()),                      # 1/r kernel, matrix-vector (q = 1)
    ("h2_imq3d_n262144", 3000, 8, ()),                          # q = 8 (8-column tiles)
    ("h2_imq3d_n262144", 2500, 17, (("admissibility", "none"),)),          # all near
    ("hss_uniform3d_n2048", 1500, 20, (("tol", 0.0), ("max_rank", 10 ** 6))),  # rank = |rows|
    ("hss_uniform3d_n2048", 1200, 9, (("tol", 1.0),)),          # every rank 0: far field vanishes
    ("h2_gmm8d_n65536", 60, 5, ()),                             # a single leaf (N <= leaf size)
]


@pytest.mark.parametrize("base,n,q,ov", CASES)
def test_fp64_matches_oracle(base, n, q, ov):
    w, H, _ = oracle_case(base, n, q, **dict(ov))
    W = rhs(w.n, q, 100 + n)
    Yref = hm.evaluate(H, W)
    Y = _gpu_eval(H, W)
    _assert_parity(Y, Yref)


def test_fp64_repeat_and_q_change_on_one_handle():
    w, H, _ = oracle_case("h2_imq3d_n262144", 3000, 64)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        for q, seed in ((64, 1), (8, 2), (130, 3), (64, 4)):
            W = rhs(w.n, q, seed)
            _assert_parity(_gpu_eval(H, W, handle=h), hm.evaluate(H, W))
        info = hp.hmat_info(h)
        assert info["n_points"] == w.n and info["near_entries"] == len(H.inter.near)
        assert info["near_values"] == hm.stored_entries(H)["near"]
    finally:
        hp.hmat_free(h)


def test_q_zero_is_a_noop_and_overlap_is_rejected():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        Wd = torch.zeros(w.n, 4, dtype=torch.float64, device="cuda")
        hp.hmat_eval(h, Wd, Wd, 0)
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_eval(h, Wd, Wd, 4)
        assert ei.value.status == hp.HMAT_EINVAL
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_eval(h, Wd, Wd, 4, mode=99)
        assert ei.value.status == hp.HMAT_EUNSUPPORTED
    finally:
        hp.hmat_free(h)


def test_load_rejects_non_finite_block():
    _, H, _ = oracle_case("hss_uniform3d_n2048", 600, 3)
    d = desc_from_oracle(H)
    near = list(d["near"])
    near[0] = np.array(near[0], copy=True)
    near[0][0, 0] = np.inf
    d["near"] = near
    with pytest.raises(hp.HmatError) as ei:
        hp.hmat_load(**d)
    assert ei.value.status == hp.HMAT_EINVAL


def test_linearity_on_gpu():
    w, H, _ = oracle_case("h2_gmm8d_n65536", 4096, 37)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        W1, W2 = rhs(w.n, 12, 1), rhs(w.n, 12, 2)
        Y1, Y2 = _gpu_eval(H, W1, handle=h), _gpu_eval(H, W2, handle=h)
        Y12 = _gpu_eval(H, 3 * W1 - 2 * W2, handle=h)
        assert np.linalg.norm(Y12 - (3 * Y1 - 2 * Y2)) <= 1e-13 * np.linalg.norm(Y12)
    finally:
        hp.hmat_free(h)
