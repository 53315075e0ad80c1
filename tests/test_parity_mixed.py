"""GPU parity of the mixed-precision mode (HMAT_MODE_MIXED) against the FP64 oracle.

The near field runs on the tcgen05 tensor cores with FP16 hi+lo splits of D and W
(22 significant bits per value, the Dl*Wl term dropped: 2^-22 relative) and FP32
accumulation drained into compensated sums every near block; the far field runs in
FP32. The target is a relative Frobenius error <= 1e-6 against the FP64 oracle
(every case prints the measured error); element by element the bound is 1e-5 of
the largest |Y| (an element can lose more relative accuracy than the norm when its
row sum cancels).
"""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-6
ELEM_TOL = 1e-5


def _eval(h, W, mode):
    Wd = torch.from_numpy(W).cuda()
    Yd = torch.full_like(Wd, float("nan"))
    hp.hmat_eval(h, Wd, Yd, W.shape[1], mode)
    assert hp.hmat_status_poll(h) == hp.HMAT_OK
    return Yd.cpu().numpy()


def _check(Y, Yref, label):
    assert np.isfinite(Y).all(), label
    err = np.linalg.norm(Y - Yref) / np.linalg.norm(Yref)
    emax = np.abs(Y - Yref).max() / np.abs(Yref).max()
    print(f"{label}: mixed relative Frobenius error {err:.3e}, max element error {emax:.3e} of max|Y|")
    assert err <= REL_TOL, (label, err)
    assert emax <= ELEM_TOL, (label, emax)
    return err


CASES = [
    ("hss_uniform3d_n2048", 2048, 16, ()),                       # HSS, leaf 64 (one k-chunk)
    ("h2_gmm8d_n65536", 4096, 37, ()),                           # leaf 128 (two k-chunks), ragged q
    ("h2_gmm8d_n65536", 4096, 256, ()),                          # q = 256: two column tiles of 128
    ("h2_imq3d_n262144", 3000, 64, ()),                          # ragged leaves (93/94 points)
    ("h2_imq3d_n262144", 5000, 130, (("leaf_size", 256),)),      # leaves > 128 rows (two m-tiles), q = 130
    ("h2_imq3d_n262144", 5000, 3, (("leaf_size", 40),)),         # leaves of 39/40 points, q = 3
    ("hss_uniform3d_n2048", 1000, 1, ()),                        # q = 1
    ("h2_imq3d_n262144", 2500, 17, (("admissibility", "none"),)),  # all near
    ("hss_uniform3d_n2048", 1500, 24, (("tol", 0.0), ("max_rank", 10 ** 6))),  # full rank: up to 6 m-tiles per node
    ("h2_invdist3d_n262144", 3000, 1, ()),                       # 1/r kernel, matrix-vector (q = 1)
    ("h2_gmm8d_n65536", 4096, 300, ()),                          # q > 256: 128-column FP32 far-field tiles
    ("hss_uniform3d_n2048", 1200, 9, (("tol", 1.0),)),           # every rank 0
    ("h2_gmm8d_n65536", 60, 5, ()),                              # a single leaf
]


@pytest.mark.parametrize("base,n,q,ov", CASES)
def test_mixed_matches_oracle(base, n, q, ov):
    w, H, _ = oracle_case(base, n, q, **dict(ov))
    W = rhs(w.n, q, 500 + n + q)
    Yref = hm.evaluate(H, W)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        _check(_eval(h, W, hp.HMAT_MODE_MIXED), Yref, f"{base} n={n} q={q} {dict(ov)}")
        # the FP64 mode of the same handle is unaffected
        Y64 = _eval(h, W, hp.HMAT_MODE_FP64)
        assert np.linalg.norm(Y64 - Yref) <= 1e-12 * np.linalg.norm(Yref)
    finally:
        hp.hmat_free(h)


def test_mixed_repeat_q_change_and_scaled_inputs():
    w, H, _ = oracle_case("h2_imq3d_n262144", 3000, 64)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        for q, seed, scale in ((64, 1, 1.0), (8, 2, 1e-12), (200, 3, 1e12), (64, 4, 1.0)):
            W = rhs(w.n, q, seed) * scale
            _check(_eval(h, W, hp.HMAT_MODE_MIXED), hm.evaluate(H, W), f"q={q} W*{scale:g}")
    finally:
        hp.hmat_free(h)


def test_mixed_zero_rhs_gives_zero():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        Y = _eval(h, np.zeros((w.n, 7)), hp.HMAT_MODE_MIXED)
        assert np.array_equal(Y, np.zeros_like(Y))
    finally:
        hp.hmat_free(h)


def test_mixed_needs_the_mixed_copy():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        Wd = torch.zeros(w.n, 4, dtype=torch.float64, device="cuda")
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_eval(h, Wd, torch.empty_like(Wd), 4, hp.HMAT_MODE_MIXED)
        assert ei.value.status == hp.HMAT_EUNSUPPORTED
    finally:
        hp.hmat_free(h)


def test_built_handle_mixed_mode():
    w, H, X = oracle_case("h2_gmm8d_n65536", 4096, 8)
    h = hp.hmat_build(X, kernel=w.kernel, kernel_param=w.kernel_param, admissibility=w.admissibility,
                      leaf_size=w.leaf_size, tol=w.tol, max_rank=w.max_rank, eta=w.eta, flags=hp.HMAT_LOAD_MIXED)
    try:
        W = rhs(w.n, 48, 9)
        Y64 = _eval(h, W, hp.HMAT_MODE_FP64)
        Ymx = _eval(h, W, hp.HMAT_MODE_MIXED)
        assert np.linalg.norm(Ymx - Y64) <= REL_TOL * np.linalg.norm(Y64)
    finally:
        hp.hmat_free(h)


@pytest.mark.parametrize("base,n,engine", [("h2_gmm8d_n65536", 4096, 1), ("h2_imq3d_n262144", 3000, 2)])
def test_mixed_coupling_engine_choice(base, n, engine):
    """Small ranks (d = 8 mixture, ranks <= 31) keep the coupling on the FP32 CUDA cores; ranks near
    100 fill the 128 x 64 tensor-core tiles and move it there. Both match the oracle."""
    w, H, _ = oracle_case(base, n, 64)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        assert hp.hmat_info(h)["coupling_engine"] == engine
        W = rhs(w.n, 40, 77)
        _check(_eval(h, W, hp.HMAT_MODE_MIXED), hm.evaluate(H, W), f"{base} n={n} engine={engine}")
    finally:
        hp.hmat_free(h)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        assert hp.hmat_info(h)["coupling_engine"] == 0
    finally:
        hp.hmat_free(h)


def test_eval_host_pipelined_mixed_and_fp64():
    """hmat_eval_host: FP64 gives hmat_eval's result bit for bit; the mixed mode at q >= 128
    evaluates two column groups with overlapped copies and stays within the mixed tolerance."""
    w, H, _ = oracle_case("h2_imq3d_n262144", 3000, 64)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        for q in (200, 130):
            W = rhs(w.n, q, 90 + q)
            Yref = hm.evaluate(H, W)
            Wh = torch.from_numpy(W).pin_memory()
            Yh = torch.empty_like(Wh).pin_memory()
            hp.hmat_eval_host(h, Wh, Yh, hp.HMAT_MODE_MIXED)
            _check(Yh.numpy(), Yref, f"eval_host mixed q={q}")
            hp.hmat_eval_host(h, Wh, Yh, hp.HMAT_MODE_FP64)
            assert np.array_equal(Yh.numpy(), _eval(h, W, hp.HMAT_MODE_FP64))
    finally:
        hp.hmat_free(h)


def test_integer_unit_conversions_match_hardware():
    """The mixed mode widens, narrows and rescales on the integer units (FP64 runs at 1/64
    rate): bitwise equal to the hardware conversions and multiply on 2^24 hashed samples."""
    bad = hp.hmat_selftest_conversions(1 << 24, seed=12345)
    print(f"integer-unit conversions, mismatches on 2^24 samples: {bad}")
    assert bad == {"widen": 0, "narrow": 0, "scale": 0}
