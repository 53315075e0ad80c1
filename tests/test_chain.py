"""The persistent far chain of the mixed mode (the upward pass, the FP32 coupling, the
downward transfers and the downward leaf step as a few persistent launches over every
tree level, with bounded dependency waits between their CTA tiles).

- Any number of CTAs gives bitwise the same result, down to a single CTA that walks
  every item in ticket order (which would time out, not hang, if an item's
  dependency came after it in the list), for both coupling engines.
- The serialised profiling mode gives bitwise the result of the overlapped one, and
  an evaluation takes fewer than ten launches.
- The FP64 mode's far field is one persistent launch too, bitwise the per-level launches.
- A chain launch whose waits cannot be met gives up after the host-chosen limit,
  reports HMAT_ETIMEOUT through the status word, and the context stays usable.
"""
import time

import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


def _mixed(h, W):
    Wd = torch.from_numpy(W).cuda()
    Yd = torch.full_like(Wd, float("nan"))
    hp.hmat_eval(h, Wd, Yd, W.shape[1], hp.HMAT_MODE_MIXED)
    assert hp.hmat_status_poll(h) == hp.HMAT_OK
    return Yd.cpu().numpy()


# (recipe, n, q, overrides, coupling engine expected: 1 FP32 in the chain, 2 tensor cores)
ENGINES = [
    ("h2_gmm8d_n65536", 4096, 40, (), 1),
    ("hss_uniform3d_n2048", 1500, 24, (("tol", 0.0), ("max_rank", 10 ** 6)), 2),
    ("h2_imq3d_n262144", 5000, 3, (("leaf_size", 40),), None),
]


@pytest.mark.parametrize("base,n,q,ov,engine", ENGINES)
def test_chain_grid_sizes_give_bitwise_the_same_result(base, n, q, ov, engine):
    w, H, _ = oracle_case(base, n, q, **dict(ov))
    W = rhs(w.n, q, 77 + q)
    Yref = hm.evaluate(H, W)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        if engine is not None:
            assert hp.hmat_info(h)["coupling_engine"] == engine
        Y0 = _mixed(h, W)
        err = np.linalg.norm(Y0 - Yref) / np.linalg.norm(Yref)
        print(f"{base} n={n} q={q}: mixed error {err:.3e}")
        assert err <= REL_TOL
        for grid in (1, 2, 3, 37, 152):
            hp.hmat_tune_apply(h, q, chain_grid=grid)
            Y = _mixed(h, W)
            assert np.array_equal(Y, Y0), grid
    finally:
        hp.hmat_free(h)


def test_serialised_profiling_is_bitwise_and_counts_launches():
    w, H, _ = oracle_case("h2_imq3d_n262144", 5000, 130, leaf_size=256)
    W = rhs(w.n, 130, 5)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        Y0 = _mixed(h, W)
        for mode in (1, 2):
            hp.hmat_profile(h, mode)
            Y = _mixed(h, W)
            ph = hp.hmat_phase_times(h)
            hp.hmat_profile(h, False)
            assert np.array_equal(Y, Y0), mode
            launches = sum(c for _, c in ph.values())
            # split (2) + up chain + [w split (2) + tensor-core coupling + down chain] + near + leaf chain
            assert launches <= 9, ph
            assert ph["far_up"][1] == 1 and ph["near"][1] == 1 and ph["down_leaf"][1] == 1, ph
            assert all(ms >= 0.0 for ms, _ in ph.values())
    finally:
        hp.hmat_free(h)


def test_chain_wait_runs_out_reports_timeout_and_context_survives():
    w, H, _ = oracle_case("h2_gmm8d_n65536", 4096, 40)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        W = rhs(w.n, 40, 11)
        Y0 = _mixed(h, W)
        t0 = time.perf_counter()
        hp.hmat_selftest_chain_timeout(h, 40, 3_000_000)   # 3 ms, then every wait gives up
        assert hp.hmat_status_poll(h) == hp.HMAT_ETIMEOUT
        assert time.perf_counter() - t0 >= 0.003
        assert hp.hmat_status_poll(h) == hp.HMAT_OK        # the poll cleared the word
        assert np.array_equal(_mixed(h, W), Y0)            # the next evaluation is unaffected
        Yref = hm.evaluate(H, W)
        Wd = torch.from_numpy(W).cuda()
        Yd = torch.empty_like(Wd)
        hp.hmat_eval(h, Wd, Yd, 40, hp.HMAT_MODE_FP64)
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        assert np.linalg.norm(Yd.cpu().numpy() - Yref) <= 1e-12 * np.linalg.norm(Yref)
        for limit in (0, -1, 20_000_000_000):
            with pytest.raises(hp.HmatError) as ei:
                hp.hmat_selftest_chain_timeout(h, 40, limit)
            assert ei.value.status == hp.HMAT_EINVAL
    finally:
        hp.hmat_free(h)


def test_tune_apply_rejects_bad_choices():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    h64 = hp.hmat_load(**desc_from_oracle(H))
    try:
        for kw in (dict(near_cols=24), dict(chain_grid=-1)):
            with pytest.raises(hp.HmatError) as ei:
                hp.hmat_tune_apply(h, 16, **kw)
            assert ei.value.status == hp.HMAT_EINVAL
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_tune_apply(h64, 16)
        assert ei.value.status == hp.HMAT_EUNSUPPORTED
    finally:
        hp.hmat_free(h)
        hp.hmat_free(h64)


@pytest.mark.parametrize("base,n,q,ov", [("h2_gmm8d_n65536", 4096, 37, ()), ("hss_uniform3d_n2048", 2048, 16, ()),
                                         ("h2_imq3d_n262144", 5000, 3, (("leaf_size", 40),)),
                                         ("hss_uniform3d_n2048", 1500, 24, (("tol", 0.0), ("max_rank", 10 ** 6)))])
def test_fp64_chain_equals_per_level_launches_bitwise(base, n, q, ov):
    """The FP64 far field as one persistent launch of 16-row tiles sums every output in the
    order of the per-level launches that hmat_eval_noalloc keeps, so the two agree bit for bit,
    for every column width the tuner may pick."""
    import ctypes
    w, H, _ = oracle_case(base, n, q, **dict(ov))
    W = rhs(w.n, q, 31 + q)
    Yref = hm.evaluate(H, W)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        fn = hp.library().hmat_eval_noalloc
        fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        fn.restype = ctypes.c_int
        Wd = torch.from_numpy(W).cuda()
        Yl = torch.full_like(Wd, float("nan"))
        assert fn(h, Wd.data_ptr(), Yl.data_ptr(), q, torch.cuda.current_stream().cuda_stream) == hp.HMAT_OK
        Yc = torch.full_like(Wd, float("nan"))
        hp.hmat_eval(h, Wd, Yc, q, hp.HMAT_MODE_FP64)
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        assert torch.equal(Yc, Yl)
        assert np.linalg.norm(Yc.cpu().numpy() - Yref) <= 1e-12 * np.linalg.norm(Yref)
        rep = hp.hmat_autotune(h, q, hp.HMAT_MODE_FP64)
        Yt = torch.full_like(Wd, float("nan"))
        hp.hmat_eval(h, Wd, Yt, q, hp.HMAT_MODE_FP64)
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        assert torch.equal(Yt, Yl), rep
    finally:
        hp.hmat_free(h)


def test_fp64_chain_wait_runs_out_and_context_survives():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 2048, 16)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        W = rhs(w.n, 16, 12)
        Wd = torch.from_numpy(W).cuda()
        Y0 = torch.empty_like(Wd)
        hp.hmat_eval(h, Wd, Y0, 16, hp.HMAT_MODE_FP64)
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        hp.hmat_selftest_chain_timeout(h, 16, 2_000_000, mode=hp.HMAT_MODE_FP64)
        assert hp.hmat_status_poll(h) == hp.HMAT_ETIMEOUT
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        Y1 = torch.empty_like(Wd)
        hp.hmat_eval(h, Wd, Y1, 16, hp.HMAT_MODE_FP64)
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        assert torch.equal(Y0, Y1)
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_selftest_chain_timeout(h, 16, 2_000_000, mode=hp.HMAT_MODE_MIXED)
        assert ei.value.status == hp.HMAT_EUNSUPPORTED
    finally:
        hp.hmat_free(h)
