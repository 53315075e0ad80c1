"""FP32 right-hand sides and results across the C ABI (hmat_eval_typed and friends).

The reference is the FP64 oracle evaluated on the widened W (every FP32 value is exact
in FP64):
- FP64 mode: the evaluation is FP64 and Y is rounded once to FP32, so Y equals the
  rounding of the FP64 path's own result bitwise, and is within 2^-24 (relative, per
  element of max|Y|) of the oracle;
- mixed mode: within the mode's 1e-6 of the oracle, and equal to the mixed result of
  the same W given as FP64 (the split starts from FP32 either way) up to the final
  rounding of Y to FP32.
Host copies, batches and the server take FP32 as well; a mixed-only handle (FP64 blocks
dropped) serves the mixed mode bitwise as the full handle does and refuses FP64.
"""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("h2_gmm8d_n65536", 4096, 37, ()), ("h2_imq3d_n262144", 5000, 130, (("leaf_size", 256),)),
         ("hss_uniform3d_n2048", 1000, 1, ())]


def _w32(n, q, seed):
    return rhs(n, q, seed).astype(np.float32)


def _eval(h, W, mode):
    Wd = torch.from_numpy(W).cuda()
    Yd = torch.full_like(Wd, float("nan"))
    hp.hmat_eval_typed(h, Wd, Yd, W.shape[1], mode)
    assert hp.hmat_status_poll(h) == hp.HMAT_OK
    return Yd.cpu().numpy()


@pytest.mark.parametrize("base,n,q,ov", CASES)
def test_f32_rhs_both_modes_match_the_oracle(base, n, q, ov):
    w, H, _ = oracle_case(base, n, q, **dict(ov))
    W32 = _w32(w.n, q, 40 + q)
    W64 = W32.astype(np.float64)
    Yref = hm.evaluate(H, W64)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        # FP64 mode: the rounding of the FP64 result of the widened W
        Y32 = _eval(h, W32, hp.HMAT_MODE_FP64)
        assert Y32.dtype == np.float32 and np.isfinite(Y32).all()
        Y64 = _eval(h, W64, hp.HMAT_MODE_FP64)
        assert np.array_equal(Y32, Y64.astype(np.float32))
        assert np.abs(Y32 - Yref).max() <= 2.0 ** -24 * np.abs(Yref).max() * 1.01
        # mixed mode
        M32 = _eval(h, W32, hp.HMAT_MODE_MIXED)
        err = np.linalg.norm(M32 - Yref) / np.linalg.norm(Yref)
        print(f"{base} n={n} q={q}: FP32 W mixed error {err:.3e}")
        assert err <= 1e-6
        M64 = _eval(h, W64, hp.HMAT_MODE_MIXED)
        assert np.array_equal(M32, M64.astype(np.float32)) or \
            np.abs(M32 - M64).max() <= 2.0 ** -23 * np.abs(M64).max()
    finally:
        hp.hmat_free(h)


def test_f32_host_batch_and_server():
    w, H, _ = oracle_case("h2_imq3d_n262144", 3000, 24)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        W32 = _w32(w.n, 24, 7)
        Yref = hm.evaluate(H, W32.astype(np.float64))
        for mode, tol in ((hp.HMAT_MODE_FP64, 1e-7), (hp.HMAT_MODE_MIXED, 1e-6)):
            dev = _eval(h, W32, mode)
            Yh = np.full_like(W32, np.nan)
            hp.hmat_eval_host_typed(h, W32, Yh, mode)
            assert np.array_equal(Yh, dev)
            b = hp.hmat_batch_create([h, h], mode)
            try:
                Ws = [torch.from_numpy(W32).cuda(), torch.from_numpy(W32[:, :5].copy()).cuda()]
                Ys = [torch.full_like(x, float("nan")) for x in Ws]
                hp.hmat_batch_eval_typed(b, Ws, Ys)
                torch.cuda.synchronize()
                assert np.array_equal(Ys[0].cpu().numpy(), dev)
                assert np.linalg.norm(Ys[1].cpu().numpy() - Yref[:, :5]) <= tol * np.linalg.norm(Yref[:, :5])
            finally:
                hp.hmat_batch_free(b)
            sv = hp.hmat_server_create([h], slots=2, memory_budget=4 << 30, max_q=64, mode=mode)
            try:
                Wp = torch.from_numpy(W32).pin_memory()
                Yp32 = torch.full(Wp.shape, float("nan"), dtype=torch.float32).pin_memory()
                W64p = torch.from_numpy(W32.astype(np.float64)).pin_memory()
                Yp64 = torch.full(W64p.shape, float("nan"), dtype=torch.float64).pin_memory()
                ids = [hp.hmat_server_submit(sv, 0, Wp, Yp32), hp.hmat_server_submit(sv, 0, W64p, Yp64)]
                for rid in ids:
                    assert hp.hmat_server_wait(sv, rid, 60000) == hp.HMAT_OK
                assert np.linalg.norm(Yp32.numpy() - Yref) <= tol * np.linalg.norm(Yref)
                assert np.linalg.norm(Yp64.numpy() - Yref) <= max(tol, 1e-12) * np.linalg.norm(Yref)
            finally:
                hp.hmat_server_free(sv)
    finally:
        hp.hmat_free(h)


def test_mixed_only_handle_serves_mixed_bitwise_and_refuses_fp64():
    w, H, _ = oracle_case("h2_gmm8d_n65536", 4096, 40)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    hm_only = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED_ONLY)
    try:
        full, only = hp.hmat_info(h), hp.hmat_info(hm_only)
        assert only["device_bytes"] + 8 * full["near_values"] <= full["device_bytes"]
        W = rhs(w.n, 40, 3)
        Wd = torch.from_numpy(W).cuda()
        Ya, Yb = torch.empty_like(Wd), torch.empty_like(Wd)
        hp.hmat_eval(h, Wd, Ya, 40, hp.HMAT_MODE_MIXED)
        hp.hmat_eval(hm_only, Wd, Yb, 40, hp.HMAT_MODE_MIXED)
        assert hp.hmat_status_poll(hm_only) == hp.HMAT_OK
        assert torch.equal(Ya, Yb)
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_eval(hm_only, Wd, Yb, 40, hp.HMAT_MODE_FP64)
        assert ei.value.status == hp.HMAT_EUNSUPPORTED
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_autotune(hm_only, 40, hp.HMAT_MODE_FP64)
        assert ei.value.status == hp.HMAT_EUNSUPPORTED
        rep = hp.hmat_autotune(hm_only, 40, hp.HMAT_MODE_MIXED)
        assert rep["near_cols"] > 0
    finally:
        hp.hmat_free(h)
        hp.hmat_free(hm_only)


def test_typed_calls_reject_unknown_dtypes():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        Wd = torch.zeros(w.n, 3, dtype=torch.float64, device="cuda")
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_eval_typed(h, Wd, torch.empty_like(Wd), 3, hp.HMAT_MODE_FP64, dtype=7)
        assert ei.value.status == hp.HMAT_EINVAL
    finally:
        hp.hmat_free(h)
