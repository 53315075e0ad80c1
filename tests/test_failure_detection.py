"""Failure detection on the GPU without a fault: a bounded device wait that runs out
reports HMAT_ETIMEOUT through the handle's status word, the poll clears it, and the
context stays usable (an evaluation right after it still matches the oracle).
"""
import time

import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_context_survives():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        t0 = time.perf_counter()
        hp.hmat_selftest_timeout(h, 2_000_000)            # a 2 ms wait that nothing ends
        assert hp.hmat_status_poll(h) == hp.HMAT_ETIMEOUT
        assert time.perf_counter() - t0 >= 0.002
        assert hp.hmat_status_poll(h) == hp.HMAT_OK        # the poll cleared the word
        W = rhs(w.n, 5, 3)
        Yref = hm.evaluate(H, W)
        for mode, tol in ((hp.HMAT_MODE_FP64, 1e-12), (hp.HMAT_MODE_MIXED, 1e-6)):
            Wd = torch.from_numpy(W).cuda()
            Yd = torch.empty_like(Wd)
            hp.hmat_eval(h, Wd, Yd, 5, mode)
            assert hp.hmat_status_poll(h) == hp.HMAT_OK
            assert np.linalg.norm(Yd.cpu().numpy() - Yref) <= tol * np.linalg.norm(Yref)
    finally:
        hp.hmat_free(h)


def test_selftest_rejects_bad_limits():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        for limit in (0, -5, 20_000_000_000):
            with pytest.raises(hp.HmatError) as ei:
                hp.hmat_selftest_timeout(h, limit)
            assert ei.value.status == hp.HMAT_EINVAL
    finally:
        hp.hmat_free(h)


@pytest.mark.parametrize("mode", [hp.HMAT_MODE_FP64, hp.HMAT_MODE_MIXED])
def test_chain_index_check_latches_edevice_and_context_survives(mode):
    """A far-chain launch whose only ticket names an item past the item array: the chain's own
    index check catches it before any read, latches HMAT_EDEVICE, and the next evaluation on
    the same context still matches the oracle."""
    w, H, _ = oracle_case("h2_gmm8d_n65536", 4096, 8)
    h = hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)
    try:
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        hp.hmat_selftest_device_check(h, 8, mode)
        assert hp.hmat_status_poll(h) == hp.HMAT_EDEVICE
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        W = rhs(w.n, 8, 21)
        Yref = hm.evaluate(H, W)
        Wd = torch.from_numpy(W).cuda()
        Yd = torch.empty_like(Wd)
        hp.hmat_eval(h, Wd, Yd, 8, mode)
        assert hp.hmat_status_poll(h) == hp.HMAT_OK
        tol = 1e-12 if mode == hp.HMAT_MODE_FP64 else 1e-6
        assert np.linalg.norm(Yd.cpu().numpy() - Yref) <= tol * np.linalg.norm(Yref)
    finally:
        hp.hmat_free(h)
