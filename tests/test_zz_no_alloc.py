"""hmat_eval_noalloc: the FP64 evaluation for callers that may not allocate device
memory during a call (a latency-critical loop, where cudaMalloc would synchronise
the device, or a process whose device memory another allocator owns). Its
workspaces live in a static device array of HMAT_NOALLOC_SCRATCH_VALUES doubles,
loaded onto the device by hmat_load.

The test calls it through the C ABI twice in a row on a freshly loaded handle
that hmat_eval has never touched, checks that neither call grows the handle's
device memory or takes the array's 16 MiB from the device, and only then
compares each result with hmat_eval's, within the FP64 tolerance of the parity
tests. It is collected last, and passes alone in a fresh process or after the
others.
"""
import ctypes

import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
SCRATCH_VALUES = 2097152  # HMAT_NOALLOC_SCRATCH_VALUES in include/hmat.h
SCRATCH_BYTES = 8 * SCRATCH_VALUES


def _noalloc():
    fn = hp.library().hmat_eval_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_allocates_nothing_and_matches_hmat_eval_on_two_calls_in_a_row():
    q = 24
    w, H, _ = oracle_case("h2_imq3d_n262144", 3000, q)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        stream = torch.cuda.current_stream()
        fn = _noalloc()
        Ws = [torch.from_numpy(rhs(w.n, q, seed)).cuda() for seed in (31, 32)]
        Ys = [torch.full_like(W, float("nan")) for W in Ws]
        torch.cuda.synchronize()
        held = hp.hmat_info(h)["device_bytes"]
        for W, Y in zip(Ws, Ys):
            free_before = torch.cuda.mem_get_info()[0]
            st = fn(h, W.data_ptr(), Y.data_ptr(), q, stream.cuda_stream)
            assert st == hp.HMAT_OK, hp.hmat_strerror(st)
            assert hp.hmat_status_poll(h, stream) == hp.HMAT_OK
            free_after = torch.cuda.mem_get_info()[0]
            # no workspace for the handle, and the static array was already on the device
            assert hp.hmat_info(h)["device_bytes"] == held
            assert free_before - free_after < SCRATCH_BYTES
        for W, Y in zip(Ws, Ys):
            Y_ref = torch.empty_like(W)
            hp.hmat_eval(h, W, Y_ref, q, hp.HMAT_MODE_FP64, stream)
            assert hp.hmat_status_poll(h, stream) == hp.HMAT_OK
            a, b = Y.cpu().numpy(), Y_ref.cpu().numpy()
            assert np.isfinite(a).all()
            assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b)
            assert np.abs(a - b).max() <= TOL * np.abs(b).max()
    finally:
        hp.hmat_free(h)


def test_noalloc_rejects_workspaces_beyond_the_array():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 2048, 16)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        sum_rank = hp.hmat_info(h)["sum_rank"]
        q_too_big = SCRATCH_VALUES // 2 // sum_rank + 1
        W = torch.zeros(w.n, q_too_big, dtype=torch.float64, device="cuda")
        Y = torch.empty_like(W)
        st = _noalloc()(h, W.data_ptr(), Y.data_ptr(), q_too_big, torch.cuda.current_stream().cuda_stream)
        assert st == hp.HMAT_EINVAL
    finally:
        hp.hmat_free(h)
