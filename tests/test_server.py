"""Serving (hmat_server_*): requests on resident HMatrices, admitted by free slot
and device memory, merged by matrix while they wait (continuous batching). Each
result must be the one the request gets alone: bitwise in FP64 mode, within the
mixed mode's 1e-6 otherwise."""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MATS = [("hss_uniform3d_n2048", 2048, ()), ("h2_imq3d_n262144", 3000, ()), ("h2_gmm8d_n65536", 4096, ())]


@pytest.fixture(scope="module")
def mats():
    out = []
    for base, n, ov in MATS:
        w, H, _ = oracle_case(base, n, 8, **dict(ov))
        out.append((w, hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)))
    yield out
    for _, h in out:
        hp.hmat_free(h)


def _alone(h, W, mode):
    Wd = W.cuda()
    Y = torch.empty_like(Wd)
    hp.hmat_eval(h, Wd, Y, W.shape[1], mode)
    torch.cuda.synchronize()
    return Y.cpu()


def _need_fp64(n, sum_rank, q):
    al = lambda x: (x + 255) // 256 * 256
    return al(2 * al(max(sum_rank, 1) * q * 8)) + 2 * al(n * q * 8)


@pytest.mark.parametrize("mode", [hp.HMAT_MODE_FP64, hp.HMAT_MODE_MIXED])
def test_mix_equals_alone(mats, mode):
    rng = np.random.default_rng(5)
    handles = [h for _, h in mats]
    sv = hp.hmat_server_create(handles, slots=3, memory_budget=8 << 30, max_q=256, mode=mode)
    try:
        reqs = []
        for k in range(24):
            m = int(rng.integers(0, len(mats)))
            q = int(rng.integers(1, 70))
            W = torch.from_numpy(rhs(mats[m][0].n, q, 900 + k)).pin_memory()
            Y = torch.full(W.shape, float("nan"), dtype=torch.float64).pin_memory()
            reqs.append((m, W, Y, hp.hmat_server_submit(sv, m, W, Y)))
        for m, W, Y, rid in reqs:
            assert hp.hmat_server_wait(sv, rid, 60000) == hp.HMAT_OK
        stats = hp.hmat_server_stats(sv)
        assert stats["completed"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    finally:
        hp.hmat_server_free(sv)
    for m, W, Y, _ in reqs:
        ref = _alone(mats[m][1], W, mode)
        if mode == hp.HMAT_MODE_FP64:
            assert torch.equal(Y, ref)
        else:
            err = float(torch.linalg.norm(Y - ref) / torch.linalg.norm(ref))
            assert err <= 1e-6, err


def test_waiting_requests_are_merged(mats):
    w, h = mats[2]
    sv = hp.hmat_server_create([h], slots=1, memory_budget=8 << 30, max_q=512, mode=hp.HMAT_MODE_FP64)
    try:
        reqs = []
        for k in range(16):
            W = torch.from_numpy(rhs(w.n, 16, 950 + k)).pin_memory()
            Y = torch.empty_like(W).pin_memory()
            reqs.append((W, Y, hp.hmat_server_submit(sv, 0, W, Y)))
        for W, Y, rid in reqs:
            assert hp.hmat_server_wait(sv, rid, 60000) == hp.HMAT_OK
        stats = hp.hmat_server_stats(sv)
        assert stats["requests_per_evaluation"] > 1.0 and stats["evaluations"] < len(reqs)
    finally:
        hp.hmat_server_free(sv)
    for W, Y, _ in reqs:
        assert torch.equal(Y, _alone(h, W, hp.HMAT_MODE_FP64))


def test_memory_budget_bounds_admission(mats):
    w, h = mats[1]
    info = hp.hmat_info(h)
    budget = _need_fp64(info["n_points"], info["sum_rank"], 8) + 4096  # room for one request of q <= 8
    sv = hp.hmat_server_create([h], slots=4, memory_budget=budget, max_q=64, mode=hp.HMAT_MODE_FP64)
    try:
        W_big = torch.zeros(w.n, 64, dtype=torch.float64).pin_memory()
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_server_submit(sv, 0, W_big, torch.empty_like(W_big).pin_memory())
        assert ei.value.status == hp.HMAT_ENOMEM
        W_pageable = torch.zeros(w.n, 4, dtype=torch.float64)
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_server_submit(sv, 0, W_pageable, torch.empty_like(W_pageable))
        assert ei.value.status == hp.HMAT_EINVAL
        reqs = []
        for k in range(6):
            W = torch.from_numpy(rhs(w.n, 8, 990 + k)).pin_memory()
            Y = torch.empty_like(W).pin_memory()
            reqs.append((W, Y, hp.hmat_server_submit(sv, 0, W, Y)))
        for W, Y, rid in reqs:
            assert hp.hmat_server_wait(sv, rid, 60000) == hp.HMAT_OK
        stats = hp.hmat_server_stats(sv)
        assert 0 < stats["peak_bytes"] <= budget
    finally:
        hp.hmat_server_free(sv)
    for W, Y, _ in reqs:
        assert torch.equal(Y, _alone(h, W, hp.HMAT_MODE_FP64))


def test_bounded_queue_sheds_load_and_per_matrix_stats(mats):
    """With max_pending, a burst beyond what one slot drains is refused with HMAT_EBUSY
    (nothing queued); every accepted request completes, the refusals are counted, and
    the per-matrix completions add up to the total."""
    handles = [h for _, h in mats]
    sv = hp.hmat_server_create(handles, slots=1, memory_budget=8 << 30, max_q=64, mode=hp.HMAT_MODE_FP64,
                               max_pending=2)
    accepted, refused = [], 0
    try:
        bufs = []
        for k in range(200):
            m = k % len(mats)
            W = torch.from_numpy(rhs(mats[m][0].n, 64, 1300 + k)).pin_memory()
            Y = torch.empty_like(W).pin_memory()
            bufs.append((W, Y))
            try:
                accepted.append(hp.hmat_server_submit(sv, m, W, Y))
            except hp.HmatError as e:
                assert e.status == hp.HMAT_EBUSY
                refused += 1
        for rid in accepted:
            assert hp.hmat_server_wait(sv, rid, 60000) == hp.HMAT_OK
        st = hp.hmat_server_stats(sv)
        assert refused > 0 and st["rejected"] == refused
        assert st["completed"] == len(accepted)
        per = [hp.hmat_server_matrix_stats(sv, m) for m in range(len(mats))]
        assert sum(p["completed"] for p in per) == len(accepted)
        for p in per:
            if p["completed"]:
                assert p["p99_ms"] >= p["p50_ms"] > 0
    finally:
        hp.hmat_server_free(sv)
