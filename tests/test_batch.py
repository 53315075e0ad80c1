"""Batched evaluation (hmat_batch_*): many HMatrices of uneven size, rank and q in
one CUDA-graph launch in which every step is one launch over all members. Every
member's result must be bitwise the one it gets when evaluated alone (the same tiles
summed in the same order, no atomics) and match the FP64 oracle within the mode's
tolerance; the mixed-mode graph holds about ten kernels however many members."""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from oracle import hmatrix as hm
from tests.fixtures import desc_from_oracle, oracle_case, rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MEMBERS = [
    ("hss_uniform3d_n2048", 2048, ()),
    ("h2_gmm8d_n65536", 3000, (("leaf_size", 64),)),
    ("h2_imq3d_n262144", 1500, (("leaf_size", 128),)),
    ("h2_imq3d_n262144", 5000, (("leaf_size", 256),)),
    ("h2_gmm8d_n65536", 1100, ()),
    ("hss_uniform3d_n2048", 1500, (("tol", 0.0), ("max_rank", 10 ** 6))),   # coupling on the tensor cores
]


@pytest.fixture(scope="module")
def loaded():
    out = []
    for base, n, ov in MEMBERS:
        w, H, _ = oracle_case(base, n, 8, **dict(ov))
        out.append((w, H, hp.hmat_load(**desc_from_oracle(H), flags=hp.HMAT_LOAD_MIXED)))
    yield out
    for _, _, h in out:
        hp.hmat_free(h)


@pytest.mark.parametrize("mode,tol", [(hp.HMAT_MODE_FP64, 1e-12), (hp.HMAT_MODE_MIXED, 1e-6)])
def test_batch_equals_members_alone(loaded, mode, tol):
    # the second member appears twice, with different right-hand sides
    members = loaded + [loaded[1]]
    qs = [5, 64, 1, 130, 17, 24, 33]
    handles = [h for _, _, h in members]
    Ws = [torch.from_numpy(rhs(w.n, q, 700 + i)).cuda() for i, ((w, _, _), q) in enumerate(zip(members, qs))]
    Ys = [torch.full_like(W, float("nan")) for W in Ws]
    b = hp.hmat_batch_create(handles, mode)
    try:
        for rep in range(3):  # capture, then two replays
            if rep == 2:
                for W in Ws:
                    W.mul_(-0.5)
            hp.hmat_batch_eval(b, Ws, Ys)
            torch.cuda.synchronize()
            info = hp.hmat_batch_info(b)
            assert info["members"] == len(members)
            if mode == hp.HMAT_MODE_MIXED:
                assert 0 < info["kernels"] <= 10, info
            for (w, H, h), W, Y in zip(members, Ws, Ys):
                alone = torch.empty_like(W)
                hp.hmat_eval(h, W, alone, W.shape[1], mode)
                torch.cuda.synchronize()
                assert torch.equal(Y, alone)
                Yref = hm.evaluate(H, W.cpu().numpy())
                err = np.linalg.norm(Y.cpu().numpy() - Yref) / np.linalg.norm(Yref)
                assert err <= tol, err
        assert all(hp.hmat_status_poll(h) == hp.HMAT_OK for h in handles)
        # the other schedules (one branch per member; a capped chain grid) and the tuner's
        # choice give bitwise the same results
        ref = [Y.clone() for Y in Ys]
        if mode == hp.HMAT_MODE_MIXED:  # a member tuned to a non-default width, then batched at either
            hp.hmat_tune_apply(handles[3], qs[3], near_cols=48)
        for branched, grid, widths in ((1, 0, 0), (0, 7, 0), (0, 0, 1), (0, 0, 0)):
            hp.hmat_batch_schedule(b, branched, grid, widths)
            for Y in Ys:
                Y.fill_(float("nan"))
            hp.hmat_batch_eval(b, Ws, Ys)
            torch.cuda.synchronize()
            info = hp.hmat_batch_info(b)
            assert info["branched"] == branched and info["default_widths"] == widths
            assert all(torch.equal(Y, R) for Y, R in zip(Ys, ref)), (branched, grid, widths)
        rep = hp.hmat_batch_autotune(b, Ws, Ys)
        assert 0 < rep["tuned_ms"] <= rep["default_ms"]
        hp.hmat_batch_eval(b, Ws, Ys)
        torch.cuda.synchronize()
        assert all(torch.equal(Y, R) for Y, R in zip(Ys, ref))
        assert all(hp.hmat_status_poll(h) == hp.HMAT_OK for h in handles)
    finally:
        hp.hmat_batch_free(b)


def test_batch_new_arguments_recapture(loaded):
    handles = [h for _, _, h in loaded]
    b = hp.hmat_batch_create(handles, hp.HMAT_MODE_FP64)
    try:
        for qs in ((3, 3, 3, 3, 3), (9, 1, 40, 2, 7)):
            Ws = [torch.from_numpy(rhs(w.n, q, 800 + q)).cuda() for (w, _, _), q in zip(loaded, qs)]
            Ys = [torch.empty_like(W) for W in Ws]
            hp.hmat_batch_eval(b, Ws, Ys)
            torch.cuda.synchronize()
            for (w, H, _), W, Y in zip(loaded, Ws, Ys):
                Yref = hm.evaluate(H, W.cpu().numpy())
                assert np.linalg.norm(Y.cpu().numpy() - Yref) <= 1e-12 * np.linalg.norm(Yref)
    finally:
        hp.hmat_batch_free(b)


def test_batch_rejects_mixed_without_mixed_copy():
    w, H, _ = oracle_case("hss_uniform3d_n2048", 1000, 1)
    h = hp.hmat_load(**desc_from_oracle(H))
    try:
        with pytest.raises(hp.HmatError) as ei:
            hp.hmat_batch_create([h], hp.HMAT_MODE_MIXED)
        assert ei.value.status == hp.HMAT_EUNSUPPORTED
    finally:
        hp.hmat_free(h)
