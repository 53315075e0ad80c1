"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a,
exports every entry point include/hmat.h declares, and hmat_load rejects invalid
HMatrix descriptions before it touches the device."""
import numpy as np
import pytest

import paper_1812_07152_gb300 as hp
from paper_1812_07152_gb300 import build as hbuild
from tests.fixtures import desc_from_oracle, oracle_case


def test_library_builds_and_exports_every_declared_symbol():
    path = hbuild.build()
    assert path.endswith("libhmat.so")
    lib = hp.library()
    declared = hp.exported_symbols()
    assert {"hmat_load", "hmat_eval", "hmat_free", "hmat_status_poll", "hmat_strerror"} <= set(declared)
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_covers_every_status():
    for s in (hp.HMAT_OK, hp.HMAT_EINVAL, hp.HMAT_ENOMEM, hp.HMAT_ECUDA, hp.HMAT_ETIMEOUT,
              hp.HMAT_EUNSUPPORTED, hp.HMAT_EDEVICE):
        assert hp.hmat_strerror(s) and hp.hmat_strerror(s) != "unknown status"
    assert hp.hmat_strerror(12345) == "unknown status"


def _valid():
    _, H, _ = oracle_case("hss_uniform3d_n2048", 600, 3)
    return desc_from_oracle(H)


def _expect_einval(d):
    with pytest.raises(hp.HmatError) as ei:
        hp.hmat_load(**d)
    assert ei.value.status == hp.HMAT_EINVAL


@pytest.mark.parametrize("mutate", [
    "perm_dup", "perm_range", "child_size", "near_idx_range", "near_ptr_order", "far_same_node",
    "far_level", "null_basis", "root_size", "negative_rank",
])
def test_load_rejects_invalid_descriptions(mutate):
    d = _valid()
    d = {k: (list(v) if isinstance(v, list) else (np.array(v, copy=True) if isinstance(v, np.ndarray) else v))
         for k, v in d.items()}
    if mutate == "perm_dup":
        d["perm"][1] = d["perm"][0]
    elif mutate == "perm_range":
        d["perm"][0] = d["n_points"]
    elif mutate == "child_size":
        d["node_size"][1] += 1
    elif mutate == "near_idx_range":
        d["near_idx"][0] = 2 ** d["levels"]
    elif mutate == "near_ptr_order":
        d["near_ptr"][1], d["near_ptr"][2] = d["near_ptr"][2], d["near_ptr"][1] - 1
    elif mutate == "far_same_node":
        d["far_idx"][0] = np.nonzero(np.diff(d["far_ptr"]))[0][0]
    elif mutate == "far_level":
        a = np.nonzero(np.diff(d["far_ptr"]))[0][0]
        d["far_idx"][d["far_ptr"][a]] = 0
    elif mutate == "null_basis":
        a = int(np.nonzero(d["rank"])[0][0])
        d["basis"][a] = None
    elif mutate == "root_size":
        d["node_size"][0] -= 1
    elif mutate == "negative_rank":
        d["rank"][3] = -1
    _expect_einval(d)


def test_null_and_out_of_range_arguments_are_rejected_before_any_device_work():
    """Every entry point that takes a handle, batch or server refuses a null one with
    HMAT_EINVAL (no CUDA call is made, so this runs without a GPU); the free calls accept
    null as a no-op; the choice-taking calls refuse out-of-range choices."""
    import ctypes
    lib = hp.library()
    V, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    null = V(0)
    calls = {
        "hmat_eval": ([V, V, V, I64, I32, V], (null, null, null, 4, hp.HMAT_MODE_FP64, null)),
        "hmat_eval_typed": ([V, V, V, I64, I32, I32, V], (null, null, null, 4, hp.HMAT_MODE_MIXED, 1, null)),
        "hmat_eval_host": ([V, V, V, I64, I32, V], (null, null, null, 4, hp.HMAT_MODE_FP64, null)),
        "hmat_eval_noalloc": ([V, V, V, I64, V], (null, null, null, 4, null)),
        "hmat_reserve": ([V, I64], (null, 4)),
        "hmat_profile": ([V, I32], (null, 1)),
        "hmat_tune_apply": ([V, V], (null, null)),
        "hmat_autotune": ([V, I64, I32, V, V], (null, 4, hp.HMAT_MODE_FP64, null, null)),
        "hmat_batch_info": ([V, V, I32], (null, null, 6)),
        "hmat_batch_schedule": ([V, I32, I32, I32], (null, 0, 0, 0)),
        "hmat_server_wait": ([V, I64, I32], (null, 0, 0)),
        "hmat_server_stats": ([V, V, I32], (null, null, 4)),
        "hmat_server_matrix_stats": ([V, I32, V, I32], (null, 0, null, 4)),
        "hmat_selftest_timeout": ([V, I64, V], (null, 1000000, null)),
        "hmat_selftest_chain_timeout": ([V, I64, I32, I64, V], (null, 4, hp.HMAT_MODE_MIXED, 1000000, null)),
        "hmat_selftest_device_check": ([V, I64, I32, V], (null, 4, hp.HMAT_MODE_MIXED, null)),
        "hmat_info": ([V, V, I32], (null, null, 4)),
    }
    for name, (argtypes, args) in calls.items():
        fn = getattr(lib, name)
        fn.argtypes, fn.restype = argtypes, ctypes.c_int
        assert fn(*args) == hp.HMAT_EINVAL, name
    for name in ("hmat_free", "hmat_batch_free", "hmat_server_free", "hmat_plan_free"):
        fn = getattr(lib, name)
        fn.argtypes, fn.restype = [V], ctypes.c_int
        assert fn(null) == hp.HMAT_OK, name
    assert hp.hmat_strerror(hp.HMAT_EBUSY) != "unknown status"
