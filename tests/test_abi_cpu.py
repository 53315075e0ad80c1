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
