"""Test helpers: turn an oracle HMatrix into the arrays of the C ABI's hmat_desc."""
import functools

import numpy as np

from oracle import hmatrix as hm
from workloads import WORKLOADS, normal_rhs, reduced


def desc_from_oracle(H: "hm.HMatrix") -> dict:
    t = H.tree
    near_ptr, near_idx = H.near_csr()
    far_ptr, far_idx = H.far_csr()
    return dict(n_points=int(t.perm.shape[0]), levels=int(t.levels), node_begin=t.begin, node_size=t.size,
                rank=H.rank, near_ptr=near_ptr, near_idx=near_idx, far_ptr=far_ptr, far_idx=far_idx,
                basis=H.basis, coupling=H.far_blocks, near=H.near_blocks, perm=t.perm)


@functools.lru_cache(maxsize=None)
def oracle_case(base: str, n: int, q: int, **overrides):
    """(workload, HMatrix, points) for a reduced-size workload, cached per process."""
    w = reduced(WORKLOADS[base], n, q=q)
    H, X = hm.compress_workload(w, **overrides)
    return w, H, X


def oracle_case_kw(base, n, q, overrides):
    return oracle_case(base, n, q, **dict(overrides))


def rhs(n: int, q: int, seed: int) -> np.ndarray:
    return normal_rhs(n, q, seed)
