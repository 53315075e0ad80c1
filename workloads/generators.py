"""Seeded point sets and right-hand sides with the shapes of the paper's workloads.

The paper evaluates on UCI and scientific point sets of N = 11k..102k points in
d = 2..780 dimensions (Table 1), with a Gaussian kernel and a random dense W of
N x Q (Section 4.1). Those data sets are not available here; the synthetic
workloads below stand in for them: uniform points in the unit cube (low d,
like the scientific sets) and a Gaussian mixture (higher d, clustered like the
machine-learning sets).

Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64) so that
the oracle and the GPU path see identical inputs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


def uniform_points(n: int, d: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0, 1]^d, float64, shape (n, d)."""
    return np.random.default_rng(seed).random((n, d))


def gmm_points(n: int, d: int, n_comp: int, seed: int, lo: float = -5.0, hi: float = 5.0) -> np.ndarray:
    """n points from an equal-weight mixture of ``n_comp`` unit-covariance
    Gaussians in R^d whose means are uniform in [lo, hi]^d."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(lo, hi, size=(n_comp, d))
    labels = rng.integers(0, n_comp, size=n)
    return means[labels] + rng.standard_normal((n, d))


def normal_rhs(n: int, q: int, seed: int) -> np.ndarray:
    """Dense right-hand side W (n x q) with i.i.d. N(0, 1) float64 entries."""
    return np.random.default_rng(seed).standard_normal((n, q))


@dataclasses.dataclass(frozen=True)
class Workload:
    """Parameters of one HMatrix evaluation workload.

    ``admissibility`` is ``"hss"`` (every pair of siblings is far: weak
    admissibility), ``"geometric"`` (boxes far when the distance of their
    centroids exceeds ``eta`` times the larger of their radii) or ``"tau"``
    (``eta`` * gap between bounding boxes > sum of their diagonals).
    ``kernel`` is ``"gaussian"`` (exp(-r^2 / (2 h^2)), param = h), ``"imq"``
    (1 / sqrt(r^2 + c^2), param = c) or ``"invdist"`` (1 / r, 0 for coincident
    points; param unused).
    """
    name: str
    n: int
    d: int
    points: str            # "uniform" or "gmm"
    admissibility: str     # "hss" or "geometric"
    kernel: str            # "gaussian", "imq" or "invdist"
    kernel_param: float
    leaf_size: int
    tol: float
    max_rank: int
    q: int
    point_seed: int = 0
    rhs_seed: int = 1
    sample_seed: int = 2
    eta: float = 2.0
    gmm_components: int = 10
    tree: str = "kd"       # "kd" or "two_means"


def make_points(w: Workload) -> np.ndarray:
    if w.points == "uniform":
        return uniform_points(w.n, w.d, w.point_seed)
    if w.points == "gmm":
        return gmm_points(w.n, w.d, w.gmm_components, w.point_seed)
    raise ValueError(f"unknown point distribution {w.points!r}")


WORKLOADS = {
    # HSS, N=2048 uniform in [0,1]^3, Gaussian h=0.5, leaf 64, ID tol 1e-6, rank <= 64, Q=16.
    "hss_uniform3d_n2048": Workload("hss_uniform3d_n2048", 2048, 3, "uniform", "hss", "gaussian", 0.5,
                                    64, 1e-6, 64, 16),
    # H2 geometric, N=65536 in d=8 from a 10-component Gaussian mixture, Gaussian h=1,
    # leaf 128, ID tol 1e-5, rank <= 128, Q=256.
    "h2_gmm8d_n65536": Workload("h2_gmm8d_n65536", 65536, 8, "gmm", "geometric", "gaussian", 1.0,
                                128, 1e-5, 128, 256),
    # H2 geometric, N=262144 uniform in [0,1]^3, inverse multiquadric c=0.1, leaf 256,
    # ID tol 1e-7, rank <= 256, Q=512.
    "h2_imq3d_n262144": Workload("h2_imq3d_n262144", 262144, 3, "uniform", "geometric", "imq", 0.1,
                                 256, 1e-7, 256, 512),
    # Matrix-vector form of the comparison with SMASH: H2 geometric, N=262144 uniform in
    # [0,1]^3, kernel 1/r, leaf 256, ID tol 1e-6, rank <= 256, Q=1.
    "h2_invdist3d_n262144": Workload("h2_invdist3d_n262144", 262144, 3, "uniform", "geometric", "invdist", 0.0,
                                     256, 1e-6, 256, 1),
}


def reduced(w: Workload, n: int, q: Optional[int] = None, name: Optional[str] = None, **kw) -> Workload:
    """Same workload recipe at a smaller size (for tests the oracle finishes in seconds)."""
    return dataclasses.replace(w, n=n, q=w.q if q is None else q, name=name or f"{w.name}_n{n}", **kw)


def batch_workloads(count: int = 64, seed: int = 0, n_lo: int = 1024, n_hi: int = 32768) -> List[Workload]:
    """Many independent HMatrices of uneven size: N log-uniform in [n_lo, n_hi],
    d alternating 3 / 8, kernels alternating Gaussian h=1 / IMQ c=0.1,
    leaf size cycling 64, 128, 256, ID tol 1e-5, Q uniform in {1..64}."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        q = int(rng.integers(1, 65))
        d = 3 if k % 2 == 0 else 8
        kern, par = ("gaussian", 1.0) if k % 2 == 0 else ("imq", 0.1)
        leaf = (64, 128, 256)[k % 3]
        out.append(Workload(f"batch{k}", n, d, "uniform" if d == 3 else "gmm", "geometric", kern, par,
                            leaf, 1e-5, 256, q, point_seed=k, rhs_seed=1000 + k, sample_seed=2000 + k))
    return out


def serving_workloads(sizes=(16384, 32768, 65536, 131072, 262144, 524288, 524288, 1048576)) -> List[Workload]:
    """Resident matrices for the serving mode: d=3 uniform points, Gaussian h=0.5,
    geometric admissibility, leaf 256, ID tol 1e-6, rank <= 256."""
    return [Workload(f"serve{k}_n{n}", n, 3, "uniform", "geometric", "gaussian", 0.5, 256, 1e-6, 256, 256,
                     point_seed=k, rhs_seed=100 + k, sample_seed=200 + k) for k, n in enumerate(sizes)]
