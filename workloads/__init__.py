"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This package holds no arithmetic of the method: it only draws point sets and
right-hand sides, and names the workload parameters.
"""
from .generators import (  # noqa: F401
    Workload, WORKLOADS, uniform_points, gmm_points, normal_rhs, make_points,
    batch_workloads, serving_workloads, reduced,
)
