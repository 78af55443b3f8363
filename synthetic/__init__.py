"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package holds input generation only: point sets, coefficient vectors and noise.
It performs none of the solver's arithmetic, so neither the CUDA path nor the CPU
oracle depends on the other through it.
"""
from .workloads import (  # noqa: F401
    BATCH_SIZES, batched_uneven, polar_grid, random_grid,
    Workload, WORKLOADS, jittered_grid, uniform_grid, complex_normal, noise_like, make_workload,
)
