"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the micromagnetic method: only the
parameter container (`Problem`), the named workloads and the counter-based
random numbers (SplitMix64) that draw the initial magnetisations.  Both the
CPU oracle and the CUDA path receive the same FP32-rounded arrays from here.
"""
from .rng import splitmix64, uniform01, random_unit_vectors, noisy_axis_vectors
from .problem import (Problem, GAMMA, MU0, PARAM_SCALARS, PARAM_VECTORS,
                      TERMS, config_c1, config_c2, config_c3, config_small,
                      batch_instances, serve_requests, stable_dt)

__all__ = [
    "splitmix64", "uniform01", "random_unit_vectors", "noisy_axis_vectors",
    "Problem", "GAMMA", "MU0", "PARAM_SCALARS", "PARAM_VECTORS", "TERMS",
    "config_c1", "config_c2", "config_c3", "config_small", "batch_instances",
    "serve_requests", "stable_dt",
]
