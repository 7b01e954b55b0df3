"""Seeded synthetic inputs shared by the oracle-side tests, the CUDA-side tests and the benchmark.

This package only *generates inputs* (grid descriptions, velocity/density models, source and receiver
positions).  It contains none of the LOSS arithmetic: no spline solve, no boundary closure, no
derivative, no time stepping and no source wavelet evaluation.  Both the FP64 oracle and the CUDA path
receive the arrays produced here unchanged.
"""
from .workloads import (  # noqa: F401
    Workload,
    WORKLOADS,
    acoustic2d_small,
    acoustic2d_gradient_case,
    elastic3d_gradient_case,
    mean_model,
    acoustic2d_layered,
    elastic3d_homogeneous,
    elastic3d_heterogeneous,
    elastic3d_double_layer,
    DOUBLE_LAYER_UPPER,
    DOUBLE_LAYER_DEEPER,
    batched_shots,
    gaussian_pulse_2d,
    random_field,
    scaled,
)
