"""Seeded synthetic sparse tensors and factor matrices.

This package only draws inputs: COO coordinates, values and dense factor
matrices.  It holds none of the arithmetic of spMTTKRP or of the FLYCOO
layout, and both the CUDA path and the FP64 oracle consume what it returns.
"""
from .tensors import (  # noqa: F401
    WORKLOADS,
    Workload,
    zipf_cdf,
    draw_zipf,
    make_coo,
    make_factors,
    make_workload,
    random_coo,
)
