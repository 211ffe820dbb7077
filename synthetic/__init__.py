"""Seeded synthetic inputs for the ridge-path workloads.

This module only *generates problem data* (A, B, the lambda grid and request
shapes).  It holds none of the IHS-BIN arithmetic: no sketch, no Gram matrix,
no preconditioner, no basis, no path evaluation.  Both the FP64 oracle and the
CUDA path take its outputs as inputs, which is the only thing they share.

The paper's experiments use LIBSVM / CIFAR-10 data (Section 6) that are not
available here; the generators below stand in for them with the shapes, value
distributions and structure of the paper's workloads (dense over-determined,
sparse over/under-determined, matrix-valued right-hand sides).
"""
from .configs import (  # noqa: F401
    Problem,
    CONFIGS,
    make_problem,
    make_split,
    spectral_norm_sq,
    lambda_grid,
    to_bf16_bits,
    bf16_bits_to_f32,
    serving_requests,
)
