"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the benchmark.

This package only *builds inputs* (block-sparse Jacobians, right-hand sides and
small scalar test matrices).  It contains none of the preconditioner or Krylov
arithmetic; both the CUDA path and the oracle receive the arrays it returns.
"""
from .jacobian import (  # noqa: F401
    BSRSystem,
    cartesian,
    knn,
    config_system,
    config_slab,
    serving_mix,
    random_bsr,
    block_tridiag_chain,
    poisson1d_csr,
    poisson3d_csr,
    pressure_embedding,
    with_volume_constraint,
    CONFIG_NAMES,
)
