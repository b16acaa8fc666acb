"""GB300 HDG trace solver for the implicit linear rotating shallow-water step.

The numerics live in the CUDA library ``lib/libhdg.so`` (C ABI in
``include/hdg.h``); this package only builds it, loads it and marshals
arguments.  ``HDGSolver`` wraps one handle.
"""
from .solver import HDGSolver, MergedBatch, solve_batch_dev
from ._lib import HDGError, HDG_FP64, HDG_MIXED_FP32, HDG_MIXED_BF16, HDG_MIXED_FGMRES64, load, default_params

__all__ = ["HDGSolver", "MergedBatch", "solve_batch_dev", "HDGError", "HDG_FP64", "HDG_MIXED_FP32", "HDG_MIXED_BF16", "HDG_MIXED_FGMRES64", "load", "default_params"]
