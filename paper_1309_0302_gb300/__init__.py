"""GB300 (sm_103a) GoDec-BRP: Python binding of the C ABI in include/godec.h.

Every step of Algorithm 1 runs in the CUDA library ``_lib/libgodec.so``; this
module only marshals arguments.  PyTorch provides device memory and streams.
There is no CPU fallback: if the library cannot be loaded, calls raise.
"""
from ._binding import (  # noqa: F401
    GoDec, GoDecBatch, GreBsmo, NaiveGoDec, LinGoDec, naive_columns, mse_train, GodecError, library, mul_ZB, mul_ZtC, run_host, hard_threshold, header_symbols, backward, batch_budgets, tc_geometry,
    PREC_FP32, PREC_BF16_REFINE, FLAG_NO_REFINE, FLAG_FP64_FACTOR, FLAG_SPARSE_FIRST, FLAG_DENSE_FIRST, MAX_RANK, BATCH_NO_TUNE,
)
from .autograd import UnrolledGoDec, unrolled_godec  # noqa: F401
