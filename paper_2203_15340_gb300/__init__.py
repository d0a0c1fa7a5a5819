"""GB300-native solver for the indefinite least squares problem.

The numerical work lives in the CUDA library ``libils.so`` (sources in
``csrc/``, C ABI in ``include/ils.h``); ``binding`` marshals arguments to it.
"""
from .binding import (  # noqa: F401
    BatchSolver, ILSError, Solver, WarmStartNet, ils_info, ils_options, lib, options, status_string,
    ILS_OK, ILS_ERR_INVALID_ARG, ILS_ERR_NOT_SPD, ILS_ERR_NO_CONVERGENCE, ILS_ERR_NONFINITE,
    ILS_ERR_TIMEOUT, ILS_ERR_CUDA, ILS_ERR_OOM, ILS_SP, ILS_SP_RK_RGS, ILS_SP_SCD,
    ILS_FP64, ILS_FP32_REFINE, ILS_BF16_REFINE, ILS_GRAM_FP64, ILS_GRAM_SPLIT,
    ILS_ROUTE_AUTO, ILS_ROUTE_EXPLICIT, ILS_ROUTE_MATRIX_FREE, MAT_GRAM1, MAT_GRAM2, MAT_CHOL, MAT_P, MAT_B,
    ILS_STOP_RELRES, ILS_STOP_PAPER_RR, ILS_STOP_ERR_BOUND, kernel_launches, tuned_shape,
)
