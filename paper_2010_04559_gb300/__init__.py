"""GB300 (sm_103a) library for the angular-multigrid-preconditioned DG
transport solver of Lathouwers & Perko (arXiv 2010.04559).

The compute path is libamgt.so (CUDA kernels behind the C ABI of
include/amgt.h); this package only builds and binds it.
"""
from ._capi import (AMGT_OK, AMGT_ERR_ARG, AMGT_ERR_CUDA, AMGT_ERR_NOMEM, AMGT_ERR_NOT_CONVERGED,
                    AMGT_ERR_BREAKDOWN, AMGT_ERR_NAN, AMGT_ERR_DEVICE_TIMEOUT, AMGT_ERR_STATE,
                    AMGT_ERR_UNSUPPORTED, AMGT_F64_SPLIT, AMGT_F32_TC3, AMGT_KT_TC3, AMGT_KT_TC3_PREP,
                    AMGT_TUNE_F32_SCATTER, AMGT_TUNE_TEST_SWEEP_HOLD, AMGT_TUNE_COARSE_F64,
                    AMGT_KT_SPLIT_AUX, AMGT_KT_SPLIT_TC, AMGT_TUNE_FP64_SCATTER,
                    AMGT_TUNE_SPLIT_ROWS, AMGT_TUNE_SWEEP_KERNEL, AMGT_TUNE_GS_KERNEL,
                    AMGT_TUNE_SWEEP_GROUP, AMGT_TUNE_SWEEP_STAGES, AMGT_TUNE_GS_GRID_BLOCKS,
                    AMGT_TUNE_GS_CLUSTER, AMGT_TUNE_GS_FORM,
                    AMGT_KRYLOV_BICGSTAB, AMGT_KRYLOV_GMRES, AMGT_F32, AMGT_F32_BF16TC, AMGT_F64, AMGT_MODE_F64, AMGT_MODE_MIXED,
                    AMGT_KT_APPLY_L, AMGT_KT_COARSE_GS, AMGT_KT_SCATTER_PREP,
                    AMGT_KT_SCATTER_F32, AMGT_KT_SCATTER_F64, AMGT_KT_SCATTER_TC, AMGT_KT_SWEEP, AMGT_PREC_MG,
                    AMGT_PREC_NONE, AMGT_PREC_SWEEP, AMGT_TUNE_GRAPHS, AMGT_TUNE_KERNEL_TIMERS, AmgtError,
                    Context,
                    EXPORTS, amgt_query_launches, amgt_setup_batch, amgt_solve_batch,
                    context_from_problem)

__all__ = ["Context", "context_from_problem", "AmgtError", "EXPORTS", "AMGT_F64", "AMGT_F32",
           "AMGT_F32_BF16TC", "AMGT_PREC_NONE", "AMGT_PREC_SWEEP", "AMGT_PREC_MG",
           "AMGT_MODE_F64", "AMGT_MODE_MIXED", "amgt_query_launches", "AMGT_TUNE_KERNEL_TIMERS",
           "AMGT_TUNE_GRAPHS", "amgt_solve_batch", "amgt_setup_batch", "AMGT_KRYLOV_GMRES",
           "AMGT_KRYLOV_BICGSTAB",
           "AMGT_KT_SWEEP", "AMGT_KT_APPLY_L", "AMGT_KT_SCATTER_PREP", "AMGT_KT_SCATTER_TC",
           "AMGT_KT_SCATTER_F32", "AMGT_KT_SCATTER_F64", "AMGT_KT_COARSE_GS",
           "AMGT_F64_SPLIT", "AMGT_F32_TC3", "AMGT_KT_TC3", "AMGT_KT_TC3_PREP",
           "AMGT_TUNE_F32_SCATTER", "AMGT_TUNE_TEST_SWEEP_HOLD", "AMGT_TUNE_COARSE_F64",
           "AMGT_KT_SPLIT_TC", "AMGT_KT_SPLIT_AUX", "AMGT_TUNE_FP64_SCATTER", "AMGT_TUNE_SPLIT_ROWS", "AMGT_TUNE_SWEEP_KERNEL",
           "AMGT_TUNE_GS_KERNEL", "AMGT_TUNE_SWEEP_GROUP", "AMGT_TUNE_SWEEP_STAGES",
           "AMGT_TUNE_GS_GRID_BLOCKS", "AMGT_TUNE_GS_CLUSTER", "AMGT_TUNE_GS_FORM", "AMGT_OK",
           "AMGT_ERR_ARG",
           "AMGT_ERR_CUDA", "AMGT_ERR_NOMEM", "AMGT_ERR_NOT_CONVERGED", "AMGT_ERR_BREAKDOWN",
           "AMGT_ERR_NAN", "AMGT_ERR_DEVICE_TIMEOUT", "AMGT_ERR_STATE", "AMGT_ERR_UNSUPPORTED"]
