"""GB300 (sm_103a) library for the angular-multigrid-preconditioned DG
transport solver of Lathouwers & Perko (arXiv 2010.04559).

The compute path is libamgt.so (CUDA kernels behind the C ABI of
include/amgt.h); this package only builds and binds it.
"""
from ._capi import (AMGT_F64_SPLIT, AMGT_KT_SPLIT_AUX, AMGT_KT_SPLIT_TC, AMGT_TUNE_FP64_SCATTER,
                    AMGT_TUNE_SPLIT_ROWS, AMGT_TUNE_SWEEP_KERNEL, AMGT_TUNE_GS_KERNEL,
                    AMGT_TUNE_SWEEP_GROUP, AMGT_TUNE_SWEEP_STAGES, AMGT_TUNE_GS_GRID_BLOCKS,
                    AMGT_TUNE_GS_CLUSTER,
                    AMGT_KRYLOV_BICGSTAB, AMGT_KRYLOV_GMRES, AMGT_F32, AMGT_F32_BF16TC, AMGT_F64, AMGT_MODE_F64, AMGT_MODE_MIXED,
                    AMGT_KT_APPLY_L, AMGT_KT_COARSE_GS, AMGT_KT_SCATTER_PREP,
                    AMGT_KT_SCATTER_F32, AMGT_KT_SCATTER_F64, AMGT_KT_SCATTER_TC, AMGT_KT_SWEEP, AMGT_PREC_MG,
                    AMGT_PREC_NONE, AMGT_PREC_SWEEP, AMGT_TUNE_GRAPHS, AMGT_TUNE_KERNEL_TIMERS, AmgtError,
                    Context,
                    EXPORTS, amgt_query_launches, amgt_solve_batch, context_from_problem)

__all__ = ["Context", "context_from_problem", "AmgtError", "EXPORTS", "AMGT_F64", "AMGT_F32",
           "AMGT_F32_BF16TC", "AMGT_PREC_NONE", "AMGT_PREC_SWEEP", "AMGT_PREC_MG",
           "AMGT_MODE_F64", "AMGT_MODE_MIXED", "amgt_query_launches", "AMGT_TUNE_KERNEL_TIMERS",
           "AMGT_TUNE_GRAPHS", "amgt_solve_batch", "AMGT_KRYLOV_GMRES", "AMGT_KRYLOV_BICGSTAB",
           "AMGT_KT_SWEEP", "AMGT_KT_APPLY_L", "AMGT_KT_SCATTER_PREP", "AMGT_KT_SCATTER_TC",
           "AMGT_KT_SCATTER_F32", "AMGT_KT_SCATTER_F64", "AMGT_KT_COARSE_GS",
           "AMGT_F64_SPLIT", "AMGT_KT_SPLIT_TC", "AMGT_KT_SPLIT_AUX", "AMGT_TUNE_FP64_SCATTER", "AMGT_TUNE_SPLIT_ROWS", "AMGT_TUNE_SWEEP_KERNEL",
           "AMGT_TUNE_GS_KERNEL", "AMGT_TUNE_SWEEP_GROUP", "AMGT_TUNE_SWEEP_STAGES",
           "AMGT_TUNE_GS_GRID_BLOCKS", "AMGT_TUNE_GS_CLUSTER"]
