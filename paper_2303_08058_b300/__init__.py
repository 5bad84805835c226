"""B300-native FP64 FMM cell-interaction kernels on octrees of 8^3 sub-grids.

The public surface is the C ABI in include/ot.h (libotfmm.so) and this thin
binding: ``OTGrid`` (grid handle and every ABI call) and ``FMMInteractions``
(torch.autograd.Function from cell densities to Taylor coefficients).
"""
from ._lib import (EXPORTS, OT_PREC_DF64, OT_PREC_DF64_POINT_MASS, OT_PREC_FP64,  # noqa: F401
                   OT_SCHED_PER_SUBGRID, OT_SCHED_PERSISTENT, OTError, load)
from .fmm import (FP64_PROBE_FMA_PER_ROUND, FMMInteractions, OTGrid, fp64_fma_probe, launch_count,  # noqa: F401
                  potential_and_gradient)

__all__ = ["OTGrid", "FMMInteractions", "potential_and_gradient", "fp64_fma_probe", "FP64_PROBE_FMA_PER_ROUND", "launch_count", "OTError", "load",
           "OT_SCHED_PERSISTENT", "OT_SCHED_PER_SUBGRID", "OT_PREC_FP64", "OT_PREC_DF64_POINT_MASS", "OT_PREC_DF64", "EXPORTS"]
