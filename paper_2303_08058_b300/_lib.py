"""ctypes binding of libotfmm.so: argument marshalling only.

Every computation runs in the library's CUDA kernels.  If the shared library
is missing this module raises ImportError: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libotfmm.so")

OT_OK, OT_EINVAL, OT_ENOMEM, OT_ECUDA, OT_ETIMEOUT, OT_ESTATE, OT_ENOTSUP, OT_EDEVICE = range(8)
STATUS_NAMES = ["OT_OK", "OT_EINVAL", "OT_ENOMEM", "OT_ECUDA", "OT_ETIMEOUT", "OT_ESTATE", "OT_ENOTSUP",
                "OT_EDEVICE"]
OT_SCHED_PERSISTENT, OT_SCHED_PER_SUBGRID = 0, 1
OT_PREC_FP64, OT_PREC_DF64_POINT_MASS, OT_PREC_DF64 = 0, 1, 2

# every entry point declared in include/ot.h
EXPORTS = ["ot_grid_create", "ot_grid_destroy", "ot_grid_info", "ot_moments", "ot_moments_backward",
           "ot_multipole_interactions", "ot_monopole_interactions", "ot_interactions",
           "ot_interactions_backward", "ot_set_schedule", "ot_autotune", "ot_grid_check",
           "ot_fp64_fma_probe", "ot_multipole_interactions_noalloc", "ot_l2l", "ot_l2l_backward",
           "ot_set_deterministic", "ot_set_precision", "ot_completion_study",
           "ot_moments_com", "ot_interactions_com", "ot_interactions_backward_com", "ot_l2l_com",
           "ot_l2l_com_backward", "ot_launch_count", "ot_last_error"]


class OTError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class GridDesc(ctypes.Structure):
    _fields_ = [("n_subgrids", ctypes.c_int32), ("level", ctypes.c_void_p), ("coord", ctypes.c_void_p),
                ("is_leaf", ctypes.c_void_p), ("h0", ctypes.c_double), ("stencil_c", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class GridInfo(ctypes.Structure):
    _fields_ = [("n_subgrids", ctypes.c_int32), ("n_virtual", ctypes.c_int32), ("max_level", ctypes.c_int32),
                ("far_offsets", ctypes.c_int32), ("near_offsets", ctypes.c_int32),
                ("root_offsets", ctypes.c_int32), ("pairs_multipole", ctypes.c_int64),
                ("pairs_monopole", ctypes.c_int64), ("pairs_virtual", ctypes.c_int64),
                ("pairs_angular", ctypes.c_int64), ("lanes_fwd", ctypes.c_int64), ("flops_fwd", ctypes.c_int64),
                ("flops_adj", ctypes.c_int64), ("ops_fwd", ctypes.c_int64), ("ops_adj", ctypes.c_int64),
                ("schedule", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("graphs_enabled", ctypes.c_int32),
                ("flops_fwd_com", ctypes.c_int64), ("flops_adj_com", ctypes.c_int64),
                ("pairs_refined", ctypes.c_int64), ("pairs_padded_fwd", ctypes.c_int64),
                ("chunked_subgrids", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("fp64_ops_fwd", ctypes.c_int64), ("fp64_ops_adj", ctypes.c_int64),
                ("fp64_ops_fwd_multi", ctypes.c_int64), ("ops_fwd_multi", ctypes.c_int64),
                ("fp64_ops_adj_multi", ctypes.c_int64), ("ops_adj_multi", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class CompletionStats(ctypes.Structure):
    _fields_ = [("wall_ms", ctypes.c_double), ("mean_latency_us", ctypes.c_double),
                ("max_latency_us", ctypes.c_double), ("launches", ctypes.c_int64)]


_lib = None


def load():
    """Load libotfmm.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libotfmm.so not built at {LIB_PATH}; run python -m paper_2303_08058_b300.build")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, S = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
    sig = {
        "ot_grid_create": [ctypes.POINTER(GridDesc), P, ctypes.POINTER(P)],
        "ot_grid_destroy": [P],
        "ot_grid_info": [P, ctypes.POINTER(GridInfo)],
        "ot_moments": [P, P, P, P, P],
        "ot_moments_backward": [P, P, P, P, P],
        "ot_multipole_interactions": [P, P, P, P, P, P],
        "ot_monopole_interactions": [P, P, P, P],
        "ot_interactions": [P, P, P, P, P, P],
        "ot_interactions_backward": [P, P, P, P, P],
        "ot_set_schedule": [P, I, I, I, I],
        "ot_autotune": [P, P, P, P, P, P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_double)],
        "ot_grid_check": [P, P],
        "ot_fp64_fma_probe": [P, I, I, I, P],
        "ot_multipole_interactions_noalloc": [P, P, P, P, P],
        "ot_l2l": [P, P, P],
        "ot_l2l_backward": [P, P, P],
        "ot_set_deterministic": [P, I],
        "ot_set_precision": [P, I],
        "ot_completion_study": [P, P, P, P, P, I, I, ctypes.c_double, ctypes.POINTER(CompletionStats)],
        "ot_moments_com": [P, P, P, P, P, P],
        "ot_interactions_com": [P, P, P, P, P, P, P],
        "ot_interactions_backward_com": [P, P, P, P, P, P],
        "ot_l2l_com": [P, P, P, P],
        "ot_l2l_com_backward": [P, P, P, P],
        "ot_launch_count": [ctypes.POINTER(ctypes.c_int64)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = S
    lib.ot_last_error.argtypes = []
    lib.ot_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != OT_OK:
        raise OTError(status, load().ot_last_error().decode())
