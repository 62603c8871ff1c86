"""ctypes binding of libgosurf.so (include/gosurf.h): the same entry points, argument
marshalling only.  Every step of the computation runs in the library's CUDA kernels; this
module never computes anything itself and raises if the library cannot be loaded."""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

GS_LEVELS, GS_FEAT, GS_MLP_PARAMS, GS_NUM_LOSS = 4, 4, 1684, 6
GS_PREC_FP32, GS_PREC_BF16 = 0, 1
GS_PROP_BINS, GS_PROP_PARAMS = 32, 1473
GS_ARCH_COMPACT, GS_ARCH_PAPER = 0, 1
GS_COLOUR_FEAT, GS_PAPER_MLP_PARAMS = 6, 3109
STATUS = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_SHAPE", 3: "GS_ERR_ALIGN", 4: "GS_ERR_CUDA",
          5: "GS_ERR_DEVICE", 6: "GS_ERR_UNSUPPORTED"}

EXPORTS = ["gs_create", "gs_destroy", "gs_param_count", "gs_sample_rays", "gs_forward", "gs_backward",
           "gs_forward_backward", "gs_adam_step", "gs_query_sdf", "gs_query_sdf_backward", "gs_eikonal", "gs_sample_importance", "gs_extract_mesh", "gs_pose_apply", "gs_pose_backward", "gs_eikonal_pose_backward", "gs_proposal_sample", "gs_proposal_backward", "gs_voxel_index", "gs_sync_status",
           "gs_last_error", "gs_forward_backward_noalloc"]


class GsConfig(ctypes.Structure):
    _fields_ = [("dims", (ctypes.c_int32 * 3) * 4), ("voxel", ctypes.c_float * 4), ("origin", ctypes.c_float * 3),
                ("n_strat", ctypes.c_int32), ("n_guided", ctypes.c_int32), ("near_m", ctypes.c_float),
                ("far_m", ctypes.c_float), ("guide_half", ctypes.c_float), ("trunc", ctypes.c_float),
                ("kappa_fs", ctypes.c_float), ("lam", ctypes.c_float * 5), ("max_rays", ctypes.c_int32),
                ("max_smooth", ctypes.c_int32), ("delta_s", ctypes.c_float), ("precision", ctypes.c_int32),
                ("store_activations", ctypes.c_int32), ("prop_samples", ctypes.c_int32),
                ("prop_guided", ctypes.c_int32), ("imp_coarse", ctypes.c_int32), ("imp_steps", ctypes.c_int32),
                ("imp_per_step", ctypes.c_int32), ("arch", ctypes.c_int32)]


class GsFrames(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("rgb", ctypes.c_void_p),
                ("depth", ctypes.c_void_p), ("c2w", ctypes.c_void_p), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class GsBatch(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("N", ctypes.c_int32), ("P", ctypes.c_int32), ("pix", ctypes.c_void_p),
                ("origin", ctypes.c_void_p), ("dir", ctypes.c_void_p), ("rgb", ctypes.c_void_p),
                ("depth", ctypes.c_void_p), ("t", ctypes.c_void_p), ("cls", ctypes.c_void_p),
                ("xs", ctypes.c_void_p), ("eps", ctypes.c_void_p), ("valid", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("w", ctypes.c_void_p), ("dz", ctypes.c_void_p),
                ("eik", ctypes.c_void_p)]


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libgosurf.so")


def lib():
    """The loaded CUDA library; raises if it has not been built (there is no fallback)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libgosurf.so is not built ({path}); run __graft_entry__.build() or "
                                   "python paper_2206_14735_gb300/build.py")
            L = ctypes.CDLL(path)
            vp, i32, i64, u64, u32, f32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                          ctypes.c_uint32, ctypes.c_float)
            L.gs_create.restype = i32
            L.gs_create.argtypes = [ctypes.POINTER(GsConfig), ctypes.POINTER(vp)]
            L.gs_destroy.restype = None
            L.gs_destroy.argtypes = [vp]
            L.gs_param_count.restype = i64
            L.gs_param_count.argtypes = [ctypes.POINTER(GsConfig), ctypes.POINTER(i64)]
            L.gs_sample_rays.restype = i32
            L.gs_sample_rays.argtypes = [vp, ctypes.POINTER(GsFrames), u64, u32, ctypes.POINTER(GsBatch), vp]
            L.gs_forward.restype = i32
            L.gs_forward.argtypes = [vp, vp, vp, ctypes.POINTER(GsBatch), vp, vp, vp, vp, vp]
            L.gs_backward.restype = i32
            L.gs_backward.argtypes = [vp, vp, vp, ctypes.POINTER(GsBatch), vp, vp, vp]
            L.gs_forward_backward.restype = i32
            L.gs_forward_backward.argtypes = [vp, vp, vp, ctypes.POINTER(GsBatch), vp, vp, vp, vp]
            L.gs_adam_step.restype = i32
            L.gs_adam_step.argtypes = [vp, vp, vp, vp, vp, i64, i64, i32, f32, f32, f32, f32, f32, vp, vp]
            L.gs_query_sdf.restype = i32
            L.gs_query_sdf.argtypes = [vp, vp, vp, i32, vp, vp, vp]
            L.gs_proposal_sample.restype = i32
            L.gs_proposal_sample.argtypes = [vp, vp, vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp, vp, vp, vp]
            L.gs_proposal_backward.restype = i32
            L.gs_proposal_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.gs_eikonal.restype = i32
            L.gs_pose_apply.restype = i32
            L.gs_pose_apply.argtypes = [vp, vp, vp, i32, vp, vp]
            L.gs_pose_backward.restype = i32
            L.gs_pose_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.gs_eikonal_pose_backward.restype = i32
            L.gs_eikonal_pose_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            L.gs_extract_mesh.restype = i32
            L.gs_extract_mesh.argtypes = [vp, vp, vp, ctypes.c_float, i32, i32, i32, ctypes.c_float, vp, vp,
                                          ctypes.c_int64, vp, vp]
            L.gs_sample_importance.restype = i32
            L.gs_sample_importance.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp, vp]
            L.gs_eikonal.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.gs_query_sdf_backward.restype = i32
            L.gs_query_sdf_backward.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
            L.gs_voxel_index.restype = i32
            L.gs_voxel_index.argtypes = [vp, vp, i32, vp, vp]
            L.gs_sync_status.restype = i32
            L.gs_sync_status.argtypes = [vp]
            L.gs_forward_backward_noalloc.restype = i32
            L.gs_forward_backward_noalloc.argtypes = [ctypes.POINTER(GsConfig), vp, ctypes.POINTER(GsBatch), vp, vp,
                                                      vp, vp]
            L.gs_last_error.restype = ctypes.c_char_p
            L.gs_last_error.argtypes = [vp]
            _LIB = L
    return _LIB


class GoSurfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
