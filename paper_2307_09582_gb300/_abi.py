"""ctypes declarations of the C ABI in include/glu.h (structs, enums, prototypes).

Loading fails loudly when libglu.so has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libglu.so")

GLU_OK = 0
GLU_ERR_INVALID_ARG = -1
GLU_ERR_SHAPE = -2
GLU_ERR_UNSUPPORTED = -3
GLU_ERR_WORKSPACE = -4
GLU_ERR_CUDA = -5
GLU_ERR_DEVICE_CHECK = -6
GLU_ERR_TIMEOUT = -7

GLU_U8, GLU_F16, GLU_F32 = 0, 1, 2
GLU_W_F32, GLU_W_F16, GLU_W_UNORM16 = 0, 1, 2
GLU_MODE_FAST, GLU_MODE_GNU, GLU_MODE_EXACT = 0, 1, 2
GLU_JOINT_STRICT, GLU_JOINT_PAPER = 0, 1
GLU_DOWN_GRID, GLU_DOWN_BOX = 0, 1
GLU_MAX_ITERS = 32
(GLU_OP_DOWNSAMPLE, GLU_OP_OPTIMIZE, GLU_OP_APPLY, GLU_OP_THETA_DECODE, GLU_OP_JOINT,
 GLU_OP_LS_JOINT, GLU_OP_LS_UPDATE, GLU_OP_APPLY_BACKWARD, GLU_OP_APPLY_BACKWARD_PLAN) = range(9)


class GluImage(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("h", ctypes.c_int32), ("w", ctypes.c_int32),
                ("c", ctypes.c_int32), ("dtype", ctypes.c_int32), ("pitch", ctypes.c_int64)]


class GluTheta(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("H", ctypes.c_int32),
                ("W", ctypes.c_int32), ("scale", ctypes.c_int32), ("S", ctypes.c_int32),
                ("wfmt", ctypes.c_int32)]


class GluParams(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int32), ("eps", ctypes.c_float), ("tau", ctypes.c_float),
                ("N", ctypes.c_int32), ("mode", ctypes.c_int32), ("joint", ctypes.c_int32),
                ("connectivity", ctypes.c_int32)]


class GluJointStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32),
                ("n_large", ctypes.c_int32 * GLU_MAX_ITERS),
                ("components", ctypes.c_int32 * GLU_MAX_ITERS),
                ("accepted", ctypes.c_int32 * GLU_MAX_ITERS),
                ("rolled_back", ctypes.c_int32 * GLU_MAX_ITERS),
                ("residual", ctypes.c_double * (GLU_MAX_ITERS + 1)),
                ("searched", ctypes.c_int64 * GLU_MAX_ITERS),
                ("multi_kernel_lists", ctypes.c_uint32)]


class GluLsStats(ctypes.Structure):
    _fields_ = [("R0", ctypes.c_double),
                ("residual", ctypes.c_double * GLU_MAX_ITERS),
                ("iterations", ctypes.c_int32),
                ("kept", ctypes.c_int32)]


class GluBatchItem(ctypes.Structure):
    _fields_ = [("hr", GluImage), ("lr", GluImage), ("theta", GluTheta),
                ("err_map", ctypes.c_void_p)]


GLU_VIDEO_MAX_SLOTS = 256
GLU_VIDEO_MAX_OPS = 4


class GluLrOp(ctypes.Structure):
    _fields_ = [("filter", ctypes.c_int32), ("saturation", ctypes.c_float),
                ("gamma", ctypes.c_float)]


class GluVideoDesc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("hr_dtype", ctypes.c_int32),
                ("out_dtype", ctypes.c_int32), ("scale", ctypes.c_int32), ("params", GluParams),
                ("wfmt", ctypes.c_int32), ("n_ops", ctypes.c_int32),
                ("ops", GluLrOp * GLU_VIDEO_MAX_OPS), ("overlap", ctypes.c_int32)]
GLU_TUNE_SEARCH, GLU_TUNE_APPLY = 0, 1

_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f = ctypes.c_float

PROTOTYPES = {
    "glu_params_default": (None, [_P(GluParams)]),
    "glu_downsample": (ctypes.c_int, [_P(GluImage), _i32, _i32, _P(GluImage), _vp]),
    "glu_optimize": (ctypes.c_int, [_P(GluImage), _P(GluImage), _P(GluParams), _P(GluTheta), _vp, _vp]),
    "glu_joint_optimize": (ctypes.c_int, [_P(GluImage), _i32, _P(GluParams), _P(GluImage),
                                          _P(GluTheta), _vp, _P(GluJointStats), _vp,
                                          ctypes.c_size_t, _vp]),
    "glu_joint_workspace_size": (ctypes.c_size_t, [_i32, _i32, _i32, _P(GluParams)]),
    "glu_optimize_batched": (ctypes.c_int, [_P(GluBatchItem), _i32, _P(GluParams), _vp]),
    "glu_joint_optimize_batched": (ctypes.c_int, [_P(GluBatchItem), _i32, _P(GluParams),
                                                  _P(GluJointStats), _vp, ctypes.c_size_t, _vp]),
    "glu_joint_batched_workspace_size": (ctypes.c_size_t, [_P(GluBatchItem), _i32,
                                                           _P(GluParams)]),
    "glu_apply": (ctypes.c_int, [_P(GluTheta), _P(GluImage), _P(GluImage), _vp]),
    "glu_theta_decode": (ctypes.c_int, [_P(GluTheta), _vp, _vp, _vp, _vp]),
    "glu_workspace_size": (ctypes.c_size_t, [_i32, _i32, _i32, _i32, _P(GluParams)]),
    "glu_apply_backward": (ctypes.c_int, [_P(GluTheta), _P(GluImage), _P(GluImage), _P(GluImage),
                                          _vp, _vp]),
    "glu_apply_backward_workspace_size": (ctypes.c_size_t, [_P(GluTheta), _i32]),
    "glu_test_set_wait_limit": (ctypes.c_int, [ctypes.c_uint64]),
    "glu_test_joint_graph_count": (_i64, []),
    "glu_test_joint_argmax_log": (ctypes.c_int, [_vp, _i64]),
    "glu_apply_backward_plan_size": (ctypes.c_size_t, [_P(GluTheta)]),
    "glu_apply_backward_plan": (ctypes.c_int, [_P(GluTheta), _vp, ctypes.c_size_t, _vp]),
    "glu_apply_backward_planned": (ctypes.c_int, [_P(GluTheta), _vp, _P(GluImage), _P(GluImage),
                                                  _P(GluImage), _vp, _vp]),
    "glu_ls_update_workspace_size": (ctypes.c_size_t, [_P(GluTheta)]),
    "glu_ls_update": (ctypes.c_int, [_P(GluImage), _P(GluTheta), _P(GluImage), _P(GluImage), _vp,
                                     ctypes.c_size_t, _vp]),
    "glu_ls_joint_workspace_size": (ctypes.c_size_t, [_i32, _i32, _i32, _P(GluParams)]),
    "glu_ls_joint_optimize": (ctypes.c_int, [_P(GluImage), _i32, _P(GluParams), _P(GluImage),
                                             _P(GluTheta), _vp, _P(GluLsStats), _vp,
                                             ctypes.c_size_t, _vp]),
    "glu_apply_backward_ws": (ctypes.c_int, [_P(GluTheta), _P(GluImage), _P(GluImage),
                                             _P(GluImage), _vp, _vp, ctypes.c_size_t, _vp]),
    "glu_joint_decisions": (ctypes.c_int64, [_vp, ctypes.c_size_t, _i32, _i32, _i32, _P(GluParams),
                                             _vp, _i64, _vp]),
    "glu_joint_profile": (ctypes.c_int, [_i32]),
    "glu_joint_profile_read": (ctypes.c_int, [_P(ctypes.c_float), _P(_i32)]),
    "glu_video_workspace_size": (ctypes.c_size_t, [_P(GluVideoDesc)]),
    "glu_video_create": (ctypes.c_int, [_P(GluVideoDesc), _vp, ctypes.c_size_t, _P(_vp)]),
    "glu_video_bind": (ctypes.c_int, [_vp, _i32, _vp, _P(_vp)]),
    "glu_video_launch": (ctypes.c_int, [_vp, _i32, _vp]),
    "glu_video_run": (ctypes.c_int, [_vp, _vp, _P(_vp), _vp]),
    "glu_video_views": (ctypes.c_int, [_vp, _P(GluImage), _P(GluImage), _P(GluTheta)]),
    "glu_video_destroy": (ctypes.c_int, [_vp]),
    "glu_tune_mode": (ctypes.c_int, [_i32]),
    "glu_tune_variants": (_i32, [_i32]),
    "glu_tune_variant_name": (ctypes.c_int, [_i32, _i32, ctypes.c_char_p, _i32]),
    "glu_tune_force": (ctypes.c_int, [_i32, _i32]),
    "glu_tune_export": (_i64, [ctypes.c_char_p, _i64]),
    "glu_tune_import": (ctypes.c_int, [ctypes.c_char_p]),
    "glu_tune_clear": (ctypes.c_int, []),
    "glu_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "glu_device_status": (ctypes.c_int, [_vp]),
    "glu_version": (ctypes.c_char_p, []),
    "glu_fx_filter3": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i64, _vp, _i64, _i32, _vp]),
    "glu_fx_point": (ctypes.c_int, [_vp, _i32, _i32, _i64, _vp, _i64, _f, _f, _vp]),
    "glu_apply_lrop": (ctypes.c_int, [_P(GluTheta), _P(GluImage), _P(GluLrOp), _P(GluImage),
                                      _P(GluImage), _vp]),
    "glu_fx_filter3_u8": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i64, _vp, _i64, _i32, _vp]),
    "glu_pipeline_host_workspace_size": (ctypes.c_size_t, [_i32, _i32, _i32, _P(GluParams)]),
    "glu_pipeline_host": (ctypes.c_int, [_vp, _i32, _i32, _i32, _P(GluParams), _i32, _f, _f,
                                         _vp, _vp, ctypes.c_size_t, _vp]),
}

_LIB = None


class GluError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {code} ({status_string(code)})")
        self.code = code


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libglu.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libglu.so not found at {p}: the CUDA library must be built first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    for name, (res, args) in PROTOTYPES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _LIB = lib
    return lib


def status_string(code: int) -> str:
    names = {0: "GLU_OK", -1: "GLU_ERR_INVALID_ARG", -2: "GLU_ERR_SHAPE",
             -3: "GLU_ERR_UNSUPPORTED", -4: "GLU_ERR_WORKSPACE", -5: "GLU_ERR_CUDA",
             -6: "GLU_ERR_DEVICE_CHECK", -7: "GLU_ERR_TIMEOUT"}
    return names.get(code, "GLU_ERR_UNKNOWN")


def check(fn: str, code: int) -> int:
    if code != GLU_OK:
        raise GluError(fn, code)
    return code
