"""ctypes declarations of include/qvts.h.

Loads the in-tree `libqvts.so`; there is no fallback: when the library is
missing or fails to load the import raises, so nothing can silently run on
another path.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# QVTS_LIB=debug loads the bounds-checked debug build (libqvts_debug.so, the
# same ABI; device bounds checks report QV_ERR_BOUNDS instead of faulting)
LIB_PATH = os.path.join(PKG, "libqvts_debug.so" if os.environ.get("QVTS_LIB") == "debug" else "libqvts.so")

(QV_OK, QV_ERR_INVALID, QV_ERR_CUDA, QV_ERR_WORKSPACE, QV_ERR_TIMEOUT, QV_ERR_NOT_CONVERGED, QV_ERR_CAPACITY,
 QV_ERR_BOUNDS) = range(8)
STATUS_NAMES = {0: "QV_OK", 1: "QV_ERR_INVALID", 2: "QV_ERR_CUDA", 3: "QV_ERR_WORKSPACE",
                4: "QV_ERR_TIMEOUT", 5: "QV_ERR_NOT_CONVERGED", 6: "QV_ERR_CAPACITY", 7: "QV_ERR_BOUNDS"}
QV_NUM_ACTIONS = 5
QV_MAX_DEPTH = 6
QV_MAX_BEACONS = 126
QV_MAX_K = 64
QV_MAX_WIDTH = 2048
QV_NOALLOC_MAX_CELLS = 4096 * 1024
QV_F32, QV_F64 = 0, 1
QV_WEIGHT_FREQ, QV_WEIGHT_MARGINAL = 0, 1
QV_LEAF_FUSED, QV_LEAF_MATERIALISE = 0, 1
QV_DEEPEST_AUTO, QV_DEEPEST_STENCIL = 0, 1


class qv_model_t(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("pitch", C.c_int32), ("d_cell", C.c_void_p),
                ("num_beacons", C.c_int32), ("goal", C.c_int32), ("slip", C.c_float),
                ("accuracy", C.c_float), ("discount", C.c_float), ("d_cost", C.c_void_p),
                ("d_beacons", C.c_void_p), ("sense_range", C.c_int32)]


class qv_plan_params_t(C.Structure):
    _fields_ = [("depth", C.c_int32), ("K", C.c_int32), ("seed", C.c_uint64), ("episode", C.c_uint32),
                ("weight_mode", C.c_int32), ("leaf_mode", C.c_int32), ("d_replay", C.c_void_p),
                ("band_cells", C.c_int32), ("items_per_cta", C.c_int32), ("grid_ctas", C.c_int32),
                ("deadline_ms", C.c_double), ("deepest_form", C.c_int32)]


class qv_tune_t(C.Structure):
    _fields_ = [("band_cells", C.c_int32), ("items_per_cta", C.c_int32), ("ms", C.c_float)]


class qv_plan_result_t(C.Structure):
    _fields_ = [("action", C.c_int32), ("value", C.c_float), ("q", C.c_float * QV_NUM_ACTIONS),
                ("nodes_per_level", C.c_int32 * (QV_MAX_DEPTH + 1)), ("boundary_samples", C.c_int64),
                ("depth_reached", C.c_int32)]


class qv_level_view_t(C.Structure):
    _fields_ = [("cap", C.c_int32), ("d_count", C.c_void_p), ("d_parent", C.c_void_p),
                ("d_action", C.c_void_p), ("d_obs", C.c_void_p), ("d_weight", C.c_void_p),
                ("d_pz", C.c_void_p), ("d_value", C.c_void_p), ("d_R", C.c_void_p), ("d_UQ", C.c_void_p),
                ("d_nchild", C.c_void_p), ("d_samples", C.c_void_p), ("d_belief", C.c_void_p),
                ("d_leaf_arg", C.c_void_p)]


class qv_bounds_view_t(C.Structure):
    _fields_ = [("d_LV", C.c_void_p), ("d_HV", C.c_void_p), ("d_EV", C.c_void_p), ("d_LQ", C.c_void_p),
                ("d_HQ", C.c_void_p), ("d_EQ", C.c_void_p)]


class qv_bf_result_t(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("nodes", C.c_int32), ("stopped", C.c_int32),
                ("root_action", C.c_int32), ("U", C.c_float), ("L", C.c_float), ("H", C.c_float),
                ("E", C.c_int32), ("q", C.c_float * QV_NUM_ACTIONS), ("boundary_samples", C.c_int64)]


class qv_bf_view_t(C.Structure):
    _fields_ = [("max_nodes", C.c_int32)] + [(k, C.c_void_p) for k in (
        "d_parent", "d_action", "d_obs", "d_depth", "d_weight", "d_U", "d_L", "d_H", "d_E", "d_R", "d_UQ", "d_LQ",
        "d_HQ", "d_EQ", "d_first", "d_count", "d_belief", "d_expanded")]


class qv_launch_time_t(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("level", C.c_int32), ("ms", C.c_float)]


QV9_NUM_ACTIONS, QV9_NUM_OBS, QV9_MAX_DEPTH, QV9_MAX_K = 9, 16, 3, 16


class qv9_model_t(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("d_occ", C.c_void_p), ("goal", C.c_int32),
                ("slip", C.c_float), ("p_sensor", C.c_float), ("discount", C.c_float)]


class qv9_plan_result_t(C.Structure):
    _fields_ = [("action", C.c_int32), ("value", C.c_float), ("q", C.c_float * QV9_NUM_ACTIONS),
                ("nodes_per_level", C.c_int32 * (QV9_MAX_DEPTH + 1)), ("boundary_samples", C.c_int64)]


class qv9_level_view_t(C.Structure):
    _fields_ = [("count", C.c_int32)] + [(k, C.c_void_p) for k in (
        "parent", "action", "obs", "weight", "pz", "value", "belief", "R", "UQ")]


# every symbol include/qvts.h declares, with (restype, argtypes)
_vp, _i32, _sz = C.c_void_p, C.c_int32, C.c_size_t
_M = C.POINTER(qv_model_t)
_PP = C.POINTER(qv_plan_params_t)
SIGNATURES = {
    "qv_last_error": (C.c_char_p, []),
    "qv_version": (C.c_char_p, []),
    "qv_model_build": (C.c_int, [_i32, _i32, _i32, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "mdp_value_iterate_workspace_bytes": (_sz, [_M, _i32]),
    "mdp_value_iterate": (C.c_int, [_M, _i32, C.c_double, _i32, _i32, _vp, _vp, _vp, _sz,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_double), _vp]),
    "fib_value_iterate_workspace_bytes": (_sz, [_M, _i32]),
    "fib_value_iterate": (C.c_int, [_M, _i32, C.c_double, _i32, _i32, _vp, _vp, _vp, _sz,
                                    C.POINTER(_i32), C.POINTER(C.c_double), _vp]),
    "qv_pbvi_init": (C.c_int, [_M, _vp, _vp]),
    "qv_pbvi_expand": (C.c_int, [_M, _vp, _i32, _i32, C.c_uint64, _vp, _vp, _vp, _vp, _vp]),
    "qv_pbvi_create": (C.c_int, [_M, _i32, C.POINTER(_vp)]),
    "qv_pbvi_workspace_bytes": (_sz, [_vp]),
    "qv_pbvi_layout": (_i32, [_vp, _vp]),
    "qv_pbvi_set_points": (C.c_int, [_vp, _vp, _i32, _vp, _sz, _vp]),
    "qv_pbvi_backup": (C.c_int, [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "qv_pbvi_backup_fixed": (C.c_int, [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "qv_pbvi_value": (C.c_int, [_vp, _vp, _i32, _vp, _i32, _vp, _vp, _vp]),
    "qv_pbvi_check": (C.c_int, [_vp, _vp]),
    "qv_pbvi_destroy": (None, [_vp]),
    "mdp_value_iterate_checkpointed": (C.c_int, [_M, _i32, _i32, _vp, _vp, _vp, _vp, _sz, _vp]),
    "mdp_value_backward_workspace_bytes": (_sz, [_M, _i32]),
    "mdp_value_backward": (C.c_int, [_M, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "belief_predict": (C.c_int, [_M, _vp, _i32, _vp, _vp]),
    "belief_correct_workspace_bytes": (_sz, [_M]),
    "belief_correct": (C.c_int, [_M, _vp, _i32, _vp, _vp, _vp, _sz, _vp]),
    "belief_correct_noalloc": (C.c_int, [_M, _vp, _i32, _vp, _vp, _vp]),
    "leaf_value": (C.c_int, [_M, _vp, _vp, _i32, _vp, _vp]),
    "qv_plan_workspace_bytes": (_sz, [_i32, _M, _PP]),
    "qv_plan_create": (C.c_int, [_i32, _M, _vp, _vp, _PP, _vp, _sz, C.POINTER(_vp), _vp]),
    "qv_plan_run": (C.c_int, [_vp, _vp]),
    "qv_plan_set_episode_word": (C.c_int, [_vp, _vp]),
    "qv_plan_capture_graph": (C.c_int, [_vp, _vp]),
    "qv_plan_read": (C.c_int, [_vp, C.POINTER(qv_plan_result_t), _vp]),
    "qv_plan_readback_bytes": (_sz, [_vp]),
    "qv_plan_read_async": (C.c_int, [_vp, _vp, _vp]),
    "qv_plan_decode": (C.c_int, [_vp, _vp, C.POINTER(qv_plan_result_t)]),
    "qv_plan_destroy": (None, [_vp]),
    "qv_plan_profile": (C.c_int, [_vp, C.POINTER(qv_launch_time_t), _i32, C.POINTER(C.c_int32), _vp]),
    "qv_plan_bounds_workspace_bytes": (_sz, [_vp, _i32]),
    "qv_plan_bounds": (C.c_int, [_vp, _i32, _vp, _vp, _sz, _vp]),
    "qv_plan_bounds_view": (C.c_int, [_vp, _i32, _i32, _vp, C.POINTER(qv_bounds_view_t)]),
    "qv_bf_create": (C.c_int, [_M, _vp, _vp, _vp, _i32, _i32, C.c_uint64, C.c_uint32, _i32, _i32, C.POINTER(_vp)]),
    "qv_bf_workspace_bytes": (_sz, [_vp]),
    "qv_bf_reset": (C.c_int, [_vp, _vp, _vp, _sz, _vp]),
    "qv_bf_run": (C.c_int, [_vp, _i32, _vp]),
    "qv_bf_set_replay": (C.c_int, [_vp, _vp, _i32]),
    "qv_bf_read": (C.c_int, [_vp, C.POINTER(qv_bf_result_t), _vp]),
    "qv_bf_view": (C.c_int, [_vp, C.POINTER(qv_bf_view_t)]),
    "qv_bf_destroy": (None, [_vp]),
    "qv_plan_actions_device": (_vp, [_vp, C.POINTER(_i32)]),
    "qv_env_step": (C.c_int, [_M, _i32, _vp, _i32, _vp, C.c_uint64, _i32, _vp, _vp, _vp, _vp, _vp]),
    "qv_belief_update_batched_workspace_bytes": (_sz, [_M, _i32]),
    "qv_belief_update_batched": (C.c_int, [_M, _i32, _vp, _vp, _i32, _vp, _vp, _sz, _vp]),
    "qv_forward_sample_workspace_bytes": (_sz, [_M, _i32]),
    "qv_forward_sample": (C.c_int, [_M, _i32, _vp, _vp, _vp, _i32, C.c_uint64, C.c_uint32, _i32, _vp, _vp, _sz, _vp]),
    "qv_plan_grid": (_i32, [_vp]),
    "qv_plan_level": (C.c_int, [_vp, _i32, _i32, C.POINTER(qv_level_view_t)]),
    "qv_plan_autotune_workspace_bytes": (_sz, [_i32, _M, _PP]),
    "qv_plan_autotune": (C.c_int, [_i32, _M, _vp, _vp, _PP, _vp, _sz, _i32, C.POINTER(qv_tune_t),
                                   C.POINTER(qv_tune_t), _i32, C.POINTER(C.c_int32), _vp]),
    "qv_plan_tuning": (C.c_int, [_vp, C.POINTER(qv_tune_t)]),
    "qv_tune_clear": (None, []),
    "qv_tree_backward_workspace_bytes": (_sz, [_vp, _i32]),
    "qv_tree_backward": (C.c_int, [_vp, _i32, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "qv_tree_plan": (C.c_int, [_M, _vp, _vp, _PP, _vp, _sz, C.POINTER(qv_plan_result_t), _vp]),
    "qv_tree_plan_batched": (C.c_int, [_i32, _M, _vp, _vp, _PP, _vp, _sz, C.POINTER(qv_plan_result_t), _vp]),
    "qv9_create": (C.c_int, [C.POINTER(qv9_model_t), _i32, _i32, C.POINTER(_vp)]),
    "qv9_workspace_bytes": (_sz, [_vp]),
    "qv9_set_workspace": (C.c_int, [_vp, _vp, _sz, _vp]),
    "qv9_destroy": (None, [_vp]),
    "qv9_value_iterate": (C.c_int, [_vp, _i32, C.c_double, _i32, _i32, _vp, _vp, C.POINTER(_i32),
                                    C.POINTER(C.c_double), _vp]),
    "qv9_plan": (C.c_int, [_vp, _vp, _vp, C.c_uint64, C.c_uint32, C.POINTER(qv9_plan_result_t), _vp]),
    "qv9_level": (C.c_int, [_vp, _i32, C.POINTER(qv9_level_view_t)]),
}

_lib = None


def lib():
    """The loaded library (raises when libqvts.so is absent: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class QVError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().qv_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, where):
    if status != QV_OK:
        raise QVError(status, where)
