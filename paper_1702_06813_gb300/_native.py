"""ctypes declarations of librendermap.so (include/rendermap.h), same names as the C ABI.

Argument marshalling only. Loading fails loudly when the library has not been built: there
is no fallback implementation of any step.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librendermap.so")

RM_OK, RM_EINVAL, RM_ENOMEM, RM_ECUDA, RM_EOVERFLOW, RM_ETIMEOUT, RM_ENOTCONV = range(7)
RM_PINHOLE, RM_RAYTABLE = 0, 1
STATUS_NAMES = {0: "RM_OK", 1: "RM_EINVAL", 2: "RM_ENOMEM", 3: "RM_ECUDA", 4: "RM_EOVERFLOW",
                5: "RM_ETIMEOUT", 6: "RM_ENOTCONV"}


class rm_intrinsics(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("az0", ctypes.c_float),
                ("az_step", ctypes.c_float), ("el0", ctypes.c_float), ("el_step", ctypes.c_float),
                ("near_m", ctypes.c_float), ("far_m", ctypes.c_float), ("rays", ctypes.c_void_p)]


class rm_scan(ctypes.Structure):
    _fields_ = [("intr", rm_intrinsics), ("depth", ctypes.c_void_p), ("cls", ctypes.c_void_p)]


class rm_problem(ctypes.Structure):
    _fields_ = [("scan", rm_scan), ("pose", ctypes.c_void_p)]


class rm_cost_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("w_fofo", ctypes.c_float), ("w_fofu", ctypes.c_float),
                ("w_fufo", ctypes.c_float)]


class rm_cost_out(ctypes.Structure):
    _fields_ = [("counts", ctypes.c_void_p), ("e_table", ctypes.c_void_p), ("e_ls", ctypes.c_void_p),
                ("grad", ctypes.c_void_p), ("jtj", ctypes.c_void_p)]


class rm_tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("bin_capacity", ctypes.c_int32), ("wave_poses", ctypes.c_int32),
                ("async_status", ctypes.c_int32), ("wait_log2", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class rm_align_params(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("lambda0", ctypes.c_double), ("lambda_up", ctypes.c_double),
                ("lambda_down", ctypes.c_double), ("step_tol", ctypes.c_double)]


class rm_align_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("e_ls_initial", ctypes.c_double), ("e_ls_final", ctypes.c_double),
                ("e_table_initial", ctypes.c_int64), ("e_table_final", ctypes.c_int64)]


class rm_icp_out(ctypes.Structure):
    _fields_ = [("n_assoc", ctypes.c_void_p), ("cost_l1", ctypes.c_void_p), ("e2", ctypes.c_void_p),
                ("jte", ctypes.c_void_p), ("jtj", ctypes.c_void_p)]


class rm_icp_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_float), ("max_iters", ctypes.c_int32), ("step_tol", ctypes.c_double)]


class rm_icp_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("n_assoc", ctypes.c_int64),
                ("cost_l1_initial", ctypes.c_double), ("cost_l1_final", ctypes.c_double)]


class rm_meshify_params(ctypes.Structure):
    _fields_ = [("max_range", ctypes.c_float), ("max_edge", ctypes.c_float), ("step", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class rm_dfo_params(ctypes.Structure):
    _fields_ = [("nm_iters", ctypes.c_int32), ("cd_iters", ctypes.c_int32), ("nm_step", ctypes.c_double),
                ("nm_tol", ctypes.c_double), ("cd_step", ctypes.c_double), ("cd_tol", ctypes.c_double),
                ("scale_t", ctypes.c_double), ("scale_r", ctypes.c_double), ("method", ctypes.c_int32),
                ("powell_iters", ctypes.c_int32), ("powell_step", ctypes.c_double),
                ("powell_tol", ctypes.c_double)]


class rm_dfo_report(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_int32), ("nm_iters", ctypes.c_int32), ("nm_shrinks", ctypes.c_int32),
                ("cd_iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("powell_iters", ctypes.c_int32),
                ("e_table_initial", ctypes.c_int64), ("e_table_final", ctypes.c_int64)]


class rm_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_SIGS = {
    "rm_map_create": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.c_int64, ctypes.POINTER(_P)]),
    "rm_map_destroy": (None, [_P]),
    "rm_map_info": (ctypes.c_int, [_P, _P, _P, _P]),
    "rm_map_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(rm_tuning)]),
    "rm_map_set_vertex_normals": (ctypes.c_int, [_P, _P, _P, _P]),
    "rm_map_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(rm_tuning)]),
    "rm_render_depth": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(rm_intrinsics), _P, _P, _P, _P]),
    "rm_cost": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P, ctypes.c_int32,
                               ctypes.POINTER(rm_cost_params), ctypes.POINTER(rm_cost_out), _P]),
    "rm_cost_grad": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P, ctypes.c_int32,
                                    ctypes.POINTER(rm_cost_params), ctypes.POINTER(rm_cost_out), _P]),
    "rm_pose_retract": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, _P]),
    "rm_twist_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P, _P]),
    "rm_cost_grad_batch": (ctypes.c_int, [_P, ctypes.POINTER(rm_problem), ctypes.c_int32,
                                          ctypes.POINTER(rm_cost_params), ctypes.POINTER(rm_cost_out), _P]),
    "rm_align_batch": (ctypes.c_int, [_P, ctypes.POINTER(rm_problem), ctypes.c_int32,
                                      ctypes.POINTER(rm_cost_params), ctypes.POINTER(rm_align_params), _P,
                                      ctypes.POINTER(rm_align_report), _P]),
    "rm_align": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P, ctypes.POINTER(rm_cost_params),
                                ctypes.POINTER(rm_align_params), _P, ctypes.POINTER(rm_align_report), _P]),
    "rm_icp_terms": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P, ctypes.c_int32, ctypes.c_float,
                                    ctypes.POINTER(rm_icp_out), _P]),
    "rm_icp_align": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P, ctypes.POINTER(rm_icp_params), _P,
                                    ctypes.POINTER(rm_icp_report), _P]),
    "rm_depth_normals": (ctypes.c_int, [ctypes.POINTER(rm_intrinsics), ctypes.c_int32, _P, _P, ctypes.c_float,
                                        ctypes.c_int32, _P, _P, _P]),
    "rm_meshify": (ctypes.c_int, [ctypes.POINTER(rm_scan), _P, ctypes.POINTER(rm_meshify_params), _P, _P, _P,
                                  _P, _P]),
    "rm_dfo_align": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P, ctypes.POINTER(rm_cost_params),
                                    ctypes.POINTER(rm_dfo_params), _P, ctypes.POINTER(rm_dfo_report), _P]),
    "rm_scan_from_range": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, _P, _P, _P]),
    "rm_pose_from_x": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "rm_depth_blur": (ctypes.c_int, [ctypes.POINTER(rm_intrinsics), ctypes.c_int32, _P, _P, ctypes.c_float, _P,
                                     _P]),
    "rm_cost_grad_vertices": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P, ctypes.c_int32,
                                             ctypes.POINTER(rm_cost_params), _P, _P]),
    "rm_icp_align_batch": (ctypes.c_int, [_P, ctypes.POINTER(rm_problem), ctypes.c_int32,
                                          ctypes.POINTER(rm_icp_params), _P, ctypes.POINTER(rm_icp_report), _P]),
    "rm_cost_sweep": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                     ctypes.POINTER(rm_cost_params), ctypes.POINTER(rm_cost_out), _P]),
    "rm_cost_grad_noalloc": (ctypes.c_int, [_P, ctypes.POINTER(rm_scan), _P,
                                            ctypes.POINTER(rm_cost_params), ctypes.POINTER(rm_cost_out), _P]),
    "rm_status_sync": (ctypes.c_int, [_P, _P]),
    "rm_profile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rm_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(rm_kernel_time), ctypes.c_int32, _P, _P]),
    "rm_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded library; raises if it has not been built (run __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"librendermap.so is not built ({LIB_PATH}); run "
                              "paper_1702_06813_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


class RenderMapError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int) -> int:
    if status != RM_OK:
        raise RenderMapError(status, lib().rm_last_error().decode(errors="replace"))
    return status
