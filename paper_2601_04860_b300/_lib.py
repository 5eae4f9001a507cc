"""ctypes binding of ``libdivas_fuse.so`` (argument marshalling only).

The structs mirror ``include/divas_fuse.h``.  Loading fails loudly when the
library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdivas_fuse.so")

DIVAS_OK = 0
STATUS_NAMES = {0: "DIVAS_OK", 1: "DIVAS_E_INVALID", 2: "DIVAS_E_OOM", 3: "DIVAS_E_CUDA",
                4: "DIVAS_E_TIMEOUT", 5: "DIVAS_E_STATE", 6: "DIVAS_E_CAPACITY"}
MASK_F32 = 0
MASK_F16 = 1
MASK_LOGIT_F32 = 2
MAX_VIEWS_PER_CALL = 32
KEEP_ZEROS = 1
MAX_PROMPTS = 15
WEIGHT_NERF_MINMAX = 1
WEIGHT_GS_BAND = 2
NERF_LLFF = 0
NERF_MIP360 = 1


ORDER_BRICKS = 1  # divas_params.flags: brick-major active list


class DivasParams(ctypes.Structure):
    _fields_ = [("tau_mask", ctypes.c_float), ("gamma", ctypes.c_float),
                ("alpha1", ctypes.c_float), ("tau_cons", ctypes.c_float),
                ("eps", ctypes.c_float), ("z_near", ctypes.c_float), ("flags", ctypes.c_uint32)]


class DivasGrid(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("g", ctypes.c_int32), ("origin", ctypes.c_float * 3),
                ("h", ctypes.c_float), ("contracted", ctypes.c_int32)]


class DivasCamera(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3)]


class DivasView(ctypes.Structure):
    _fields_ = [("cam", DivasCamera), ("depth", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("mask_type", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class DivasTupleView(ctypes.Structure):
    _fields_ = [("cam", DivasCamera), ("d_min", ctypes.c_void_p), ("d_med", ctypes.c_void_p),
                ("d_max", ctypes.c_void_p), ("n_samp", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("mask_type", ctypes.c_int32),
                ("d_cam", ctypes.c_float)]


class DivasTupleParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("beta", "gamma_st", "tau_thin", "rho_cover", "rho_occ", "n_abs", "dist_gate",
                 "behind_margin", "k_dg", "rho_thin")]


class DivasNerfParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("gamma", "beta", "b_max", "lambda_range", "rho_thin", "rho_cover", "tau_thin",
                 "m_thin", "k_dg")] + [("reserved", ctypes.c_int32)]


class DivasWeightView(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("mask_type", ctypes.c_int32), ("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("n_prompts", ctypes.c_int32), ("prompt_xy", ctypes.c_int32 * (2 * 15))]


class DivasOccupancyParams(ctypes.Structure):
    _fields_ = [("alpha_v", ctypes.c_double), ("beta_v", ctypes.c_double), ("pad", ctypes.c_double),
                ("g0", ctypes.c_int32), ("g_max", ctypes.c_int32), ("tau_tf", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class DivasSceneFrame(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double * 3), ("r_fg", ctypes.c_double), ("b", ctypes.c_double),
                ("s_bar", ctypes.c_double), ("h", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("g", ctypes.c_int32), ("pad", ctypes.c_int32)]


class DivasSurfelParams(ctypes.Structure):
    _fields_ = [("tau_m", ctypes.c_float), ("tau_kappa", ctypes.c_float),
                ("eps_aspect", ctypes.c_float), ("reserved", ctypes.c_int32)]


class DivasError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "divas_default_params": (None, [ctypes.POINTER(DivasParams)]),
    "divas_fuse_init": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(DivasGrid), _P, _P,
                                       ctypes.c_int64, ctypes.POINTER(DivasParams), _P]),
    "divas_fuse_set_occupancy": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
    "divas_fuse_add_view": (ctypes.c_int, [_P, ctypes.POINTER(DivasCamera), _P, _P,
                                           ctypes.c_int32, _P]),
    "divas_fuse_add_views": (ctypes.c_int, [_P, ctypes.POINTER(DivasView), ctypes.c_int32, _P]),
    "divas_fuse_finalize": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int64), _P]),
    "divas_label_points": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "divas_fuse_reset": (ctypes.c_int, [_P, _P]),
    "divas_fuse_sync": (ctypes.c_int, [_P, _P]),
    "divas_fuse_n_active": (ctypes.c_int64, [_P]),
    "divas_fuse_n_views": (ctypes.c_int32, [_P]),
    "divas_fuse_active_coords": (ctypes.c_int, [_P, _P, _P]),
    "divas_fuse_export_state": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "divas_fuse_import_state": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, _P]),
    "divas_fuse_backward": (ctypes.c_int, [_P, ctypes.POINTER(DivasView), ctypes.c_int32, _P,
                                           ctypes.POINTER(_P), ctypes.POINTER(_P), _P]),
    "divas_debug_project": (ctypes.c_int, [_P, ctypes.POINTER(DivasCamera), _P, _P]),
    "divas_debug_rcp": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P]),
    "divas_debug_integral_images": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                                    _P]),
    "divas_fuse_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.POINTER(DivasView),
                                       ctypes.c_int32, _P, _P, _P, ctypes.c_int64, _P, _P]),
    "divas_default_tuple_params": (DivasTupleParams, []),
    "divas_depth_weight": (ctypes.c_int, [_P, ctypes.POINTER(DivasWeightView), ctypes.c_int32,
                                          ctypes.c_int32, _P, _P]),
    "divas_fuse_add_views_weighted": (ctypes.c_int, [_P, ctypes.POINTER(DivasView),
                                                     ctypes.POINTER(DivasWeightView),
                                                     ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "divas_default_occupancy_params": (DivasOccupancyParams, []),
    "divas_default_surfel_params": (DivasSurfelParams, []),
    "divas_overlay": (ctypes.c_int, [_P, ctypes.POINTER(DivasCamera), _P, _P, _P]),
    "divas_default_nerf_params": (DivasNerfParams, [ctypes.c_int32]),
    "divas_fuse_add_views_nerf": (ctypes.c_int, [_P, ctypes.POINTER(DivasTupleView), ctypes.c_int32,
                                                 ctypes.POINTER(DivasNerfParams), _P, _P]),
    "divas_fuse_add_views_nerf_profiled": (ctypes.c_int, [_P, ctypes.POINTER(DivasTupleView),
                                                          ctypes.c_int32,
                                                          ctypes.POINTER(DivasNerfParams), _P, _P,
                                                          _P]),
    "divas_density_floor": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_float, _P, _P]),
    "divas_surfel_labels": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64,
                                           ctypes.POINTER(DivasCamera), ctypes.POINTER(_P),
                                           ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(DivasSurfelParams), _P, _P, _P, _P]),
    "divas_scene_frame_from_gaussians": (ctypes.c_int, [_P, _P, ctypes.c_int64,
                                                        ctypes.POINTER(DivasOccupancyParams),
                                                        ctypes.POINTER(DivasSceneFrame), _P]),
    "divas_occupancy_from_gaussians": (ctypes.c_int, [_P, _P, ctypes.c_int64,
                                                      ctypes.POINTER(DivasSceneFrame),
                                                      ctypes.c_float, _P, _P, _P]),
    "divas_fuse_add_views_tuple": (ctypes.c_int, [_P, ctypes.POINTER(DivasTupleView),
                                                  ctypes.c_int32,
                                                  ctypes.POINTER(DivasTupleParams), _P]),
    "divas_fuse_add_views_tuple_profiled": (ctypes.c_int, [_P, ctypes.POINTER(DivasTupleView),
                                                           ctypes.c_int32,
                                                           ctypes.POINTER(DivasTupleParams), _P,
                                                           _P]),
    "divas_fuse_update": (ctypes.c_int, [_P, ctypes.POINTER(DivasView), ctypes.c_int32, _P, _P,
                                         ctypes.c_uint32, _P]),
    "divas_fuse_step_profiled": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64,
                                                ctypes.POINTER(DivasView), ctypes.c_int32, _P, _P,
                                                _P, ctypes.c_int64, _P, ctypes.POINTER(_P), _P]),
    "divas_fuse_dense_noalloc": (ctypes.c_int, [ctypes.POINTER(DivasGrid), _P,
                                                ctypes.POINTER(DivasView), ctypes.c_int32,
                                                ctypes.POINTER(DivasParams), _P, _P, _P]),
    "divas_noalloc_last_error": (ctypes.c_char_p, []),
    "divas_fuse_destroy": (None, [_P]),
    "divas_last_error": (ctypes.c_char_p, [_P]),
}

# batched sessions (bound in batch.py)
EXPORTED = tuple(_SIGS) + ("divas_batch_create", "divas_batch_queue", "divas_batch_fuse",
                           "divas_batch_finalize", "divas_batch_clear", "divas_batch_size",
                           "divas_batch_last_error", "divas_batch_destroy")


def load(path: str = LIB_PATH):
    """Load the CUDA library once; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first (python -c 'import "
            "__graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, ctx=None):
    if status != DIVAS_OK:
        msg = load().divas_last_error(ctx)
        raise DivasError(status, msg.decode() if msg else "")
