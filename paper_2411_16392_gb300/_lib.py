"""ctypes binding of libqgs.so (argument marshalling only; all work runs in the library).

The library must have been built (``python -m paper_2411_16392_gb300.build``); loading
fails loudly otherwise. There is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqgs.so")

STATUS = {0: "QGS_OK", 1: "QGS_EINVAL", 2: "QGS_ENOMEM", 3: "QGS_ECAPACITY", 4: "QGS_ECUDA",
          5: "QGS_ETIMEDOUT", 6: "QGS_EBUSY", 7: "QGS_ENOTFOUND", 8: "QGS_ESTATE"}


class QGSError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class qgs_camera(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R_cw", C.c_float * 9), ("t_cw", C.c_float * 3),
                ("near_plane", C.c_float)]


class qgs_scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("mean", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p),
                ("curv", C.c_void_p), ("opacity", C.c_void_p), ("sh", C.c_void_p)]


class qgs_image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("alpha", C.c_void_p), ("depth", C.c_void_p), ("normal", C.c_void_p),
                ("curvature", C.c_void_p), ("distortion", C.c_void_p), ("median_depth", C.c_void_p)]


class qgs_scene_grad(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("quat", C.c_void_p), ("scale", C.c_void_p), ("curv", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p)]


class qgs_config(C.Structure):
    _fields_ = [("alpha_max", C.c_float), ("alpha_min", C.c_float), ("T_min", C.c_float),
                ("grazing_eps", C.c_float), ("sort_mode", C.c_int32), ("density", C.c_int32),
                ("order", C.c_int32)]


class qgs_frame_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("n_primitives", "n_visible", "n_instances", "n_tiles", "pair_evals",
                                         "pair_isect", "pair_hits", "pair_blended", "grazing_resolves",
                                         "bwd_pairs", "bwd_contrib", "launches_fwd", "launches_bwd")] + \
              [(k, C.c_float) for k in ("ms_preprocess", "ms_depth_sort", "ms_emit", "ms_tile_sort",
                                        "ms_raster_fwd", "ms_raster_bwd", "ms_preprocess_bwd")]


class qgs_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("rejected", C.c_int64), ("max_in_flight", C.c_int64), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("frames_per_s", C.c_double),
                ("bytes_budget", C.c_int64), ("bytes_reserved_peak", C.c_int64), ("batches", C.c_int64),
                ("max_batch", C.c_int64)]


# (name, restype, argtypes) of every exported entry point declared in include/*.h
_P = C.c_void_p
EXPORTS = [
    ("qgs_config_default", None, [C.POINTER(qgs_config)]),
    ("qgs_create", C.c_int, [C.POINTER(_P), C.POINTER(qgs_config), C.c_int32]),
    ("qgs_destroy", None, [_P]),
    ("qgs_last_error", C.c_char_p, [_P]),
    ("render_forward", C.c_int, [_P, C.POINTER(qgs_scene), C.POINTER(qgs_camera), C.POINTER(qgs_image), _P]),
    ("render_backward", C.c_int, [_P, C.POINTER(qgs_scene), C.POINTER(qgs_camera), C.POINTER(qgs_image),
                                  C.POINTER(qgs_scene_grad), _P]),
    ("qgs_get_frame_stats", C.c_int, [_P, C.POINTER(qgs_frame_stats)]),
    ("qgs_copy_binning", C.c_int, [_P, _P, _P, C.c_int64, _P, _P, C.POINTER(C.c_int64)]),
    ("qgs_copy_residue", C.c_int, [_P, _P, _P]),
    ("qgs_check_frame", C.c_int, [_P]),
    ("qgs_debug_withhold_sort_chunk", C.c_int, [_P, C.c_int32]),
    ("qgs_debug_check_word", C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_uint32)]),
    ("qgs_set_profiling", C.c_int, [_P, C.c_int32]),
    ("qgs_set_tile_mask_capacity", C.c_int, [_P, C.c_int64]),
    ("qgs_set_pair_counters", C.c_int, [_P, C.c_int32]),
    ("render_forward_batch", C.c_int, [_P, C.POINTER(qgs_scene), C.c_int32, C.POINTER(qgs_camera),
                                       C.POINTER(qgs_image), _P]),
    ("render_forward_noalloc", C.c_int, [C.POINTER(qgs_scene), C.POINTER(qgs_camera), C.POINTER(qgs_image), _P]),
    ("serve_create", C.c_int, [C.POINTER(_P), C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                               C.c_double]),
    ("serve_destroy", None, [_P]),
    ("serve_load_scene", C.c_int, [_P, C.POINTER(qgs_scene), C.POINTER(C.c_int32)]),
    ("serve_submit", C.c_int, [_P, C.c_int32, C.POINTER(qgs_camera), C.c_int32, C.POINTER(qgs_image),
                               C.POINTER(C.c_uint64)]),
    ("serve_wait", C.c_int, [_P, C.c_uint64, C.c_int32, C.POINTER(qgs_image), C.POINTER(qgs_scene_grad)]),
    ("serve_stats", C.c_int, [_P, C.POINTER(qgs_serve_stats)]),
    ("serve_reset_stats", C.c_int, [_P]),
]

_lib = None


def load():
    """Load libqgs.so (or the library at LIB_PATH, e.g. the bounds-checked build
    libqgs_check.so when a process sets it before the first load) and declare its entry
    points. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libqgs.so not built ({LIB_PATH} missing): run "
                           "`python -m paper_2411_16392_gb300.build` (needs nvcc); there is no fallback")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in EXPORTS:
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols(header_dir=None):
    """Function names declared in include/*.h (parsed from the headers)."""
    import re
    if header_dir is None:
        header_dir = os.path.join(os.path.dirname(_HERE), "include")
    names = []
    for f in sorted(os.listdir(header_dir)):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(header_dir, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             txt, flags=re.M):
            names.append(m.group(1))
    return names


def check(status, ctx=None):
    if status != 0:
        msg = ""
        if ctx:
            m = load().qgs_last_error(ctx)
            msg = m.decode() if m else ""
        raise QGSError(status, msg)
