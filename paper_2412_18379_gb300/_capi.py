"""ctypes declarations of the C ABI in include/cnnsns.h (argument marshalling only).

The shared library is built in-tree by paper_2412_18379_gb300.build. If it is
missing the import fails loudly: there is no CPU fallback for any entry point.
"""

import ctypes
import os

from . import build as _build

LIB_PATH = _build.LIB

CS_OK = 0
CS_SNS, CS_CNN_SNS, CS_ASG_DIRECT = 0, 1, 2
CS_FOUND, CS_OUTSIDE, CS_FOUND_VIA_FALLBACK, CS_INVALID = 0, 1, 2, 3
CS_EPS = 1e-12
CS_NO_FIELD = -1

ERRORS = {
    -1: "CS_EINVAL", -2: "CS_ENOMEM", -3: "CS_ENOMESH", -4: "CS_EBUSY",
    -5: "CS_ECUDA", -6: "CS_EMESH", -7: "CS_ENOPRED", -8: "CS_EDEVICE",
}

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double


class MeshInfo(ctypes.Structure):
    _fields_ = [
        ("dim", _i32),
        ("n_vertices", _i64),
        ("n_elements", _i64),
        ("asg_grid", _i32 * 3),
        ("bucket_grid", _i32 * 3),
        ("bucket_items", _i64),
        ("lo", _dbl * 3),
        ("hi", _dbl * 3),
        ("tau", _dbl),
        ("step_cap", _i32),
        ("record_bytes", _i32),
        ("device_bytes", ctypes.c_size_t),
        ("pred_stride", _i32),
        ("pred_grid", _i32 * 3),
    ]


# name -> (restype, argtypes); every symbol include/cnnsns.h declares
SIGNATURES = {
    "cs_create": (_i32, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t]),
    "cs_memory_usage": (_i32, [_vp, ctypes.POINTER(ctypes.c_size_t),
                               ctypes.POINTER(ctypes.c_size_t)]),
    "cs_field_upload": (_i32, [_vp, _i32, _vp, ctypes.POINTER(_i32)]),
    "cs_field_release": (_i32, [_vp, _i32]),
    "cs_destroy": (None, [_vp]),
    "cs_last_error": (ctypes.c_char_p, [_vp]),
    "cs_mesh_upload": (_i32, [_vp, ctypes.c_int, _i64, _vp, _i64, _vp, _vp,
                              ctypes.POINTER(_i32)]),
    "cs_mesh_release": (_i32, [_vp, _i32]),
    "cs_mesh_query": (_i32, [_vp, _i32, ctypes.POINTER(MeshInfo)]),
    "cs_node_start_elements": (_i32, [_vp, _i32, _vp]),
    "cs_seed_grid": (_i32, [_vp, _i32, _vp]),
    "cs_track": (_i32, [_vp, _i32, _i32, _i64, _vp, _vp, _dbl, _vp, ctypes.c_int, _vp, _vp,
                        _vp, _vp, _vp]),
    "cs_track_host": (_i32, [_vp, _i32, _i32, _i64, _vp, _vp, _dbl, _vp, ctypes.c_int, _vp,
                             _vp, _vp, _vp]),
    "cs_track_nodes_host": (_i32, [_vp, _i32, _i32, _vp, _dbl, ctypes.c_int, _vp, _vp, _vp,
                                   _vp]),
    "cs_track_noalloc": (_i32, [_vp, _i32, _i32, _i64, _vp, _vp, _dbl, _vp, ctypes.c_int, _vp,
                                _vp, _vp, _vp, _vp]),
    "cs_track_stats": (_i32, [_vp, _i64, _vp, _vp, ctypes.POINTER(_i64), _vp]),
    "cs_kernel_launches": (_i64, [_vp]),
    "cs_predictor_precision": (_i32, [_vp, ctypes.c_int]),
    "cs_predictor_engine": (_i32, [_vp, ctypes.c_int]),
    "cs_predictor_tile_rows": (_i32, [_vp, ctypes.c_int]),
    "cs_predictor_tile3": (_i32, [_vp, ctypes.c_int]),
    "cs_debug_hold_predictor": (_i32, [_vp, ctypes.c_int]),
    "cs_device_status": (_i32, [_vp]),
    "cs_predictor_size": (_i64, [ctypes.c_int]),
    "cs_predictor_load": (_i32, [_vp, ctypes.c_int, _vp, _i64]),
    "cs_predictor_save": (_i32, [_vp, ctypes.c_int, _vp, _i64]),
    "cs_predictor_grid": (_i32, [_vp, _i32, _i32]),
    "cs_grid_velocity": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "cs_windows": (_i32, [_vp, _i32, _vp, _dbl, _vp, _i64, _vp, _vp]),
    "cs_predictor_forward": (_i32, [_vp, ctypes.c_int, _i64, _vp, _vp]),
    "cs_predict": (_i32, [_vp, _i32, _dbl, _vp, _vp]),
    "cs_predictor_train": (_i32, [_vp, ctypes.c_int, _vp, _vp, _i64, _i64, _i64, ctypes.c_float,
                                  ctypes.c_uint64, _vp]),
    "cs_training_pairs": (_i32, [_vp, _i32, _i64, _vp, _vp, _dbl, _vp, _vp, _vp, _vp]),
    "cs_predictor_grad": (_i32, [_vp, ctypes.c_int, _i64, _vp, _vp, _vp, _vp]),
    "cs_track_dhat": (_i32, [_vp, _i32, _i64, _vp, _vp, _dbl, _vp, _vp, _vp, _vp, _vp, _vp,
                             _vp]),
    "cs_classifier_size": (_i64, [ctypes.c_int]),
    "cs_classifier_window": (_i32, [ctypes.c_int]),
    "cs_classifier_load": (_i32, [_vp, ctypes.c_int, _vp, _i64]),
    "cs_classifier_save": (_i32, [_vp, ctypes.c_int, _vp, _i64]),
    "cs_departure": (_i32, [_vp, _i32, _i64, _vp, _vp, _dbl, _vp, _vp]),
    "cs_classifier_features": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp, _vp]),
    "cs_classifier_forward": (_i32, [_vp, _i32, _i64, _vp, _vp]),
    "cs_classifier_labels": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp, _vp]),
    "cs_classifier_pairs": (_i32, [_vp, _i32, _i64, _vp, _vp, _dbl, _vp, _vp, _vp, _vp]),
    "cs_classifier_grad": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp, _vp]),
    "cs_classifier_train": (_i32, [_vp, _i32, _vp, _vp, _i64, _i64, _i64, ctypes.c_float,
                                   ctypes.c_uint64, _vp]),
    "cs_classifier_start": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "cs_track_classifier": (_i32, [_vp, _i32, _i64, _vp, _vp, _dbl, _vp, _vp, _vp, _vp, _vp,
                                   _vp]),
    "cs_profile_enable": (_i32, [_vp, ctypes.c_int]),
    "cs_profile_read": (_i32, [_vp, _vp, ctypes.c_int]),
}

STAGES = ["walk", "fallback", "resample", "cnn", "train"]


class ServeCfg(ctypes.Structure):
    _fields_ = [("slots", _i32), ("arena_bytes", ctypes.c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("mesh_id", _i32), ("field_id", _i32), ("n", _i64), ("x", _vp), ("u", _vp),
                ("dt", _dbl),
                ("start", _vp), ("mode", _i32), ("host_out", _vp), ("path_len_out", _vp),
                ("status_out", _vp)]


class ServeStats(ctypes.Structure):
    _fields_ = [("completed", _i64), ("rejected", _i64), ("particles", _i64),
                ("p50_ms", _dbl), ("p99_ms", _dbl), ("mean_ms", _dbl), ("max_ms", _dbl),
                ("wall_s", _dbl), ("particles_per_s", _dbl), ("peak_bytes", _i64),
                ("max_concurrent", _i32)]


class ServeRecord(ctypes.Structure):
    _fields_ = [("ticket", _i64), ("n", _i64), ("mesh_id", _i32), ("mode_used", _i32),
                ("slot", _i32), ("in_flight", _i32), ("result", _i32), ("reserved", _i32),
                ("dt", _dbl), ("submit_ms", _dbl), ("admit_ms", _dbl), ("done_ms", _dbl),
                ("h2d_ms", _dbl), ("predict_ms", _dbl), ("walk_ms", _dbl), ("d2h_ms", _dbl)]


SIGNATURES.update({
    "cs_serve_start": (_i32, [_vp, ctypes.POINTER(ServeCfg)]),
    "cs_serve_submit": (_i32, [_vp, ctypes.POINTER(Request), ctypes.POINTER(_i64)]),
    "cs_serve_wait": (_i32, [_vp, _i64, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "cs_serve_report": (_i32, [_vp, ctypes.POINTER(ServeStats)]),
    "cs_serve_trace": (_i32, [_vp, _i64, ctypes.POINTER(ServeRecord), ctypes.POINTER(_i64)]),
    "cs_serve_stop": (_i32, [_vp]),
})


class ErrorStats(ctypes.Structure):
    _fields_ = [("n_err", _i64), ("err_sum", _dbl), ("err_max", _dbl), ("n_disp", _i64),
                ("disp_sum", _dbl), ("disp_max", _dbl)]


SIGNATURES["cs_track_error"] = (_i32, [_vp, _i32, _i64, _vp, _vp, _dbl, _vp, _vp, _vp,
                                       ctypes.POINTER(ErrorStats), _vp])


class Profile(ctypes.Structure):
    _fields_ = [("launches", _i64 * 8), ("ms", _dbl * 8)]

_LIB = None


def load(path=None):
    """Load libcnnsns.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libcnnsns.so not built: run paper_2412_18379_gb300.build.build() "
                          "(expected at %s)" % p)
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib


class CsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code
