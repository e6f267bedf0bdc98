"""ctypes declarations of the C ABI in include/gsr.h and the loader of libgsr.so.

Argument marshalling only.  The library is built in-tree by ``build.py``
(``__graft_entry__.build()``); loading fails loudly if it is missing: there is
no CPU fallback for the rasterizer.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

GSR_OK = 0
GSR_ERR_INVALID_ARG = 1
GSR_ERR_CAPACITY = 2
GSR_ERR_CUDA = 3
GSR_ERR_TIMEOUT = 4
GSR_ERR_NOT_SUPPORTED = 5
GSR_ERR_OUT_OF_MEMORY = 6
GSR_MAX_VIEWS = 64
GSR_NOALLOC_MAX_INSTANCES = 524288   # include/gsr.h
GSR_FLAG_NO_SYNC = 1
GSR_DEBUG_WITHHOLD_PREFIX = 1

_STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CAPACITY", 3: "CUDA", 4: "TIMEOUT", 5: "NOT_SUPPORTED",
                 6: "OUT_OF_MEMORY"}


class GsrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gsr error {_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("tile_w", C.c_int), ("tile_h", C.c_int), ("blend_batch", C.c_int), ("sh_degree", C.c_int),
                ("near_plane", C.c_float), ("bg", C.c_float * 3), ("flags", C.c_uint32),
                ("blend_batch_bwd", C.c_int), ("list_prefix", C.c_float)]


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class View(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("viewmat", C.c_float * 16), ("subset", C.c_void_p),
                ("subset_count", C.c_int64)]


class Outputs(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("alpha", C.c_void_p)]


class Grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("pose", C.c_void_p), ("focal", C.c_void_p)]


class InsertParams(C.Structure):
    _fields_ = [("sigma", C.c_float), ("tau_a", C.c_float)]


class Image(C.Structure):
    _fields_ = [("data", C.c_void_p), ("width", C.c_int), ("height", C.c_int), ("factor", C.c_int)]


class MergeParams(C.Structure):
    _fields_ = [("tau_d", C.c_float), ("near_plane", C.c_float)]


class MergeOutputs(C.Structure):
    _fields_ = [("sample_action", C.c_void_p), ("sample_means", C.c_void_p), ("sample_scale", C.c_void_p),
                ("sample_depth", C.c_void_p), ("sample_dc", C.c_void_p), ("existing_action", C.c_void_p),
                ("existing_dc", C.c_void_p)]


class SavedInfo(C.Structure):
    _fields_ = [("n_records", C.c_int64), ("n_visible", C.c_int64), ("n_instances", C.c_int64),
                ("n_tiles", C.c_int64), ("n_pixels", C.c_int64), ("fwd_pairs", C.c_int64),
                ("bwd_pairs", C.c_int64), ("tile_w", C.c_int), ("tile_h", C.c_int), ("blend_batch", C.c_int),
                ("blended_pairs", C.c_int64), ("warp_entries_fwd", C.c_int64), ("warp_entries_bwd", C.c_int64),
                ("n_instances_full", C.c_int64), ("grad_rows", C.c_int64), ("list_prefix", C.c_float),
                ("n_instances_second", C.c_int64), ("open_tiles", C.c_int64), ("list_span", C.c_int64)]


GSR_FLAG_PROFILE = 2
GSR_FLAG_NO_PAIR_COUNTS = 4
GSR_LIST_BUCKETS = 64
PHASES = ["preprocess", "depth_sort", "duplicate", "tile_sort", "ranges", "blend_fwd", "bwd_clear", "blend_bwd",
          "preprocess_bwd"]


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("phase_ms", C.c_double * len(PHASES)), ("calls", C.c_int64 * len(PHASES))]


# every symbol declared in include/gsr.h: (name, restype, argtypes)
_P = C.c_void_p
SIGNATURES = [
    ("gsr_config_default", None, [C.POINTER(Config)]),
    ("gsr_create", C.c_int, [C.POINTER(_P), C.POINTER(Config)]),
    ("gsr_destroy", None, [_P]),
    ("gsr_last_error", C.c_char_p, [_P]),
    ("gsr_set_config", C.c_int, [_P, C.POINTER(Config)]),
    ("gsr_get_config", C.c_int, [_P, C.POINTER(Config)]),
    ("gsr_saved_create", C.c_int, [_P, C.POINTER(_P)]),
    ("gsr_saved_destroy", None, [_P]),
    ("gsr_saved_get_info", C.c_int, [_P, C.POINTER(SavedInfo)]),
    ("gsr_reserve", C.c_int, [_P, _P, C.c_int64, C.c_int64]),
    ("gsr_forward", C.c_int, [_P, C.POINTER(Gaussians), C.POINTER(View), C.c_int, C.POINTER(Outputs), _P, _P]),
    ("gsr_backward", C.c_int, [_P, C.POINTER(Gaussians), C.POINTER(View), C.c_int, _P, _P, _P, _P,
                               C.POINTER(Grads), _P]),
    ("gsr_check", C.c_int, [_P, _P, _P]),
    ("gsr_l1_loss_grad", C.c_int, [_P, _P, C.c_int64, _P, _P, _P]),
    ("gsr_insert_params_default", None, [C.POINTER(InsertParams)]),
    ("gsr_insertion", C.c_int, [_P, C.POINTER(InsertParams), _P, C.c_int, _P, _P, _P, _P, _P, _P, C.c_int64, _P,
                                _P]),
    ("gsr_merge_params_default", None, [C.POINTER(MergeParams)]),
    ("gsr_merge", C.c_int, [_P, C.POINTER(MergeParams), _P, C.c_int64, _P, _P, _P, C.c_int64, C.c_int64, _P, _P, _P,
                            _P, C.POINTER(MergeOutputs), _P]),
    ("gsr_dft_energy", C.c_int, [_P, C.POINTER(Image), C.c_int, _P, _P]),
    ("gsr_frequency_schedule", C.c_int, [_P, C.c_int, _P, _P, _P, C.c_float, _P, C.c_int, _P, _P, _P, _P, _P]),
    ("gsr_rig_chain", C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, C.c_int, C.c_int, _P, _P, _P, _P]),
    ("gsr_tune", C.c_int, [_P, C.POINTER(Gaussians), C.POINTER(View), C.c_int, C.POINTER(Outputs), _P, _P,
                           C.POINTER(Grads), C.POINTER(Config), _P]),
    ("gsr_debug_lists", C.c_int, [_P, _P, _P, _P, _P]),
    ("gsr_debug_list_slice", C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P]),
    ("gsr_debug_records", C.c_int, [_P, _P, _P, _P, _P]),
    ("gsr_debug_pixels", C.c_int, [_P, _P, _P, _P]),
    ("gsr_debug_record_grads", C.c_int, [_P, _P, _P]),
    ("gsr_debug_set_wait", C.c_int, [_P, C.c_uint64, C.c_uint32]),
    ("gsr_get_stats", C.c_int, [_P, C.POINTER(Stats)]),
    ("gsr_list_prefix_choice", C.c_float, [_P, _P, C.c_uint64]),
    ("gsr_list_bucket_edge", C.c_double, [C.c_int]),
    ("gsr_forward_noalloc", C.c_int, [C.POINTER(Config), C.POINTER(Gaussians), C.POINTER(View), C.c_int,
                                      C.POINTER(Outputs), _P]),
    ("gsr_version", C.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libgsr.so (built by build.py) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(f"libgsr.so not found at {p}: build it first (python -c 'import __graft_entry__ as g; "
                               f"g.build()'); the rasterizer has no CPU fallback")
        lib = C.CDLL(p)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib
