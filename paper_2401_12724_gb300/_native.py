"""ctypes declarations of libbysdf (include/bysdf.h).  Marshalling only."""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None


class MaterialDesc(C.Structure):
    _fields_ = [
        ("n_plies", C.c_int32), ("fibers_per_ply", C.c_int32), ("map_texels", C.c_int32),
        ("trace_iters", C.c_int32), ("k_max", C.c_int32), ("flags", C.c_int32),
        ("yarn_radius", C.c_float), ("ply_twist_deg", C.c_float), ("fiber_twist_deg", C.c_float),
        ("eta", C.c_float), ("albedo", C.c_float * 3), ("k_spec", C.c_float),
        ("beta_deg", C.c_float * 2), ("body_B", C.c_float), ("body_r", C.c_float),
        ("sigma_t", C.c_float), ("shadow_density", C.c_float), ("packing", C.c_float),
        ("albedo_y", C.c_float * 3),
        ("migration_maps", C.c_int32), ("migration_seed", C.c_int32),
        ("migration_length", C.c_float), ("migration_blend", C.c_float),
    ]


class Hits(C.Structure):
    _fields_ = [("h", C.c_void_p), ("u", C.c_void_p), ("v", C.c_void_p), ("wi", C.c_void_p),
                ("wo", C.c_void_p), ("ratio", C.c_void_p), ("mat_id", C.c_void_p),
                ("seg_offsets", C.c_void_p)]


class LaunchConfig(C.Structure):
    _fields_ = [("block", C.c_int32), ("items", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("occupancy", C.c_int32)]


class Outputs(C.Structure):
    _fields_ = [("f_rgb", C.c_void_p), ("pdf", C.c_void_p), ("status", C.c_void_p),
                ("wo", C.c_void_p), ("weight", C.c_void_p), ("pdf_s", C.c_void_p),
                ("lobe_status", C.c_void_p), ("grad_params", C.c_void_p)]


class Stochastic(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("index_offset", C.c_int64), ("flags", C.c_uint32),
                ("reserved", C.c_uint32)]


STOCH_JITTER_NODES, STOCH_ROUGH_ENTRY = 1, 2


class Rays(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("o", "d", "o1", "d1", "o2", "d2")]

# (name, restype, argtypes) of every symbol declared in include/bysdf.h
P = C.c_void_p
SYMBOLS = [
    ("bysdf_version", C.c_char_p, []),
    ("bysdf_last_error", C.c_char_p, []),
    ("bysdf_create_materials", C.c_int, [C.POINTER(MaterialDesc), C.c_int32, P, C.POINTER(P)]),
    ("bysdf_destroy_materials", C.c_int, [P]),
    ("bysdf_num_materials", C.c_int32, [P]),
    ("bysdf_set_params", C.c_int, [P, P, P]),
    ("bysdf_get_params", C.c_int, [P, P, P]),
    ("bysdf_set_params_ext", C.c_int, [P, P, P]),
    ("bysdf_get_params_ext", C.c_int, [P, P, P]),
    ("bysdf_workspace_size", C.c_size_t, [P, C.c_int64]),
    ("bysdf_eval", C.c_int, [P, C.POINTER(Hits), C.c_int64, P, P, P, P, C.c_size_t, P]),
    ("bysdf_sample", C.c_int, [P, C.POINTER(Hits), P, P, C.c_int64, P, P, P, P, P, C.c_size_t, P]),
    ("bysdf_pdf", C.c_int, [P, C.POINTER(Hits), C.c_int64, P, P, P, C.c_size_t, P]),
    ("bysdf_eval_sample_pdf", C.c_int,
     [P, C.POINTER(Hits), P, P, C.c_int64, P, P, P, P, P, P, P, P, C.c_size_t, P]),
    ("bysdf_eval_stochastic", C.c_int,
     [P, C.POINTER(Hits), C.POINTER(Stochastic), C.c_int64, P, P, P, P, C.c_size_t, P]),
    ("bysdf_eval_sample_pdf_stochastic", C.c_int,
     [P, C.POINTER(Hits), C.POINTER(Stochastic), P, P, C.c_int64, P, P, P, P, P, P, P, P,
      C.c_size_t, P]),
    ("bysdf_trace_yarns", C.c_int,
     [P, C.c_int32, C.POINTER(Rays), C.c_int64, C.POINTER(C.c_float), P, P, P, P, P, P, P, P, P,
      P]),
    ("bysdf_eval_backward", C.c_int, [P, C.POINTER(Hits), C.c_int64, P, P, C.c_int, P, C.c_size_t, P]),
    ("bysdf_eval_backward_ext", C.c_int,
     [P, C.POINTER(Hits), C.c_int64, P, P, P, P, C.c_int, P, C.c_size_t, P]),
    ("bysdf_plain", C.c_int, [C.c_int, P, C.POINTER(Hits), P, P, P, C.c_int64, P, P, P, P, P, P]),
    ("bysdf_eval_l2_backward", C.c_int,
     [P, C.POINTER(Hits), C.c_int64, P, P, P, P, P, C.c_int, P, C.c_size_t, P]),
    ("bysdf_plain_fused", C.c_int,
     [P, C.POINTER(Hits), P, P, P, C.c_int64, C.POINTER(Outputs), P]),
    ("bysdf_set_launch_config", C.c_int, [P, C.c_int, C.POINTER(LaunchConfig)]),
    ("bysdf_get_launch_config", C.c_int, [P, C.c_int, C.POINTER(LaunchConfig)]),
    ("bysdf_autotune", C.c_int, [P, C.c_int, C.POINTER(Hits), P, P, P, C.c_int64,
                                 C.POINTER(Outputs), P, C.c_size_t, P, C.POINTER(LaunchConfig)]),
    ("bysdf_workspace_error", C.c_int, [P, P, C.POINTER(C.c_uint32)]),
    ("bysdf_eval_noalloc", C.c_int, [P, C.POINTER(Hits), C.c_int64, P, P, P, P]),
    ("bysdf_noalloc_error", C.c_int, [P, C.POINTER(C.c_uint32)]),
    ("bysdf_test_stall_table_waits", C.c_int, [P, C.c_uint32]),
    ("bysdf_test_fail_allocations", C.c_int, [C.c_int32]),
    ("bysdf_test_math", C.c_int, [C.c_int32, P, P, C.c_int64, P, P]),
    ("bysdf_host_pipeline_create", C.c_int, [P, C.c_int64, C.c_int, C.POINTER(P)]),
    ("bysdf_host_pipeline_destroy", C.c_int, [P]),
    ("bysdf_eval_sample_pdf_host", C.c_int,
     [P, C.POINTER(Hits), P, P, C.c_int64, P, P, P, P, P, P, P, P]),
]

OP_EVAL, OP_SAMPLE, OP_PDF, OP_FUSED, OP_BACKWARD = range(5)
NPARAM, NPARAM_EXT = 8, 15


def bounds_checks() -> bool:
    """BYSDF_BOUNDS_CHECKS=1 selects the index-checking build of the library."""
    return os.environ.get("BYSDF_BOUNDS_CHECKS") == "1"


def lib_path() -> str:
    return _build.BOUNDS_LIB_PATH if bounds_checks() else _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libbysdf.so (building it first if asked).  There is no fallback:
    without the library every call raises."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if build_if_missing:
            _build.build(bounds=bounds_checks())
        if not os.path.exists(path):
            raise RuntimeError(f"libbysdf not built: {path} is missing")
        L = C.CDLL(path)
        for name, res, args in SYMBOLS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


def check(rc: int, what: str):
    if rc != 0:
        msg = load().bysdf_last_error().decode(errors="replace")
        raise RuntimeError(f"{what} failed ({rc}): {msg}")
