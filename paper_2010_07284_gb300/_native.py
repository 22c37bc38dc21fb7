"""ctypes binding of include/vl.h.  Argument marshalling only: every step of
the evaluation runs in the library's CUDA kernels.  There is no CPU path: if
the shared library cannot be built or loaded, every call raises."""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import buildlib as _build

_LOCK = threading.Lock()
_LIB = None

# vl_status
OK, ERR_ARG, ERR_FORMULA, ERR_SHAPE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_INTERNAL, ERR_CANCELLED = range(10)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_FORMULA", 3: "ERR_SHAPE", 4: "ERR_OOM",
                5: "ERR_CUDA", 6: "ERR_TIMEOUT", 7: "ERR_BUSY", 8: "ERR_INTERNAL",
                9: "ERR_CANCELLED"}

OPCODES = {"TRUE": 0, "FALSE": 1, "THR_GT": 2, "THR_LT": 3, "PCT_GT": 4, "PCT_LT": 5,
           "MASK": 6, "NOT": 7, "AND": 8, "NEAR": 9, "REACH": 10, "OR": 11,
           "INTERIOR": 12, "SURROUNDED": 13, "GROW": 14, "TOUCH": 15,
           "VALUE": 16, "ADD": 17, "SUB": 18, "MUL": 19, "DIV": 20}
PX_F32, PX_U16 = 0, 1

EXEC_FUSED, EXEC_PLAIN = 0, 1


class VlNode(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32),
                ("image", C.c_int32), ("channel", C.c_int32), ("t", C.c_float),
                ("q", C.c_double)]


class VlConfig(C.Structure):
    _fields_ = [("device", C.c_int32), ("exec_mode", C.c_int32), ("use_graphs", C.c_int32),
                ("trace", C.c_int32), ("spin_limit", C.c_int64),
                ("memory_budget", C.c_int64), ("tile_rows", C.c_int32),
                ("tile_words", C.c_int32), ("reserved", C.c_int32 * 6)]


class VlJob(C.Structure):
    _fields_ = [("formula", C.c_void_p), ("images", C.POINTER(C.c_void_p)),
                ("n_images", C.c_int32), ("reserved", C.c_int32)]


class VlFormulaStats(C.Structure):
    _fields_ = [("n_primitive", C.c_int64), ("n_reach", C.c_int64), ("n_threshold", C.c_int64),
                ("n_not", C.c_int64), ("n_and", C.c_int64), ("n_near", C.c_int64),
                ("n_roots", C.c_int32), ("n_images", C.c_int32), ("n_steps", C.c_int32),
                ("n_groups", C.c_int32), ("n_selects", C.c_int32),
                ("n_channels_read", C.c_int32), ("mask_writes", C.c_int64),
                ("mask_reads", C.c_int64), ("max_halo", C.c_int32), ("n_number_images", C.c_int32)]


class VlPlanSizes(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("n_insns", C.c_int32), ("n_selects", C.c_int32),
                ("n_pct", C.c_int32), ("n_inter_slots", C.c_int32), ("n_root_slots", C.c_int32),
                ("n_mask_slots", C.c_int32), ("n_roots", C.c_int32),
                ("n_rank_tables", C.c_int32), ("n_rank_values", C.c_int32),
                ("n_rank_planes", C.c_int32), ("n_deps", C.c_int32)]


class VlPlanStep(C.Structure):
    _fields_ = [("kind", C.c_int32), ("insn_off", C.c_int32), ("insn_cnt", C.c_int32),
                ("halo", C.c_int32), ("sel_off", C.c_int32), ("sel_cnt", C.c_int32),
                ("pct_off", C.c_int32), ("pct_cnt", C.c_int32),
                ("rank_mask", C.c_int32), ("rank_halo", C.c_int32), ("n_bufs", C.c_int32)]


class VlPlanInsn(C.Structure):
    _fields_ = [("op", C.c_uint8), ("dst", C.c_uint8), ("a", C.c_uint8), ("b", C.c_uint8),
                ("halo", C.c_int16), ("slot", C.c_int16), ("image", C.c_int16),
                ("channel", C.c_int16), ("t", C.c_float)]


class VlPlanSelect(C.Structure):
    _fields_ = [("phi1_slot", C.c_int16), ("phi2_slot", C.c_int16), ("z_slot", C.c_int16),
                ("scratch", C.c_int16)]


class VlPlanPct(C.Structure):
    _fields_ = [("image", C.c_int16), ("channel", C.c_int16), ("slot", C.c_int16),
                ("pad", C.c_int16), ("q", C.c_double)]


class VlPlanRank(C.Structure):
    _fields_ = [("image", C.c_int32), ("channel", C.c_int32), ("m", C.c_int32),
                ("nbits", C.c_int32), ("value_off", C.c_int32), ("plane0", C.c_int32)]


class VlPlanArith(C.Structure):
    _fields_ = [("op", C.c_uint8), ("dst", C.c_uint8), ("a", C.c_uint8), ("b", C.c_uint8),
                ("image", C.c_int16), ("channel", C.c_int16), ("c", C.c_float)]


class VlServerConfig(C.Structure):
    _fields_ = [("max_inflight_batches", C.c_int32), ("max_batch_jobs", C.c_int32),
                ("memory_budget", C.c_int64), ("batch_window_us", C.c_int64),
                ("reserved", C.c_int32 * 8)]


class VlServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("cancelled", C.c_int64),
                ("failed", C.c_int64), ("batches", C.c_int64), ("bytes_in_use", C.c_int64),
                ("peak_bytes", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


class VlTileChoice(C.Structure):
    _fields_ = [("tile_rows", C.c_int32), ("tile_words", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("status", C.c_int32), ("ms", C.c_double)]


# (name, restype, argtypes)
_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)
_I32, _I64 = C.c_int32, C.c_int64
SIGNATURES = [
    ("vl_config_default", None, [C.POINTER(VlConfig)]),
    ("vl_context_create", C.c_int, [C.POINTER(VlConfig), _PP]),
    ("vl_last_error", C.c_char_p, [_P]),
    ("vl_free", None, [_P]),
    ("vl_image_create", C.c_int, [_P, _I32, _I32, _I32, _P, _I32, _P, _PP]),
    ("vl_image_create_u16", C.c_int, [_P, _I32, _I32, _I32, _P, _I32, _P, _PP]),
    ("vl_image_format", C.c_int, [_P, C.POINTER(_I32)]),
    ("vl_volume_create", C.c_int, [_P, _I32, _I32, _I32, _I32, _P, _I32, _P, _PP]),
    ("vl_volume_create_u16", C.c_int, [_P, _I32, _I32, _I32, _I32, _P, _I32, _P, _PP]),
    ("vl_mask_volume_create", C.c_int, [_P, _I32, _I32, _I32, _P, _I32, _P, _PP]),
    ("vl_image_depth", C.c_int, [_P, C.POINTER(_I32)]),
    ("vl_result_depth", C.c_int, [_P, C.POINTER(_I32)]),
    ("vl_mask_create", C.c_int, [_P, _I32, _I32, _P, _I32, _P, _PP]),
    ("vl_mask_create_packed", C.c_int, [_P, _I32, _I32, _P, _I32, _P, _PP]),
    ("vl_image_info", C.c_int, [_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)]),
    ("vl_formula_compile", C.c_int, [_P, C.POINTER(VlNode), _I32, C.POINTER(_I32), _I32, _I32, _PP]),
    ("vl_formula_compile_text", C.c_int, [_P, C.c_char_p, _I32, _PP, C.c_char_p, _I32]),
    ("vl_formula_spec_names", C.c_int, [_P, _I32, C.POINTER(_I32), _I32, C.c_char_p, _I32]),
    ("vl_formula_step_deps", C.c_int, [_P, C.POINTER(_I32), C.POINTER(_I32)]),
    ("vl_formula_rank_tables", C.c_int, [_P, C.POINTER(VlPlanRank), C.POINTER(C.c_float)]),
    ("vl_formula_arith", C.c_int, [_P, C.POINTER(VlPlanArith), C.POINTER(_I32), C.POINTER(_I32),
                                   C.POINTER(_I32)]),
    ("vl_formula_info", C.c_int, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I32)]),
    ("vl_formula_stats_get", C.c_int, [_P, C.POINTER(VlFormulaStats)]),
    ("vl_formula_plan", C.c_int, [_P, C.POINTER(VlPlanSizes), C.POINTER(VlPlanStep),
                                  C.POINTER(VlPlanInsn), C.POINTER(VlPlanSelect),
                                  C.POINTER(VlPlanPct), C.POINTER(_I32), C.POINTER(_I32)]),
    ("vl_eval", C.c_int, [_P, _P, _PP, _I32, _P, _PP]),
    ("vl_eval_mode", C.c_int, [_P, _P, _PP, _I32, _I32, _P, _PP]),
    ("vl_eval_batch", C.c_int, [_P, C.POINTER(VlJob), _I32, _P, _PP]),
    ("vl_batch_prepare", C.c_int, [_P, C.POINTER(VlJob), _I32, _P, _PP]),
    ("vl_batch_run", C.c_int, [_P, _P]),
    ("vl_batch_result", C.c_int, [_P, _I32, _PP]),
    ("vl_batch_info", C.c_int, [_P, C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I64)]),
    ("vl_batch_trace", C.c_int, [_P, C.POINTER(_I64), _I64, C.POINTER(_I64)]),
    ("vl_autotune", C.c_int, [_P, C.POINTER(VlJob), _I32, _P, _I32, C.POINTER(VlTileChoice),
                              _I32, C.POINTER(_I32), C.POINTER(VlTileChoice)]),
    ("vl_tile_shape", C.c_int, [_P, C.POINTER(VlJob), _I32, C.POINTER(VlTileChoice),
                                C.POINTER(_I32)]),
    ("vl_tune_save", C.c_int, [_P, C.c_char_p]),
    ("vl_tune_load", C.c_int, [_P, C.c_char_p]),
    ("vl_result_sync", C.c_int, [_P]),
    ("vl_result_status_word", C.c_int, [_P, C.POINTER(_I32)]),
    ("vl_result_info", C.c_int, [_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)]),
    ("vl_result_mask", C.c_int, [_P, _I32, _P, _I32, _P]),
    ("vl_result_mask_u8", C.c_int, [_P, _I32, _P, _I32, _P]),
    ("vl_result_masks", C.c_int, [_P, _P, _I32, _P]),
    ("vl_result_device_ptr", C.c_int, [_P, _I32, _PP]),
    ("vl_ccl", C.c_int, [_P, _P, _I32, _P, _P]),
    ("vl_ccl_status", C.c_int, [_P, _P]),
    ("vl_ccl_pointer_jumping", C.c_int, [_P, _P, _I32, _I32, _I32, _P, _P, C.POINTER(_I32)]),
    ("vl_ccl_noalloc", C.c_int, [_P, _I32, _I32, _I32, _P, _I32, _P]),
    ("vl_server_create", C.c_int, [_P, C.POINTER(VlServerConfig), _PP]),
    ("vl_server_submit", C.c_int, [_P, _P, _PP, _I32, C.POINTER(_I64)]),
    ("vl_server_wait", C.c_int, [_P, _I64, _I64, _PP]),
    ("vl_server_cancel", C.c_int, [_P, _I64]),
    ("vl_server_stats_get", C.c_int, [_P, C.POINTER(VlServerStats)]),
]


def lib_path() -> str:
    return _build.lib_path()


def load(build_if_needed: bool = True) -> C.CDLL:
    """Load (building first if stale) the CUDA library."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.build() if build_if_needed else _build.lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path} (run build())")
        lib = C.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
        return lib


class VlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code
