"""ctypes declarations of the C ABI in include/exactz.h (marshalling only).

The shared library is loaded from this package directory.  There is no
fallback: if it is missing or cannot be loaded, importing raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libexactz.so")

EXACTZ_OK = 0
EXACTZ_EINVAL = -1
EXACTZ_ENONFINITE = -2
EXACTZ_EBOUND = -3
EXACTZ_ENOMEM = -4
EXACTZ_ECAP = -5
EXACTZ_ENODEV = -6
EXACTZ_ESIZE = -7
ERROR_NAMES = {-1: "EINVAL", -2: "ENONFINITE", -3: "EBOUND", -4: "ENOMEM", -5: "ECAP",
               -6: "ENODEV", -7: "ESIZE"}

CONVERGED, STUCK, ITER_LIMIT = 1, 2, 3
MODE_PLAIN, MODE_FRONTIER, MODE_GRAPH, MODE_FUSED = 0, 1, 2, 3


class Dims(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_uint32), ("ny", ctypes.c_uint32), ("nz", ctypes.c_uint32)]


class Opts(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("mode", ctypes.c_uint32), ("max_iters", ctypes.c_uint64),
                ("want_edit_list", ctypes.c_uint32), ("profile", ctypes.c_uint32),
                ("events", ctypes.c_uint32), ("direction", ctypes.c_uint32)]


class Edit(ctypes.Structure):
    _fields_ = [("idx", ctypes.c_uint64), ("value", ctypes.c_float), ("k", ctypes.c_uint8),
                ("lossless", ctypes.c_uint8), ("reserved", ctypes.c_uint16)]


class Result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint64), ("n_edits", ctypes.c_uint64),
                ("n_lossless", ctypes.c_uint64), ("residual_violations", ctypes.c_uint64),
                ("n_critical", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("passes", ctypes.c_uint64),
                ("total_critical", ctypes.c_uint64), ("sum_requests", ctypes.c_uint64),
                ("sum_tiles", ctypes.c_uint64), ("sum_pairs", ctypes.c_uint64),
                ("stage_ms", ctypes.c_float * 8), ("loop_kernel_ms", ctypes.c_float * 3),
                ("reserved", ctypes.c_uint32), ("loop_passes", ctypes.c_uint64),
                ("sum_visits", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("stencil_blocks_per_sm", ctypes.c_uint32), ("apply_blocks_per_sm", ctypes.c_uint32),
                ("pairs_blocks_per_sm", ctypes.c_uint32), ("chunked_schedule", ctypes.c_uint32),
                ("best_ms", ctypes.c_float)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_fields", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("opts", Opts)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("passes", ctypes.c_uint64),
                ("resident", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("max_resident", ctypes.c_uint64),
                ("admitted_vertices", ctypes.c_uint64), ("capacity_vertices", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64), ("busy_s", ctypes.c_double), ("error", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("cancelled", ctypes.c_uint64)]


STAGES = ["setup", "compact", "sort", "first_pass", "loop", "finish", "edit_list", "total"]

assert ctypes.sizeof(Edit) == 16 and ctypes.sizeof(Result) == 48

EXPORTS = ["exactz_default_opts", "exactz_correct", "exactz_correct_batch", "exactz_workspace_create",
           "exactz_workspace_destroy", "exactz_workspace_bytes", "exactz_ws_correct", "exactz_ws_correct_sequence", "exactz_ws_correct_batch_sequence", "exactz_classify",
           "exactz_cp_order", "exactz_version", "exactz_ws_stats", "exactz_correct_noalloc",
           "exactz_ws_get_tuning", "exactz_ws_set_tuning", "exactz_ws_autotune", "exactz_server_create",
           "exactz_server_submit", "exactz_server_poll", "exactz_server_wait", "exactz_server_stats",
           "exactz_server_destroy", "exactz_server_cancel", "exactz_encode_edits", "exactz_decode_edits",
           "exactz_debug_fail_allocations"]

_lib = None


def lib():
    """Load the in-tree CUDA library (raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run paper_2604_01397_b300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    PP = ctypes.POINTER(ctypes.c_void_p)
    L.exactz_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.exactz_default_opts.restype = None
    L.exactz_correct.argtypes = [P, P, Dims, ctypes.c_float, ctypes.POINTER(Opts), P, P, ctypes.c_uint64,
                                 ctypes.POINTER(Result), P]
    L.exactz_correct.restype = ctypes.c_int
    L.exactz_correct_batch.argtypes = [ctypes.c_uint32, PP, PP, ctypes.POINTER(Dims),
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(Opts), PP, PP,
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Result), P]
    L.exactz_correct_batch.restype = ctypes.c_int
    L.exactz_workspace_create.argtypes = [ctypes.c_uint32, ctypes.POINTER(Dims)]
    L.exactz_workspace_create.restype = P
    L.exactz_workspace_destroy.argtypes = [P]
    L.exactz_workspace_destroy.restype = None
    L.exactz_workspace_bytes.argtypes = [P]
    L.exactz_workspace_bytes.restype = ctypes.c_uint64
    L.exactz_ws_correct.argtypes = [P, ctypes.c_uint32, PP, PP, ctypes.POINTER(Dims),
                                    ctypes.POINTER(ctypes.c_float), ctypes.POINTER(Opts), PP, PP,
                                    ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Result), P, ctypes.c_int]
    L.exactz_ws_correct.restype = ctypes.c_int
    L.exactz_ws_correct_sequence.argtypes = [P, ctypes.c_uint32, PP, PP, Dims, ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(Opts), PP, PP, ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(Result), P]
    L.exactz_ws_correct_sequence.restype = ctypes.c_int
    L.exactz_ws_correct_batch_sequence.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(Dims), PP, PP,
                                                   ctypes.POINTER(ctypes.c_float), ctypes.POINTER(Opts), PP, PP,
                                                   ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Result), P]
    L.exactz_ws_correct_batch_sequence.restype = ctypes.c_int
    L.exactz_ws_get_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    L.exactz_ws_get_tuning.restype = ctypes.c_int
    L.exactz_ws_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    L.exactz_ws_set_tuning.restype = ctypes.c_int
    L.exactz_ws_autotune.argtypes = [P, ctypes.c_uint32, PP, PP, ctypes.POINTER(Dims),
                                     ctypes.POINTER(ctypes.c_float), ctypes.POINTER(Opts), P, ctypes.c_uint32,
                                     ctypes.POINTER(Tuning)]
    L.exactz_ws_autotune.restype = ctypes.c_int
    L.exactz_ws_stats.argtypes = [P, ctypes.POINTER(Stats)]
    L.exactz_ws_stats.restype = ctypes.c_int
    L.exactz_classify.argtypes = [P, Dims, P, P, P]
    L.exactz_classify.restype = ctypes.c_int
    L.exactz_cp_order.argtypes = [P, Dims, P, ctypes.POINTER(ctypes.c_uint64), P]
    L.exactz_cp_order.restype = ctypes.c_int
    L.exactz_correct_noalloc.argtypes = [P, P, Dims, ctypes.c_float, ctypes.POINTER(Opts), P, P,
                                         ctypes.c_uint64, ctypes.POINTER(Result), P]
    L.exactz_correct_noalloc.restype = ctypes.c_int
    L.exactz_encode_edits.argtypes = [P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, P, P, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_uint64), P]
    L.exactz_encode_edits.restype = ctypes.c_int
    L.exactz_decode_edits.argtypes = [P, ctypes.c_uint64, ctypes.c_float, ctypes.c_uint32, ctypes.c_uint32, P, P, P,
                                      P]
    L.exactz_decode_edits.restype = ctypes.c_int
    L.exactz_server_create.argtypes = [ctypes.POINTER(ServerConfig)]
    L.exactz_server_create.restype = P
    L.exactz_server_submit.argtypes = [P, P, P, Dims, ctypes.c_float, P, P, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_uint64)]
    L.exactz_server_submit.restype = ctypes.c_int
    L.exactz_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(Result), ctypes.POINTER(ctypes.c_double)]
    L.exactz_server_poll.restype = ctypes.c_int
    L.exactz_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Result),
                                     ctypes.POINTER(ctypes.c_double)]
    L.exactz_server_wait.restype = ctypes.c_int
    L.exactz_server_stats.argtypes = [P, ctypes.POINTER(ServerInfo)]
    L.exactz_server_stats.restype = ctypes.c_int
    L.exactz_server_cancel.argtypes = [P, ctypes.c_uint64]
    L.exactz_server_cancel.restype = ctypes.c_int
    L.exactz_debug_fail_allocations.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    L.exactz_debug_fail_allocations.restype = ctypes.c_int
    L.exactz_server_destroy.argtypes = [P]
    L.exactz_server_destroy.restype = None
    L.exactz_version.argtypes = []
    L.exactz_version.restype = ctypes.c_char_p
    _lib = L
    return L


def ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = ctypes.c_void_p(p) if p else None
    return arr
