"""ctypes declarations of the libptk C ABI (include/ptk.h).

Argument marshalling only: every computation runs in libptk's CUDA kernels.
Loading fails loudly when the in-tree libptk.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

MAX_ORDER = 10
MAX_RANK = 16

OK, ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_BUSY, ERR_NUMERIC = range(8)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "UNSUPPORTED", 5: "TIMEOUT",
                6: "BUSY", 7: "NUMERIC"}

F32, F64 = 0, 1
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "bf16x3": 4}
VARIANT = {"plain": 0, "cache": 1, "approx": 2}
TRUNC = {"r_beta": 0, "magnitude": 1}
SCHEDULE = {"auto": 0, "entries": 1, "rows_static": 2, "rows_dynamic": 3, "tensor": 4}
TIMERS = ["slices", "delta", "gram", "solve", "error", "cache", "approx", "qr", "foldin"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libptk.so")


class Coo(C.Structure):
    _fields_ = [("order", C.c_int32), ("dims", C.c_int64 * MAX_ORDER), ("nnz", C.c_int64),
                ("idx", C.c_void_p), ("vals", C.c_void_p), ("dtype", C.c_int)]


class Model(C.Structure):
    _fields_ = [("order", C.c_int32), ("J", C.c_int32 * MAX_ORDER), ("dims", C.c_int64 * MAX_ORDER),
                ("core", C.c_void_p), ("factors", C.c_void_p * MAX_ORDER), ("ld", C.c_int64 * MAX_ORDER),
                ("dtype", C.c_int)]


class AlsOpts(C.Structure):
    _fields_ = [("variant", C.c_int), ("precision", C.c_int), ("lam", C.c_double), ("trunc_rate", C.c_double),
                ("trunc_rule", C.c_int), ("error_pass", C.c_int32), ("schedule", C.c_int)]


class SweepStats(C.Structure):
    _fields_ = [("sse", C.c_double), ("error", C.c_double), ("rmse", C.c_double), ("loss", C.c_double),
                ("core_nnz", C.c_int64), ("bad_rows", C.c_int64)]


class Problem(C.Structure):
    _fields_ = [("x", Coo), ("slices", C.c_void_p * MAX_ORDER), ("model", Model)]


class FitOpts(C.Structure):
    _fields_ = [("als", AlsOpts), ("max_sweeps", C.c_int32), ("tol", C.c_double), ("finalize_qr", C.c_int32),
                ("lanes", C.c_int32), ("graphs", C.c_int32), ("autotune", C.c_int32)]


TUNE_MAX = 16


class TuneReport(C.Structure):
    _fields_ = [("candidates", C.c_int32), ("best", C.c_int32), ("entries", C.c_int64),
                ("backend", C.c_int32 * TUNE_MAX), ("chunk_kb", C.c_int32 * TUNE_MAX),
                ("ctas_per_sm", C.c_int32 * TUNE_MAX), ("entries_per_thread", C.c_int32 * TUNE_MAX),
                ("ms", C.c_float * TUNE_MAX)]


class FoldinBatch(C.Structure):
    _fields_ = [("count", C.c_int32), ("obs_ptr", C.c_void_p), ("obs_idx", C.c_void_p), ("obs_vals", C.c_void_p),
                ("query_ptr", C.c_void_p), ("query_idx", C.c_void_p), ("rows_out", C.c_void_p),
                ("preds_out", C.c_void_p), ("total_obs", C.c_int64), ("total_query", C.c_int64)]


class ServerOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("lam", C.c_double), ("precision", C.c_int), ("max_batch_requests", C.c_int32),
                ("max_batch_entries", C.c_int64), ("max_batch_queries", C.c_int64), ("memory_cap_bytes", C.c_int64),
                ("slots", C.c_int32), ("max_queue", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64), ("batches", C.c_int64),
                ("queued", C.c_int64), ("inflight_bytes", C.c_int64), ("max_inflight_bytes", C.c_int64)]


class DServerOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("lam", C.c_double), ("ring", C.c_int32), ("arena_bytes", C.c_int64),
                ("max_queries", C.c_int64), ("max_pending", C.c_int64), ("workers", C.c_int32),
                ("idle_ms", C.c_double)]


class DServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64), ("launches", C.c_int64),
                ("idle_exits", C.c_int64), ("served_on_device", C.c_int64), ("bad_rows", C.c_int64),
                ("pending", C.c_int64), ("inflight", C.c_int64), ("running", C.c_int32)]


# every symbol include/ptk.h declares, with its ctypes signature
SIGNATURES = {
    "ptk_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "ptk_destroy": (None, [C.c_void_p]),
    "ptk_last_error": (C.c_char_p, []),
    "ptk_version": (C.c_char_p, []),
    "ptk_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "ptk_read_timers": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ptk_launch_count": (C.c_int64, []),
    "ptk_build_mode_slices": (C.c_int, [C.c_void_p, C.POINTER(Coo), C.c_int32, C.c_int, C.POINTER(C.c_void_p),
                                        C.c_void_p]),
    "ptk_slices_destroy": (None, [C.c_void_p]),
    "ptk_slices_view": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "ptk_slices_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ptk_als_mode": (C.c_int, [C.c_void_p, C.POINTER(Coo), C.c_void_p, C.POINTER(Model), C.c_int32, C.c_int64,
                               C.c_int64, C.POINTER(AlsOpts), C.c_void_p]),
    "ptk_als_sweep": (C.c_int, [C.c_void_p, C.POINTER(Coo), C.POINTER(C.c_void_p), C.POINTER(Model),
                                C.POINTER(AlsOpts), C.POINTER(SweepStats), C.c_void_p]),
    "ptk_sweep_stats_read": (C.c_int, [C.c_void_p, C.POINTER(SweepStats), C.c_void_p]),
    "ptk_error": (C.c_int, [C.c_void_p, C.POINTER(Coo), C.POINTER(Model), C.c_double, C.POINTER(SweepStats),
                            C.c_void_p]),
    "ptk_partial_error": (C.c_int, [C.c_void_p, C.POINTER(Coo), C.POINTER(Model), C.c_void_p, C.c_void_p]),
    "ptk_fit": (C.c_int, [C.c_void_p, C.POINTER(Problem), C.c_int32, C.POINTER(FitOpts), C.c_void_p, C.c_void_p,
                          C.c_void_p]),
    "ptk_qr_finalize": (C.c_int, [C.c_void_p, C.POINTER(Model), C.c_void_p]),
    "ptk_autotune_delta": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Model), C.c_int, C.c_int64, C.c_int32,
                                     C.POINTER(TuneReport), C.c_void_p]),
    "ptk_autotune_clear": (None, [C.c_void_p]),
    "ptk_selftest_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "ptk_delta": (C.c_int, [C.c_void_p, C.POINTER(Model), C.c_int32, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                            C.c_void_p]),
    "ptk_delta_noalloc": (C.c_int, [C.POINTER(Model), C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ptk_row_sums": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                               C.c_int64, C.c_int64, C.c_int, C.c_int32, C.c_void_p, C.c_void_p]),
    "ptk_delta_tc_supported": (C.c_int, [C.POINTER(Model), C.c_int32, C.c_int]),
    "ptk_predict": (C.c_int, [C.c_void_p, C.POINTER(Model), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "ptk_foldin": (C.c_int, [C.c_void_p, C.POINTER(Model), C.c_int32, C.POINTER(FoldinBatch), C.c_double, C.c_int,
                             C.c_void_p]),
    "ptk_server_create": (C.c_int, [C.POINTER(Model), C.c_int, C.POINTER(ServerOpts), C.POINTER(C.c_void_p)]),
    "ptk_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.POINTER(C.c_uint64)]),
    "ptk_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32),
                                  C.POINTER(C.c_double)]),
    "ptk_server_read_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "ptk_server_destroy": (None, [C.c_void_p]),
    "ptk_dserver_create": (C.c_int, [C.POINTER(Model), C.c_int, C.POINTER(DServerOpts), C.POINTER(C.c_void_p)]),
    "ptk_dserver_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double,
                                     C.POINTER(C.c_uint64)]),
    "ptk_dserver_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_double)]),
    "ptk_dserver_read_stats": (C.c_int, [C.c_void_p, C.POINTER(DServerStats)]),
    "ptk_dserver_destroy": (None, [C.c_void_p]),
    "ptk_clock_seconds": (C.c_double, []),
}

_lib = None


class PtkError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libptk.so (built by ``paper_1710_02261_gb300.build``); raises when absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libptk.so not found at {path}: build it with "
                          f"`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != OK:
        raise PtkError(status, where, load().ptk_last_error().decode())
