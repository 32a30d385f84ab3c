"""ctypes binding of ``libdpgpu.so`` (the C ABI in ``include/dpgpu.h``).

Argument marshalling only: every step of the solvers runs in the library's
CUDA kernels.  PyTorch tensors provide device memory and streams.  The
library is loaded from this package directory; when it is missing the
binding raises instead of computing anything another way.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdpgpu.so")

DP_OK, DP_EINVAL, DP_ENOMEM, DP_ECUDA, DP_EOVERFLOW, DP_ETIMEOUT, DP_EBUSY, DP_EPENDING = range(8)
DP_COST_I32, DP_COST_I64 = 0, 1
DP_OP_MIN, DP_OP_ADD_MOD32 = 0, 1
DP_REQ_MCM, DP_REQ_SDP = 0, 1

STATUS_NAMES = {0: "DP_OK", 1: "DP_EINVAL", 2: "DP_ENOMEM", 3: "DP_ECUDA", 4: "DP_EOVERFLOW",
                5: "DP_ETIMEOUT", 6: "DP_EBUSY", 7: "DP_EPENDING"}

# Every function declared in include/dpgpu.h (checked by the ABI test).
HEADER_SYMBOLS = [
    "dp_last_error", "dp_version", "dp_sync_status", "dp_profile_begin", "dp_profile_end", "dp_measure_int32_rates",
    "mcm_solve", "interval_dp_solve", "mcm_solve_noalloc", "mcm_traceback", "mcm_solve_host", "mcm_plan_create", "mcm_solve_batched",
    "mcm_plan_autotune", "mcm_plan_config", "mcm_plan_destroy",
    "sdp_solve", "sdp_solve_host", "sdp_plan_create", "sdp_solve_batched", "sdp_plan_destroy",
    "serve_create", "serve_submit", "serve_poll", "serve_release", "serve_release_stream", "serve_now", "serve_destroy",
]


class DpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_cap_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("num_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("device", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("cost", ctypes.c_int32), ("n", ctypes.c_int64),
                ("dims", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("k", ctypes.c_int32),
                ("op", ctypes.c_int32), ("preset", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("n", ctypes.c_int64),
                ("m_dev", ctypes.c_void_p), ("s_dev", ctypes.c_void_p), ("st_dev", ctypes.c_void_p),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Loads the library (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"native library {p} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (there is no fallback path)")
        lib = ctypes.CDLL(p)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        sig = {
            "dp_last_error": ([], ctypes.c_char_p),
            "dp_version": ([], ctypes.c_char_p),
            "dp_sync_status": ([vp, vp], ctypes.c_int),
            "dp_profile_begin": ([], ctypes.c_int),
            "dp_profile_end": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)], ctypes.c_int),
            "dp_measure_int32_rates": ([ctypes.POINTER(ctypes.c_double), i32, vp], ctypes.c_int),
            "mcm_solve": ([vp, i32, ctypes.c_int, vp, vp, vp, vp], ctypes.c_int),
            "mcm_solve_noalloc": ([vp, i32, vp, vp, vp, vp], ctypes.c_int),
            "mcm_traceback": ([vp, i32, vp, vp, vp], ctypes.c_int),
            "interval_dp_solve": ([vp, vp, i32, ctypes.c_int, vp, vp, vp, vp], ctypes.c_int),
            "mcm_solve_host": ([vp, i32, ctypes.c_int, vp, vp, vp], ctypes.c_int),
            "mcm_plan_create": ([i32, vp, ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
            "mcm_solve_batched": ([vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
            "mcm_plan_autotune": ([vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
            "mcm_plan_config": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
            "mcm_plan_destroy": ([vp], ctypes.c_int),
            "dp_mcm_plan_tasks": ([vp], i64),
            "dp_test_host_range_device_address": ([vp, ctypes.c_size_t, ctypes.c_int], vp),
            "dp_test_mcm_queue": ([vp, i32, i32, vp, i32], i32),
            "dp_test_sdp_jump_chunks": ([i64, vp, i32], i32),
            "dp_test_sdp_jump_plan": ([i64, vp, i32, i32, vp], i32),
            "dp_test_sdp_jump": ([vp, i64, vp, i32, i32, vp, vp], ctypes.c_int),
            "dp_test_sdp_min_jump_chunks": ([i64, vp, i32], i32),
            "dp_test_sdp_min_jump_plan": ([i64, vp, i32, i32, vp], i32),
            "dp_test_sdp_min_jump": ([vp, i64, vp, i32, i32, vp, vp], ctypes.c_int),
            "dp_test_mcm_drop_task": ([vp, i32, ctypes.c_int, vp, vp, vp, vp, i32, ctypes.c_longlong], ctypes.c_int),
            "sdp_solve": ([vp, i64, vp, i32, ctypes.c_int, vp, vp], ctypes.c_int),
            "sdp_solve_host": ([vp, i64, vp, i32, ctypes.c_int, vp], ctypes.c_int),
            "sdp_plan_create": ([i32, vp, vp, vp, ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
            "sdp_solve_batched": ([vp, vp, vp, vp, vp], ctypes.c_int),
            "sdp_plan_destroy": ([vp], ctypes.c_int),
            "serve_create": ([ctypes.POINTER(ServeConfig), ctypes.POINTER(vp)], ctypes.c_int),
            "serve_submit": ([vp, ctypes.POINTER(Request), ctypes.POINTER(u64)], ctypes.c_int),
            "serve_poll": ([vp, u64, ctypes.POINTER(Result)], ctypes.c_int),
            "serve_release": ([vp, u64], ctypes.c_int),
            "serve_release_stream": ([vp, u64, vp], ctypes.c_int),
            "serve_now": ([vp], ctypes.c_double),
            "serve_destroy": ([vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name, None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def last_error() -> str:
    return load().dp_last_error().decode(errors="replace")


def check(code: int) -> None:
    if code != DP_OK:
        raise DpError(code, last_error())
