"""ctypes declarations of the C ABI in include/mplpp.h (argument marshalling only).

The library is built in-tree (``build.py``) and loaded from
``paper_2004_08227_gb300/_build/libmplpp.so``.  If it cannot be built or
loaded, every entry point raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_i32, c_i64, c_f32p, c_i32p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p

MPLPP_OK = 0
STATUS = {0: "MPLPP_OK", -1: "MPLPP_E_INVALID", -2: "MPLPP_E_NOMEM", -3: "MPLPP_E_CUDA",
          -4: "MPLPP_E_TIMEOUT", -5: "MPLPP_E_NONFINITE", -6: "MPLPP_E_STATE", -7: "MPLPP_E_UNSUPPORTED"}
SCHED = {"round_robin": 0, "greedy_color": 1, "alg1": 2, "user": 3}
MODE = {"auto": 0, "looped": 1, "persistent": 2, "warp": 3, "structured": 4, "queue": 5, "resident": 6,
        "structured_queue": 7}
PAIR = {"dense": 0, "trunc_linear": 1, "trunc_quad": 2}  # tables, or w min(|s - t|, tau) / w min((s - t)^2, tau)
MODE_NAME = {v: k for k, v in MODE.items()}
RULE = {"H": 0, "M": 1, "U": 2}  # Sec. 4: eqs. (H), (M), (U)

# Every symbol include/mplpp.h declares.
EXPORTS = ["mplpp_options_default", "mplpp_schedule", "mplpp_create", "mplpp_run", "mplpp_bound",
           "mplpp_labeling", "mplpp_backward", "mplpp_reset", "mplpp_state_size", "mplpp_save_state",
           "mplpp_load_state", "mplpp_info", "mplpp_sync", "mplpp_last_error", "mplpp_destroy",
           "mplpp_bound_noalloc", "mplpp_noalloc_last_error", "mplpp_autotune", "mplpp_update_costs"]


class MplppModel(ctypes.Structure):
    _fields_ = [("n_nodes", c_i32), ("n_edges", c_i32), ("labels", ctypes.c_void_p),
                ("edge_u", ctypes.c_void_p), ("edge_v", ctypes.c_void_p), ("unary", ctypes.c_void_p),
                ("pairwise", ctypes.c_void_p), ("schedule_kind", c_i32), ("n_matchings", c_i32),
                ("matching_off", ctypes.c_void_p), ("edge_order", ctypes.c_void_p), ("pair_kind", c_i32),
                ("reserved", c_i32), ("pair_param", ctypes.c_void_p)]


class MplppOptions(ctypes.Structure):
    _fields_ = [("mode", c_i32), ("use_graph", c_i32), ("inputs_on_device", c_i32), ("record_every", c_i32),
                ("cluster", c_i32), ("threads", c_i32), ("test_unreachable_wait", c_i32), ("rule", c_i32),
                ("spin_limit", c_i64), ("test_backward", c_i32), ("reserved", c_i32)]


class MplppInfo(ctypes.Structure):
    _fields_ = [("iterations", c_i64), ("bytes_per_iteration", c_i64), ("edges", c_i64), ("phases", c_i32),
                ("mode", c_i32), ("cluster", c_i32), ("threads", c_i32), ("grid", c_i32),
                ("launches_per_iteration", c_i32), ("labeling_launches", c_i32), ("poller_warp", c_i32),
                ("device_bytes", c_i64)]


class MplppStateHeader(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint32), ("shape_hash", ctypes.c_uint64),
                ("iterations", c_i64), ("n_unary", c_i64), ("n_msg", c_i64)]


class MplppError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Loads (building first if needed) the solver library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"solver library missing: {_build.LIB} (run __graft_entry__.build())")
        lib = ctypes.CDLL(_build.LIB)
        P = ctypes.c_void_p
        lib.mplpp_options_default.argtypes = [P]
        lib.mplpp_options_default.restype = None
        lib.mplpp_schedule.argtypes = [c_i32, c_i32, c_i32, P, P, P, P, P]
        lib.mplpp_create.argtypes = [P, c_i32, P, P, P]
        lib.mplpp_run.argtypes = [P, c_i32]
        lib.mplpp_bound.argtypes = [P, P, c_i32]
        lib.mplpp_labeling.argtypes = [P, P, P]
        lib.mplpp_backward.argtypes = [P, P, P, P]
        lib.mplpp_reset.argtypes = [P]
        lib.mplpp_update_costs.argtypes = [P, P, P]
        lib.mplpp_state_size.argtypes = [P, P]
        lib.mplpp_save_state.argtypes = [P, P, ctypes.c_size_t]
        lib.mplpp_load_state.argtypes = [P, P, ctypes.c_size_t]
        lib.mplpp_info.argtypes = [P, P]
        lib.mplpp_sync.argtypes = [P]
        lib.mplpp_last_error.argtypes = [P]
        lib.mplpp_last_error.restype = ctypes.c_char_p
        lib.mplpp_destroy.argtypes = [P]
        lib.mplpp_destroy.restype = None
        lib.mplpp_bound_noalloc.argtypes = [c_i32, c_i32, P, P, P, P, P, P, P, P]
        lib.mplpp_autotune.argtypes = [P, c_i32, P, ctypes.c_size_t]
        lib.mplpp_noalloc_last_error.argtypes = []
        lib.mplpp_noalloc_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("mplpp_options_default", "mplpp_last_error", "mplpp_destroy", "mplpp_noalloc_last_error"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def check(status: int, solver=None):
    if status != MPLPP_OK:
        lib = load()
        msg = lib.mplpp_last_error(solver)
        raise MplppError(status, msg.decode() if msg else "")
