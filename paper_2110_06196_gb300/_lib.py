"""ctypes binding of libgrape_walk (include/grape_walk.h): argument marshalling only.

Every step of the walk runs in the library's CUDA kernels.  If the library
cannot be built or loaded, this module raises.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_i32, c_i64, c_u32, c_u64, c_dbl, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p)

GRAPE_UNDIRECTED = 1
GRAPE_VALIDATE = 2
GRAPE_FAULT_NO_HEARTBEAT = 1

STATUS = {0: "GRAPE_OK", 1: "GRAPE_ERR_INVALID_ARG", 2: "GRAPE_ERR_INVALID_GRAPH",
          3: "GRAPE_ERR_NOMEM", 4: "GRAPE_ERR_CUDA", 5: "GRAPE_ERR_TIMEOUT", 6: "GRAPE_ERR_BUSY",
          7: "GRAPE_ERR_CANCELLED", 8: "GRAPE_ERR_DEVICE", 9: "GRAPE_ERR_NOT_FOUND"}
CODES = {v: k for k, v in STATUS.items()}


class GrapeError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__(f"{what}: {self.name}" if what else self.name)


class GraphInfo(ctypes.Structure):
    _fields_ = [("num_nodes", c_i64), ("num_entries", c_i64), ("max_degree", c_i32),
                ("weighted", c_i32), ("undirected", c_i32), ("pad", c_i32),
                ("device_bytes", c_i64), ("edge_hash_bytes", c_i64)]


class Tuning(ctypes.Structure):
    _fields_ = [("trial_cap", c_i64), ("shorter_min", c_i32), ("block_threads", c_i32),
                ("blocks_per_sm", c_i32), ("chunk_walks", c_i32), ("interp_search", c_i32),
                ("l2_fetch_bytes", c_i32), ("pivot_min", c_i32), ("warp_search_min", c_i32),
                ("l2_persist_mb", c_i32), ("edge_hash", c_i32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


class WalkRequest(ctypes.Structure):
    _fields_ = [("starts", c_vp), ("num_starts", c_i64), ("walk_len", c_i32),
                ("walks_per_node", c_i32), ("p", c_dbl), ("q", c_dbl), ("seed", c_u64),
                ("out", c_vp)]


class Counters(ctypes.Structure):
    _fields_ = [("steps", c_i64), ("trials", c_i64), ("gathers", c_i64), ("searches", c_i64),
                ("probes", c_i64), ("fallbacks", c_i64), ("walks", c_i64),
                ("filtered", c_i64), ("pivot_probes", c_i64), ("hash_probes", c_i64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("output_cap_bytes", c_i64), ("max_inflight", c_i32), ("chunk_walks", c_i32),
                ("max_chunks", c_i64), ("idle_exit_us", c_i64), ("admit_timeout_ms", c_i32),
                ("kernel_wait_ms", c_i32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", c_i64), ("admitted", c_i64), ("completed", c_i64),
                ("cancelled", c_i64), ("rejected", c_i64), ("inflight", c_i64),
                ("bytes_reserved", c_i64), ("kernel_launches", c_i64), ("steps", c_i64),
                ("kernel_timeouts", c_i64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class EFInfo(ctypes.Structure):
    _fields_ = [("num_nodes", c_i64), ("num_entries", c_i64), ("universe", c_i64),
                ("num_zeros", c_i64), ("high_bits", c_i64), ("low_words", c_i64),
                ("high_words", c_i64), ("ones_index_len", c_i64), ("zeros_index_len", c_i64),
                ("structure_bytes", c_i64), ("device_bytes", c_i64), ("code_bits", c_i32),
                ("low_bits", c_i32), ("quantum", c_i32), ("weighted", c_i32),
                ("max_degree", c_i32), ("directory_rows", c_i32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class EFCounters(ctypes.Structure):
    _fields_ = [("steps", c_i64), ("trials", c_i64), ("codes_read", c_i64),
                ("membership_tests", c_i64), ("sectors", c_i64), ("fallbacks", c_i64),
                ("walks", c_i64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# name -> (restype, argtypes); mirrors include/grape_walk.h
SIGNATURES = {
    "grape_status_string": (ctypes.c_char_p, [c_i32]),
    "grape_graph_create": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i64, c_u32, c_vp, c_vp]),
    "grape_graph_destroy": (None, [c_vp]),
    "grape_graph_info": (c_i32, [c_vp, c_vp]),
    "grape_graph_get_tuning": (c_i32, [c_vp, c_vp]),
    "grape_graph_set_tuning": (c_i32, [c_vp, c_vp]),
    "grape_walks": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_dbl, c_dbl, c_u64, c_vp, c_vp]),
    "grape_walks_range": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_dbl, c_dbl, c_u64, c_i64,
                                  c_i64, c_vp, c_vp]),
    "grape_walks_host": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_dbl, c_dbl, c_u64, c_vp,
                                 c_vp]),
    "grape_trim_scratch": (c_i32, [c_i64]),
    "grape_batch_plan_create": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp]),
    "grape_batch_plan_launch": (c_i32, [c_vp, c_vp]),
    "grape_batch_plan_destroy": (None, [c_vp]),
    "grape_walks_batched": (c_i32, [c_vp, c_vp, c_i32, c_vp]),
    "grape_walks_batched_static": (c_i32, [c_vp, c_vp, c_i32, c_vp]),
    "grape_autotune_batched": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp]),
    "grape_stream_status": (c_i32, [c_vp, c_vp]),
    "grape_counters_enable": (c_i32, [c_vp, c_i32]),
    "grape_counters_read": (c_i32, [c_vp, c_vp]),
    "grape_walk_server_create": (c_i32, [c_vp, c_vp, c_vp]),
    "grape_walk_server_submit": (c_i32, [c_vp, c_vp, c_vp]),
    "grape_walk_server_wait": (c_i32, [c_vp, c_u64, c_i64, c_vp]),
    "grape_walk_server_wait_any": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp]),
    "grape_walk_server_cancel": (c_i32, [c_vp, c_u64]),
    "grape_walk_server_stats": (c_i32, [c_vp, c_vp]),
    "grape_walk_server_inject_fault": (c_i32, [c_vp, c_u32]),
    "grape_walk_server_destroy": (None, [c_vp]),
    "grape_philox4x32_10": (c_i32, [c_vp, c_i64, c_vp, c_vp]),
    "grape_sector_probe": (c_i32, [c_vp, c_i64, c_i64, c_u64, c_i32, c_i32, c_i32, c_i32, c_vp,
                                   c_vp, c_vp, c_vp]),
    "grape_contexts_from_rows": (c_i32, [c_vp, c_i64, c_i32, c_i32, c_vp, c_vp]),
    "grape_walks_approx": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_dbl, c_dbl, c_u64, c_i32,
                                   c_vp, c_vp]),
    "grape_walk_contexts": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_dbl, c_dbl, c_u64, c_i32,
                                    c_i64, c_i64, c_vp, c_vp, c_vp]),
    "grape_walks_cumsum": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_dbl, c_dbl, c_u64, c_vp,
                                   c_vp]),
    "grape_ef_graph_create": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i64, c_i32, c_u32, c_vp, c_vp]),
    "grape_ef_graph_destroy": (None, [c_vp]),
    "grape_ef_graph_info": (c_i32, [c_vp, c_vp]),
    "grape_ef_graph_export": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "grape_ef_select": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "grape_ef_rank": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "grape_ef_walks": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_dbl, c_dbl, c_u64, c_i64, c_vp,
                               c_vp]),
    "grape_ef_stream_status": (c_i32, [c_vp, c_vp]),
    "grape_ef_counters_enable": (c_i32, [c_vp, c_i32]),
    "grape_ef_counters_read": (c_i32, [c_vp, c_vp]),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libgrape_walk (building it with nvcc when stale).  Raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgrape_walk is not built ({path}); run "
                               "python -c 'import __graft_entry__ as g; g.build()'")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(code: int, what: str = ""):
    if code != 0:
        raise GrapeError(code, what)
