"""ctypes binding of libdtwknn.so (the C ABI of include/dtwknn.h).

Argument marshalling only: every step of the cascade runs in the library's
CUDA kernels.  Importing this module loads the in-tree library and fails
loudly when it is missing; there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdtwknn.so")

DTW_OK = 0
STATUS_NAMES = {
    0: "DTW_OK",
    1: "DTW_ERR_INVALID_ARG",
    2: "DTW_ERR_CUDA",
    3: "DTW_ERR_OOM",
    4: "DTW_ERR_TIMEOUT",
    5: "DTW_ERR_NO_BUCKET",
    6: "DTW_ERR_INTERNAL",
}
MODE_IMPROVED, MODE_KEOGH, MODE_NOPRUNE = 0, 1, 2
MAX_N = 4096
MAX_K = 128


class DtwError(RuntimeError):
    """A library call returned a status other than DTW_OK."""

    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


class Stats(ctypes.Structure):
    _fields_ = [
        ("candidates", ctypes.c_int64),
        ("seeds", ctypes.c_int64),
        ("pruned_summary", ctypes.c_int64),
        ("pruned_keogh", ctypes.c_int64),
        ("pruned_improved", ctypes.c_int64),
        ("dtw_computed", ctypes.c_int64),
        ("dtw_abandoned", ctypes.c_int64),
        ("dtw_cells", ctypes.c_int64),
        ("seed_cells", ctypes.c_int64),
        ("dtw_lane_rows", ctypes.c_int64),
        ("dtw_rows", ctypes.c_int64),
        ("seed_rows", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


NUM_STAGES = 10
STAGE_NAMES = ["envelope", "lb_keogh", "seed_select", "seed_dtw", "seed_kth", "lb_improved", "dtw", "finalize",
               "db_prep", "group"]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * NUM_STAGES), ("launches", ctypes.c_int64 * NUM_STAGES)]

    def as_dict(self) -> dict:
        return {name: {"ms": float(self.ms[i]), "launches": int(self.launches[i])} for i, name in enumerate(STAGE_NAMES)}


class Options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("slack", ctypes.c_float), ("seeds", ctypes.c_int32),
                ("parts", ctypes.c_int32), ("dtw_path", ctypes.c_int32), ("filter_path", ctypes.c_int32),
                ("lb_abandon", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("parts", ctypes.c_int32), ("seeds", ctypes.c_int32), ("seg_len", ctypes.c_int32),
                ("ms", ctypes.c_float), ("dtw_path", ctypes.c_int32), ("filter_warps", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"parts": int(self.parts), "seeds": int(self.seeds), "seg_len": int(self.seg_len),
                "ms": float(self.ms), "dtw_path": int(self.dtw_path), "filter_warps": int(self.filter_warps)}


class IndexStats(ctypes.Structure):
    _fields_ = [("buckets", ctypes.c_int32), ("graphs_cached", ctypes.c_int32),
                ("resident_bytes", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("graph_captures", ctypes.c_int64), ("graph_replays", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


BATCH_GRAPH, BATCH_AUTOTUNE, BATCH_SERIAL, BATCH_PER_QUERY, BATCH_PERSISTENT = 1, 2, 4, 8, 16


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("slot_bytes", ctypes.c_int64),
                ("max_wait_us", ctypes.c_int32), ("flags", ctypes.c_int32), ("batch_timeout_ms", ctypes.c_int32)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("k", ctypes.c_int32),
                ("arrival_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in ("submitted", "completed", "failed", "batches",
                                                     "max_inflight_batches", "max_batch_seen", "pending",
                                                     "inflight_batches", "timed_out")]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_f32 = ctypes.c_float

# name -> argtypes; every entry point returns dtw_status (int)
SIGNATURES = {
    "dtw_envelope": [_vp, _i64, _i32, _i32, _vp, _vp, _vp],
    "lb_keogh": [_vp, _i64, _vp, _vp, _i32, _i32, _vp, _vp],
    "lb_piecewise": [_vp, _i64, _vp, _vp, _i32, _i32, _i32, _vp, _vp],
    "lb_improved": [_vp, _i64, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp],
    "dtw_band": [_vp, _vp, _i64, _i32, _i32, _i32, _i32, _f32, _vp, _vp],
    "dtw_band_noalloc": [_vp, _vp, _i64, _i32, _i32, _i32, _i32, _f32, _vp, _vp],
    "dtw_triangle": [_vp, _vp, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp],
    "knn_search": [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _i32, _vp, _vp, ctypes.POINTER(Stats), _vp],
    "dtw_profile_enable": [_i32],
    "dtw_profile_read": [ctypes.c_void_p, _i32],
    "knn_search_ex": [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _i32, ctypes.POINTER(Options), _vp, _vp,
                      ctypes.POINTER(Stats), _vp],
    "knn_seed_thresholds": [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _i32, ctypes.POINTER(Options), _vp, _vp],
    "knn_search_bounded": [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _i32, ctypes.POINTER(Options), _vp, _vp, _vp,
                           ctypes.POINTER(Stats), _vp],
    "knn_merge_topk": [_vp, _vp, _i32, _i64, _i32, _i32, _vp, _vp, _vp],
    "dtw_index_create": [_i32, ctypes.POINTER(Options), ctypes.POINTER(_vp)],
    "dtw_index_add_bucket": [_vp, _vp, _i64, _i32],
    "dtw_index_tune": [_vp, _vp, _i64, _i32, _i32, _i32, ctypes.POINTER(Tuning)],
    "dtw_index_get_tuning": [_vp, _i32, _i32, _i32, ctypes.POINTER(Tuning)],
    "dtw_index_set_tuning": [_vp, _i32, _i32, _i32, ctypes.POINTER(Tuning)],
    "dtw_index_search": [_vp, _vp, _i64, _vp, _vp, _vp, _i32, _i32, _vp, _vp, ctypes.POINTER(Stats), _vp],
    "dtw_index_info": [_vp, ctypes.POINTER(IndexStats)],
    "dtw_index_destroy": [_vp],
    "dtw_server_create": [_vp, ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)],
    "dtw_server_submit": [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _i64, ctypes.POINTER(ctypes.c_uint64)],
    "dtw_server_poll": [_vp, _vp, _i32, ctypes.POINTER(_i32), _i32],
    "dtw_server_info": [_vp, ctypes.POINTER(ServerStats)],
    "dtw_server_destroy": [_vp],
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdtwknn.so is not built (%s); run `python -m paper_0811_3301_gb300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.dtw_last_error.argtypes = []
    lib.dtw_last_error.restype = ctypes.c_char_p
    lib.dtw_version.argtypes = []
    lib.dtw_version.restype = ctypes.c_char_p
    lib.dtw_monotonic_ns.argtypes = []
    lib.dtw_monotonic_ns.restype = ctypes.c_int64
    return lib


lib = _load()


def check(status: int) -> None:
    if status != DTW_OK:
        raise DtwError(status, lib.dtw_last_error().decode(errors="replace"))


def profile_enable(on: bool) -> None:
    check(lib.dtw_profile_enable(1 if on else 0))


def profile_read(reset: bool = True) -> dict:
    p = Profile()
    check(lib.dtw_profile_read(ctypes.byref(p), 1 if reset else 0))
    return p.as_dict()


def version() -> str:
    return lib.dtw_version().decode()
