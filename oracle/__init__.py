"""FP64 CPU oracle for the DTW retrieval cascade (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It wraps `dtw_oracle.c` (plain C, fp64)
through ctypes; it shares no code with the CUDA library.  The C source is
compiled on first use with the host compiler (`build()`).

Every function takes fp32 numpy arrays (the exact values the CUDA path
receives) and returns float64 results.  ctypes releases the GIL during a
foreign call, so the per-query loops below run on several host threads when
`threads > 1` without changing any arithmetic.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dtw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile dtw_oracle.c into liboracle.so beside it (host gcc, fp64, no fast-math)."""
    stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_envelope.argtypes = [_f32p, _i64, _i64, _f64p, _f64p]
            lib.oracle_envelope.restype = None
            lib.oracle_envelope_d.argtypes = [_f64p, _i64, _i64, _f64p, _f64p]
            lib.oracle_envelope_d.restype = None
            lib.oracle_projection.argtypes = [_f64p, _f64p, _f64p, _i64, _f64p]
            lib.oracle_projection.restype = None
            lib.oracle_lb_keogh_pow.argtypes = [_f32p, _f64p, _f64p, _i64, ctypes.c_int]
            lib.oracle_lb_keogh_pow.restype = ctypes.c_double
            lib.oracle_lb_improved_pow.argtypes = [_f32p, _f32p, _f64p, _f64p, _i64, _i64, ctypes.c_int, _f64p]
            lib.oracle_lb_improved_pow.restype = ctypes.c_double
            lib.oracle_lb_piecewise_pow.argtypes = [_f32p, _f64p, _f64p, _i64, _i64, ctypes.c_int]
            lib.oracle_lb_piecewise_pow.restype = ctypes.c_double
            lib.oracle_dtw_pow.argtypes = [_f32p, _f32p, _i64, _i64, ctypes.c_int]
            lib.oracle_dtw_pow.restype = ctypes.c_double
            lib.oracle_knn_bruteforce.argtypes = [_f32p, _i64, _f32p, _i64, _i64, ctypes.c_int, ctypes.c_int, _i64p, _f64p]
            lib.oracle_knn_bruteforce.restype = None
            lib.oracle_knn_cascade.argtypes = [_f32p, _i64, _f32p, _i64, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p, _f64p, _i64p]
            lib.oracle_knn_cascade.restype = None
            _lib = lib
    return _lib


def _f32(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _check_w(w: int) -> int:
    if w < 0:
        raise ValueError("w must be >= 0")
    return int(w)


def envelope(y, w: int):
    """(U, L) of one series y (Sec. 5 definition), float64."""
    lib = _load()
    y = _f32(y)
    n = y.shape[-1]
    U = np.empty(n, np.float64)
    L = np.empty(n, np.float64)
    lib.oracle_envelope(_ptr(y, _f32p), n, _check_w(w), _ptr(U, _f64p), _ptr(L, _f64p))
    return U, L


def envelope_f64(y, w: int):
    """(U, L) of a float64 series (used for envelopes of projections)."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = y.shape[-1]
    U = np.empty(n, np.float64)
    L = np.empty(n, np.float64)
    lib.oracle_envelope_d(_ptr(y, _f64p), n, _check_w(w), _ptr(U, _f64p), _ptr(L, _f64p))
    return U, L


def projection(x, U, L):
    """H(x, y) given U = U(y), L = L(y) (Eq. 1), float64."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    H = np.empty_like(x)
    lib.oracle_projection(_ptr(x, _f64p), _ptr(U, _f64p), _ptr(L, _f64p), x.shape[-1], _ptr(H, _f64p))
    return H


def lb_keogh_pow(x, y, w: int, p: int) -> float:
    """LB_Keogh_p(x, y)^p (Sec. 7)."""
    lib = _load()
    x = _f32(x)
    U, L = envelope(y, w)
    return lib.oracle_lb_keogh_pow(_ptr(x, _f32p), _ptr(U, _f64p), _ptr(L, _f64p), x.shape[-1], int(p))


def lb_improved_pow(x, y, w: int, p: int, with_first: bool = False):
    """LB_Improved_p(x, y)^p (Sec. 8); with_first also returns LB_Keogh_p^p."""
    lib = _load()
    x = _f32(x)
    y = _f32(y)
    U, L = envelope(y, w)
    first = ctypes.c_double(0.0)
    r = lib.oracle_lb_improved_pow(_ptr(x, _f32p), _ptr(y, _f32p), _ptr(U, _f64p), _ptr(L, _f64p),
                                   x.shape[-1], _check_w(w), int(p), ctypes.byref(first))
    return (r, first.value) if with_first else r


def lb_piecewise_pow(x, y, w: int, d: int, p: int) -> float:
    """Piecewise-sum bound of Sec. 9 (p-th power), cover of d parts."""
    lib = _load()
    x = _f32(x)
    n = x.shape[-1]
    if not 1 <= d <= n:
        raise ValueError("1 <= d <= n required")
    U, L = envelope(y, w)
    return lib.oracle_lb_piecewise_pow(_ptr(x, _f32p), _ptr(U, _f64p), _ptr(L, _f64p), n, int(d), int(p))


def dtw_pow(x, y, w: int, p: int) -> float:
    """DTW_p(x, y)^p by the Sec. 4 recursion (p = 0: DTW_inf itself)."""
    lib = _load()
    x = _f32(x)
    y = _f32(y)
    if x.shape != y.shape:
        raise ValueError("equal-length series required")
    return lib.oracle_dtw_pow(_ptr(x, _f32p), _ptr(y, _f32p), x.shape[-1], _check_w(w), int(p))


def dtw(x, y, w: int, p: int) -> float:
    """DTW_p(x, y) with the root taken (p = 0: DTW_inf)."""
    v = dtw_pow(x, y, w, p)
    if p in (0, 1):
        return v
    return v ** (1.0 / p)


def _per_query(fn, queries: np.ndarray, threads: int):
    if threads <= 1 or len(queries) <= 1:
        return [fn(qi) for qi in range(len(queries))]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, range(len(queries))))


def knn_bruteforce(db, queries, w: int, p: int, k: int, threads: int = 1):
    """Exact k-NN by definition: (idx int64 [Q,k], dist float64 [Q,k]), DTW_p with root."""
    lib = _load()
    db = _f32(db)
    queries = _f32(np.atleast_2d(queries))
    N, n = db.shape
    Q = queries.shape[0]
    if queries.shape[1] != n:
        raise ValueError("query length must equal the database length")
    idx = np.empty((Q, k), np.int64)
    dist = np.empty((Q, k), np.float64)

    def one(qi):
        lib.oracle_knn_bruteforce(_ptr(db, _f32p), N, _ptr(queries[qi], _f32p), n, _check_w(w), int(p), int(k),
                                  _ptr(idx[qi], _i64p), _ptr(dist[qi], _f64p))

    _per_query(one, queries, threads)
    return idx, dist


def knn_cascade(db, queries, w: int, p: int, k: int, mode: int = 1, threads: int = 1):
    """Algorithm 2 (mode 0) or Algorithm 3 (mode 1) scan per query.

    Returns (idx [Q,k], dist [Q,k], stats [Q,4]) where stats columns are
    candidates, discarded by LB_Keogh, discarded by LB_Improved, DTW computed.
    """
    lib = _load()
    db = _f32(db)
    queries = _f32(np.atleast_2d(queries))
    N, n = db.shape
    Q = queries.shape[0]
    if queries.shape[1] != n:
        raise ValueError("query length must equal the database length")
    idx = np.empty((Q, k), np.int64)
    dist = np.empty((Q, k), np.float64)
    stats = np.zeros((Q, 4), np.int64)

    def one(qi):
        lib.oracle_knn_cascade(_ptr(db, _f32p), N, _ptr(queries[qi], _f32p), n, _check_w(w), int(p), int(k), int(mode),
                               _ptr(idx[qi], _i64p), _ptr(dist[qi], _f64p), _ptr(stats[qi], _i64p))

    _per_query(one, queries, threads)
    return idx, dist, stats
