"""Python entry points of the DTW retrieval cascade, one per C-ABI call.

Each function checks and marshals torch tensors (device memory and the
current CUDA stream come from PyTorch) and calls the same-named function of
libdtwknn.so; all arithmetic runs in the library's sm_103a kernels.
Bounds and distances carry the p-th root, as in the paper.
"""

from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _native as N

__all__ = ["dtw_envelope", "lb_keogh", "lb_piecewise", "lb_improved", "dtw_band", "dtw_triangle", "knn_search",
           "DtwIndex",
           "DtwServer", "DtwError", "monotonic_ns", "version"]

DtwError = N.DtwError
version = N.version

_MODES = {"improved": N.MODE_IMPROVED, "keogh": N.MODE_KEOGH, "noprune": N.MODE_NOPRUNE}


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _cuda_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float32:
        raise TypeError("%s must be float32" % name)
    return t.contiguous()


def _f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32:
        raise TypeError("%s must be a float32 tensor" % name)
    return t.contiguous()


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def dtw_envelope(y: torch.Tensor, w: int, U: torch.Tensor | None = None, L: torch.Tensor | None = None):
    """Warping envelope (U, L) of each row of y ([count, n] or [n]), Sec. 5."""
    y = _cuda_f32(y, "y")
    y2 = y.reshape(-1, y.shape[-1])
    U = torch.empty_like(y2) if U is None else U
    L = torch.empty_like(y2) if L is None else L
    N.check(N.lib.dtw_envelope(_ptr(y2), y2.shape[0], y2.shape[1], int(w), _ptr(U), _ptr(L), _stream()))
    return U.reshape(y.shape), L.reshape(y.shape)


def lb_keogh(cand: torch.Tensor, U: torch.Tensor, L: torch.Tensor, p: int, out: torch.Tensor | None = None):
    """LB_Keogh_p of every row of cand [N, n] against one query envelope U, L [n] (Sec. 7)."""
    cand = _cuda_f32(cand, "cand")
    U = _cuda_f32(U, "U")
    L = _cuda_f32(L, "L")
    n = cand.shape[-1]
    if U.numel() != n or L.numel() != n:
        raise ValueError("U and L must have n = %d elements" % n)
    out = torch.empty(cand.shape[0], device=cand.device, dtype=torch.float32) if out is None else out
    N.check(N.lib.lb_keogh(_ptr(cand), cand.shape[0], _ptr(U), _ptr(L), n, int(p), _ptr(out), _stream()))
    return out


def lb_piecewise(cand: torch.Tensor, U: torch.Tensor, L: torch.Tensor, d: int, p: int,
                 out: torch.Tensor | None = None):
    """Piecewise-sum bound of Sec. 9 (d parts) of every row of cand [N, n] against one envelope."""
    cand = _cuda_f32(cand, "cand")
    U = _cuda_f32(U, "U")
    L = _cuda_f32(L, "L")
    n = cand.shape[-1]
    if U.numel() != n or L.numel() != n:
        raise ValueError("U and L must have n = %d elements" % n)
    out = torch.empty(cand.shape[0], device=cand.device, dtype=torch.float32) if out is None else out
    N.check(N.lib.lb_piecewise(_ptr(cand), cand.shape[0], _ptr(U), _ptr(L), n, int(d), int(p), _ptr(out),
                               _stream()))
    return out


def lb_improved(cand: torch.Tensor, q: torch.Tensor, U: torch.Tensor, L: torch.Tensor, w: int, p: int,
                out: torch.Tensor | None = None):
    """LB_Improved_p of every row of cand [N, n] against query q [n] with envelope U, L (Sec. 8)."""
    cand = _cuda_f32(cand, "cand")
    q = _cuda_f32(q, "q")
    U = _cuda_f32(U, "U")
    L = _cuda_f32(L, "L")
    n = cand.shape[-1]
    if q.numel() != n or U.numel() != n or L.numel() != n:
        raise ValueError("q, U and L must have n = %d elements" % n)
    out = torch.empty(cand.shape[0], device=cand.device, dtype=torch.float32) if out is None else out
    N.check(N.lib.lb_improved(_ptr(cand), cand.shape[0], _ptr(q), _ptr(U), _ptr(L), n, int(w), int(p),
                              _ptr(out), _stream()))
    return out


def _p_code(p) -> int:
    """The C ABI's code for p: 1, 2, 4, or DTW_P_INF (0) for p = infinity."""
    if p in (math.inf, "inf"):
        return 0
    return int(p)


def dtw_band(x: torch.Tensor, y: torch.Tensor, w: int, p, threshold: float = math.inf,
             out: torch.Tensor | None = None):
    """DTW_p with band w of the rows of x [N, n] against y ([n] shared, or [N, n] per pair), Sec. 4.

    p is 1, 2, 4 or math.inf (DTW_inf).  With a finite threshold, pairs whose
    DTW_p exceeds it return +inf.
    """
    x = _cuda_f32(x, "x")
    y = _cuda_f32(y, "y")
    n = x.shape[-1]
    if y.dim() == 1:
        if y.shape[0] != n:
            raise ValueError("y must have n = %d elements" % n)
        stride = 0
    else:
        if y.shape != x.shape:
            raise ValueError("per-pair y must have the shape of x")
        stride = n
    out = torch.empty(x.shape[0], device=x.device, dtype=torch.float32) if out is None else out
    N.check(N.lib.dtw_band(_ptr(x), _ptr(y), x.shape[0], stride, n, int(w), _p_code(p), float(threshold),
                           _ptr(out), _stream()))
    return out


def dtw_triangle(x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, w: int, p: int, with_distances: bool = False):
    """Triangle-inequality ratios DTW_p(x,z) / (DTW_p(x,y) + DTW_p(y,z)) of the
    rows of x, y, z ([N, n] each), App. B.  With with_distances also the
    [3, N] distances (x,y), (y,z), (x,z)."""
    x = _cuda_f32(x, "x")
    y = _cuda_f32(y, "y")
    z = _cuda_f32(z, "z")
    if not (x.shape == y.shape == z.shape) or x.dim() != 2:
        raise ValueError("x, y and z must be [N, n] of one shape")
    N_, n = x.shape
    ratio = torch.empty(N_, device=x.device, dtype=torch.float32)
    d3 = torch.empty((3, N_), device=x.device, dtype=torch.float32) if with_distances else None
    N.check(N.lib.dtw_triangle(_ptr(x), _ptr(y), _ptr(z), N_, n, int(w), int(p), _ptr(ratio), _ptr(d3), _stream()))
    return (ratio, d3) if with_distances else ratio


def _knn_args(db, queries, mode, slack, seeds, parts, dtw_path, filter_path, lb_abandon):
    db = _f32(db, "db")
    queries = _f32(queries, "queries")
    if queries.dim() == 1:
        queries = queries.unsqueeze(0)
    if db.dim() != 2 or queries.dim() != 2 or db.shape[1] != queries.shape[1]:
        raise ValueError("db [N, n] and queries [Q, n] must share n")
    if mode not in _MODES:
        raise ValueError("mode must be one of %s" % sorted(_MODES))
    opt = N.Options(_MODES[mode], float(slack), int(seeds), int(parts), int(dtw_path), int(filter_path),
                    int(lb_abandon))
    return db, queries, opt


def knn_search(db: torch.Tensor, queries: torch.Tensor, w: int, p: int, k: int = 1, *, mode: str = "improved",
               slack: float = 1e-6, seeds: int = 0, parts: int = 0, dtw_path: int = 0, filter_path: int = 0,
               lb_abandon: int = 0,
               out_idx: torch.Tensor | None = None,
               out_dist: torch.Tensor | None = None, return_stats: bool = False,
               thr_in: torch.Tensor | None = None):
    """Exact k nearest neighbours of each query row under DTW_p with band w (Sec. 7-8).

    db [N, n] and queries [Q, n] may live on the GPU or in host memory
    (host tensors are copied by the library).  Returns (idx int64 [Q, k],
    dist float32 [Q, k]) ordered by (distance, index); with return_stats
    also the cascade counters.  Outputs default to the device of `queries`
    when it is a CUDA tensor, else to host memory.

    thr_in (float32 [Q], power units as knn_seed_thresholds gives them)
    makes this the search of one shard of a candidate-sharded database (the
    C call knn_search_bounded): each query's threshold is lowered to thr_in,
    and only candidates within the final threshold are listed.
    """
    db, queries, opt = _knn_args(db, queries, mode, slack, seeds, parts, dtw_path, filter_path, lb_abandon)
    Q, n = queries.shape
    dev = queries.device
    if out_idx is None:
        out_idx = torch.empty((Q, k), dtype=torch.int64, device=dev, pin_memory=not queries.is_cuda and torch.cuda.is_available())
    if out_dist is None:
        out_dist = torch.empty((Q, k), dtype=torch.float32, device=dev, pin_memory=not queries.is_cuda and torch.cuda.is_available())
    st = N.Stats()
    stp = ctypes.byref(st) if return_stats else None
    if thr_in is None:
        N.check(N.lib.knn_search_ex(_ptr(db), db.shape[0], _ptr(queries), Q, n, int(w), int(p), int(k),
                                    ctypes.byref(opt), _ptr(out_idx), _ptr(out_dist), stp, _stream()))
    else:
        thr_in = _f32(thr_in, "thr_in")
        if thr_in.shape != (Q,):
            raise ValueError("thr_in must be [Q]")
        N.check(N.lib.knn_search_bounded(_ptr(db), db.shape[0], _ptr(queries), Q, n, int(w), int(p), int(k),
                                         ctypes.byref(opt), _ptr(thr_in), _ptr(out_idx), _ptr(out_dist), stp,
                                         _stream()))
    if return_stats:
        return out_idx, out_dist, st.as_dict()
    return out_idx, out_dist


def knn_search_bounded(db: torch.Tensor, queries: torch.Tensor, w: int, p: int, k: int, thr_in: torch.Tensor,
                       **kw):
    """knn_search of one shard of a candidate-sharded database with every
    query's threshold lowered to thr_in (float32 [Q], power units, e.g. the
    minimum over the shards of knn_seed_thresholds); keyword arguments as in
    knn_search."""
    return knn_search(db, queries, w, p, k, thr_in=thr_in, **kw)


def knn_seed_thresholds(db: torch.Tensor, queries: torch.Tensor, w: int, p: int, k: int = 1, *,
                    mode: str = "improved", slack: float = 1e-6, seeds: int = 0, parts: int = 0,
                    dtw_path: int = 0, filter_path: int = 0, out: torch.Tensor | None = None) -> torch.Tensor:
    """Each query's k-th smallest seed DTW against this shard of a
    candidate-sharded database: float32 [Q] in the
    cascade's power units (DTW_p^p; DTW_inf for p = infinity), +inf where the
    shard has fewer than k seeds.  The minimum over the shards is a valid
    threshold for every shard's knn_search_bounded."""
    db, queries, opt = _knn_args(db, queries, mode, slack, seeds, parts, dtw_path, filter_path, 0)
    Q, n = queries.shape
    if out is None:
        out = torch.empty(Q, dtype=torch.float32, device=queries.device,
                          pin_memory=not queries.is_cuda and torch.cuda.is_available())
    N.check(N.lib.knn_seed_thresholds(_ptr(db), db.shape[0], _ptr(queries), Q, n, int(w), int(p), int(k),
                                      ctypes.byref(opt), _ptr(out), _stream()))
    return out


def knn_merge_topk(idx: torch.Tensor, dist: torch.Tensor, k: int):
    """The k smallest (distance, index) per query of R per-shard lists idx,
    dist [R, Q, k_in] (CUDA tensors; global indices below 2^31, -1 / +inf for
    empty entries): (idx int64 [Q, k], dist float32 [Q, k]), padded with
    -1 / +inf."""
    if not (idx.is_cuda and dist.is_cuda):
        raise ValueError("knn_merge_topk takes CUDA tensors")
    if idx.dim() != 3 or idx.shape != dist.shape:
        raise ValueError("idx and dist must both be [R, Q, k_in]")
    idx = idx.to(torch.int64).contiguous()
    dist = dist.to(torch.float32).contiguous()
    R, Q, kin = idx.shape
    oi = torch.empty((Q, k), dtype=torch.int64, device=idx.device)
    od = torch.empty((Q, k), dtype=torch.float32, device=idx.device)
    N.check(N.lib.knn_merge_topk(_ptr(idx), _ptr(dist), R, Q, kin, int(k), _ptr(oi), _ptr(od), _stream()))
    return oi, od


def _i32_host(v, Q: int, name: str) -> np.ndarray:
    a = np.asarray(v, dtype=np.int64)
    if a.ndim == 0:
        a = np.full(Q, int(a), dtype=np.int64)
    if a.shape != (Q,):
        raise ValueError("%s must be a scalar or have one entry per query" % name)
    return np.ascontiguousarray(a, dtype=np.int32)


class DtwIndex:
    """Length buckets resident on the device and batched k-NN search over
    queries of mixed length, band and k (the dtw_index_* calls).

    Every query gets the result knn_search gives it against the bucket of its
    length; grouping, concurrent streams, CUDA graphs and autotuning only
    change the speed.
    """

    def __init__(self, p: int, *, mode: str = "improved", slack: float = 1e-6, seeds: int = 0, parts: int = 0,
                 dtw_path: int = 0, filter_path: int = 0):
        if mode not in _MODES:
            raise ValueError("mode must be one of %s" % sorted(_MODES))
        opt = N.Options(_MODES[mode], float(slack), int(seeds), int(parts), int(dtw_path), int(filter_path))
        h = ctypes.c_void_p()
        N.check(N.lib.dtw_index_create(int(p), ctypes.byref(opt), ctypes.byref(h)))
        self._h = h
        self.p = int(p)
        self.lengths: list[int] = []

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            N.check(N.lib.dtw_index_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_bucket(self, db: torch.Tensor) -> None:
        """Adds the bucket of length n = db.shape[1] (db [N, n], host or CUDA; copied)."""
        db = _f32(db, "db")
        if db.dim() != 2:
            raise ValueError("db must be [N, n]")
        N.check(N.lib.dtw_index_add_bucket(self._h, _ptr(db), db.shape[0], db.shape[1]))
        self.lengths.append(int(db.shape[1]))

    def tune(self, sample: torch.Tensor, w: int, k: int) -> dict:
        """Times candidate parameters on sample [count, n] and keeps the fastest for (n, w, k)."""
        sample = _f32(sample, "sample")
        t = N.Tuning()
        N.check(N.lib.dtw_index_tune(self._h, _ptr(sample), sample.shape[0], sample.shape[1], int(w), int(k),
                                     ctypes.byref(t)))
        return t.as_dict()

    def get_tuning(self, n: int, w: int, k: int) -> dict:
        t = N.Tuning()
        N.check(N.lib.dtw_index_get_tuning(self._h, int(n), int(w), int(k), ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, n: int, w: int, k: int, *, parts: int, seeds: int, seg_len: int, dtw_path: int = 0,
                   filter_warps: int = 0) -> None:
        t = N.Tuning(int(parts), int(seeds), int(seg_len), -1.0, int(dtw_path), int(filter_warps))
        N.check(N.lib.dtw_index_set_tuning(self._h, int(n), int(w), int(k), ctypes.byref(t)))

    def info(self) -> dict:
        st = N.IndexStats()
        N.check(N.lib.dtw_index_info(self._h, ctypes.byref(st)))
        return st.as_dict()

    def search_flat(self, flat: torch.Tensor, lengths, w, k, *, k_stride: int | None = None, graph: bool = False,
                    autotune: bool = False, serial: bool = False, per_query: bool = False, persistent: bool = False,
                    out_idx: torch.Tensor | None = None, out_dist: torch.Tensor | None = None,
                    return_stats: bool = False):
        """Batched search over queries concatenated in `flat` (1-D float32, host or CUDA).

        lengths, w and k are per-query sequences (or scalars for w and k).
        Returns (idx int64 [Q, k_stride], dist float32 [Q, k_stride]) on the
        device of `flat`; entries past a query's k are -1 / +inf.
        """
        flat = _f32(flat, "flat").reshape(-1)
        lens = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64), dtype=np.int32)
        Q = lens.shape[0]
        ws = _i32_host(w, Q, "w")
        ks = _i32_host(k, Q, "k")
        if int(lens.astype(np.int64).sum()) != flat.numel():
            raise ValueError("sum of lengths (%d) must equal the number of values (%d)" % (int(lens.sum()), flat.numel()))
        ks_max = int(ks.max()) if Q else 1
        k_stride = ks_max if k_stride is None else int(k_stride)
        dev = flat.device
        pin = not flat.is_cuda and torch.cuda.is_available()
        if out_idx is None:
            out_idx = torch.empty((Q, k_stride), dtype=torch.int64, device=dev, pin_memory=pin)
        if out_dist is None:
            out_dist = torch.empty((Q, k_stride), dtype=torch.float32, device=dev, pin_memory=pin)
        flags = ((N.BATCH_GRAPH if graph else 0) | (N.BATCH_AUTOTUNE if autotune else 0) |
                 (N.BATCH_SERIAL if serial else 0) | (N.BATCH_PER_QUERY if per_query else 0) |
                 (N.BATCH_PERSISTENT if persistent else 0))
        st = N.Stats()
        N.check(N.lib.dtw_index_search(self._h, _ptr(flat) if flat.numel() else None, Q,
                                       lens.ctypes.data, ws.ctypes.data, ks.ctypes.data, k_stride, flags,
                                       _ptr(out_idx), _ptr(out_dist),
                                       ctypes.byref(st) if return_stats else None, _stream()))
        if return_stats:
            return out_idx, out_dist, st.as_dict()
        return out_idx, out_dist

    def search(self, queries, w, k, **kw):
        """Batched search over a list of 1-D query tensors of mixed length (see search_flat)."""
        qs = [_f32(q, "query").reshape(-1) for q in queries]
        if not qs:
            raise ValueError("no queries")
        lengths = [q.numel() for q in qs]
        return self.search_flat(torch.cat(qs), lengths, w, k, **kw)


def monotonic_ns() -> int:
    """The request server's clock (CLOCK_MONOTONIC), in nanoseconds."""
    return int(N.lib.dtw_monotonic_ns())


class DtwServer:
    """Continuous-batching request server over a DtwIndex (the dtw_server_* calls).

    submit() queues one query and returns a ticket; poll() returns finished
    requests with their neighbours and their arrival, admission and
    completion times.  The index must outlive the server and must not change
    while it runs.
    """

    def __init__(self, index: DtwIndex, *, slots: int = 4, max_batch: int = 512, slot_bytes: int = 0,
                 max_wait_us: int = 0, graph: bool = False, serial: bool = False, per_query: bool = False,
                 batch_timeout_ms: int = 0):
        flags = ((N.BATCH_GRAPH if graph else 0) | (N.BATCH_SERIAL if serial else 0) |
                 (N.BATCH_PER_QUERY if per_query else 0))
        cfg = N.ServerConfig(int(slots), int(max_batch), int(slot_bytes), int(max_wait_us), flags,
                             int(batch_timeout_ms))
        h = ctypes.c_void_p()
        N.check(N.lib.dtw_server_create(index._h, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._index = index  # keeps the index alive
        self._out: dict[int, tuple] = {}
        self._buf = (N.Completion * 4096)()

    def submit(self, query, w: int, k: int, arrival_ns: int = 0) -> int:
        """Queues one query (1-D float32, host); returns its ticket."""
        q = np.ascontiguousarray(np.asarray(query, dtype=np.float32).reshape(-1))
        oi = np.empty(int(k), np.int64)
        od = np.empty(int(k), np.float32)
        t = ctypes.c_uint64()
        N.check(N.lib.dtw_server_submit(self._h, q.ctypes.data, q.shape[0], int(w), int(k), oi.ctypes.data,
                                        od.ctypes.data, int(arrival_ns), ctypes.byref(t)))
        self._out[int(t.value)] = (oi, od)
        return int(t.value)

    def poll(self, max_items: int = 4096, wait_ms: int = 0) -> list[dict]:
        """Finished requests: dicts with ticket, status, k, arrival/admit/done ns, idx, dist."""
        cnt = ctypes.c_int32()
        m = min(int(max_items), len(self._buf))
        N.check(N.lib.dtw_server_poll(self._h, self._buf, m, ctypes.byref(cnt), int(wait_ms)))
        out = []
        for i in range(cnt.value):
            c = self._buf[i]
            oi, od = self._out.pop(int(c.ticket))
            out.append({"ticket": int(c.ticket), "status": int(c.status), "k": int(c.k),
                        "arrival_ns": int(c.arrival_ns), "admit_ns": int(c.admit_ns), "done_ns": int(c.done_ns),
                        "idx": oi, "dist": od})
        return out

    def info(self) -> dict:
        st = N.ServerStats()
        N.check(N.lib.dtw_server_info(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            N.check(N.lib.dtw_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
