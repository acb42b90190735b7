"""Multi-GPU decompositions of the retrieval (one process per GPU).

The candidates of a k-NN query are independent (Sec. 7-8 problem
statement), so the search shards two ways:

- by query: every rank holds the whole database and searches its own queries;
  nothing is exchanged on the data path (weak scaling);
- by candidate: every rank holds a contiguous candidate range and searches
  every query in it; the per-rank top-k lists, with global indices, are
  gathered and merged by (distance, index).  The merge is the exact top-k of
  the whole database: a true neighbour is among the k best of its own range,
  and ordering by (distance, index) keeps the lower index first on ties, as
  the single-GPU search does.

  Before the bounds, the ranks exchange thresholds: each rank's seeds give
  every query a threshold at least that rank's k-th smallest DTW, and their
  minimum (an all-reduce) is at least the k-th smallest over the whole
  database, so every rank prunes with the tightest one and still keeps every
  true neighbour.

The collectives are torch.distributed's all_reduce and all_gather over the
caller's process group (NCCL between GPUs, gloo on CPU).
"""

from __future__ import annotations

import numpy as np


def query_range(Q: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [start, stop) of the Q queries that rank searches."""
    base, extra = divmod(Q, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def candidate_range(N: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [start, stop) of the N candidates that rank holds."""
    return query_range(N, world, rank)


def merge_topk(idx: np.ndarray, dist: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Merges per-shard top-k lists idx, dist [R][Q][kk] (global indices, -1 /
    +inf for empty entries) into the k best per query by (distance, index)."""
    idx = np.asarray(idx, dtype=np.int64)
    dist = np.asarray(dist, dtype=np.float32)
    R, Q, kk = idx.shape
    ci = np.transpose(idx, (1, 0, 2)).reshape(Q, R * kk)
    cd = np.transpose(dist, (1, 0, 2)).reshape(Q, R * kk)
    empty = ci < 0
    key_i = np.where(empty, np.iinfo(np.int64).max, ci)
    key_d = np.where(empty, np.inf, cd)
    out_i = np.full((Q, k), -1, np.int64)
    out_d = np.full((Q, k), np.inf, np.float32)
    for q in range(Q):
        order = np.lexsort((key_i[q], key_d[q]))[:k]
        keep = ~empty[q][order]
        m = int(keep.sum())
        out_i[q, :m] = ci[q][order][keep]
        out_d[q, :m] = cd[q][order][keep]
    return out_i, out_d


def exchange_thresholds(thr, group=None):
    """Every rank's per-query thresholds [Q] (torch tensor) replaced, in
    place, by their minimum over the ranks of the group; returned."""
    import torch.distributed as dist

    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(thr, op=dist.ReduceOp.MIN, group=group)
    return thr


def gather_merge(local_idx, local_dist, k: int, group=None):
    """All-gathers every rank's [Q][k] top-k (torch tensors with global indices)
    and returns the merged exact top-k on every rank (same device as input):
    on the GPU by the library's merge kernel, for host tensors (ranks
    without a GPU) by merge_topk above."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    gi = [torch.empty_like(local_idx) for _ in range(world)]
    gd = [torch.empty_like(local_dist) for _ in range(world)]
    if world > 1:
        dist.all_gather(gi, local_idx.contiguous(), group=group)
        dist.all_gather(gd, local_dist.contiguous(), group=group)
    else:
        gi, gd = [local_idx.contiguous()], [local_dist.contiguous()]
    if local_idx.is_cuda:
        from . import api

        return api.knn_merge_topk(torch.stack(gi), torch.stack(gd), k)
    idx = np.stack([t.numpy() for t in gi])
    dd = np.stack([t.numpy() for t in gd])
    mi, md = merge_topk(idx, dd, k)
    return torch.from_numpy(mi), torch.from_numpy(md)


def sharded_knn_search(db_shard, offset: int, queries, w: int, p: int, k: int, group=None, exchange: bool = True,
                       **kw):
    """knn_search over this rank's candidate range (db_shard = rows
    [offset, offset + len)), then the exact global top-k by gather_merge.
    With exchange, the ranks first share their seeds' thresholds
    (knn_seed_thresholds, exchange_thresholds) and every rank searches with
    the tightest (knn_search_bounded)."""
    import torch

    from . import api

    if exchange:
        skw = {key: v for key, v in kw.items() if key in ("mode", "slack", "seeds", "parts", "dtw_path", "filter_path")}
        thr = exchange_thresholds(api.knn_seed_thresholds(db_shard, queries, w, p, k, **skw), group)
        idx, dd = api.knn_search_bounded(db_shard, queries, w, p, k, thr, **kw)
    else:
        idx, dd = api.knn_search(db_shard, queries, w, p, k, **kw)
    idx = torch.where(idx >= 0, idx + int(offset), idx)
    return gather_merge(idx, dd, k, group=group)
