"""Multi-GPU decompositions, tested on CPU: two gloo ranks shard the database
by candidate range, search their range (here with the oracle, the CPU
stand-in for each rank's GPU search) and merge the gathered top-k lists with
the package's merge; the result must be the oracle's top-k over the whole
database.  Query sharding must cover every query exactly once."""

import os
import tempfile

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")


def test_ranges_partition_the_work():
    from paper_0811_3301_gb300 import shard

    for total in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            parts = [shard.query_range(total, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == total
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
            assert shard.candidate_range(total, world, 1 % world) == parts[1 % world]


def test_merge_orders_by_distance_then_index_and_pads():
    from paper_0811_3301_gb300 import shard

    # two shards, two queries, k = 3; ties across shards go to the lower index
    idx = np.array([[[4, 2, -1], [0, 1, 3]], [[9, 7, -1], [12, -1, -1]]], np.int64)
    dist = np.array([[[1.0, 2.0, np.inf], [5.0, 5.0, 6.0]], [[1.0, 0.5, np.inf], [4.0, np.inf, np.inf]]], np.float32)
    mi, md = shard.merge_topk(idx, dist, 3)
    assert mi.tolist() == [[7, 4, 9], [12, 0, 1]]
    assert md.tolist() == [[0.5, 1.0, 1.0], [4.0, 5.0, 5.0]]
    # fewer candidates than k: the tail is -1 / +inf
    mi, md = shard.merge_topk(idx[:, :1, :2], dist[:, :1, :2], 6)
    assert mi.tolist() == [[7, 4, 9, 2, -1, -1]]
    assert np.isinf(md[0, 4:]).all()


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    from paper_0811_3301_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        db = synth.random_walks(601, 48, seed=44)
        qs = synth.random_walks(5, 48, seed=44, stream=synth.STREAM_QUERY)
        w, p, k = 4, 1, 6
        a, b = shard.candidate_range(db.shape[0], world, rank)
        li, ld = oracle.knn_bruteforce(db[a:b], qs, w, p, k)
        li = np.where(li >= 0, li + a, li)
        mi, md = shard.gather_merge(torch.from_numpy(li), torch.from_numpy(ld.astype(np.float32)), k)
        if rank == 0:
            np.savez(out_path, idx=mi.numpy(), dist=md.numpy())
    finally:
        dist.destroy_process_group()


def test_candidate_sharding_over_two_gloo_ranks_equals_the_full_search():
    import torch.multiprocessing as mp

    port = 29500 + (os.getpid() % 2000)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "merged.npz")
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        r = np.load(out)
        mi, md = r["idx"], r["dist"]
    db = synth.random_walks(601, 48, seed=44)
    qs = synth.random_walks(5, 48, seed=44, stream=synth.STREAM_QUERY)
    ri, rd = oracle.knn_bruteforce(db, qs, 4, 1, 6)
    np.testing.assert_array_equal(mi, ri)
    np.testing.assert_allclose(md, rd.astype(np.float32), rtol=0, atol=0)


def _rank_exchange_main(rank, world, port, out_path):
    # each rank: a stand-in for its seeds' threshold (the k-th smallest DTW
    # of its first 20 candidates, by the oracle), the all-reduce minimum over
    # the ranks, then its range's top-k restricted to that threshold (what
    # the bounded GPU search lists), and the merge
    import torch.distributed as dist

    from paper_0811_3301_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        db = synth.random_walks(601, 48, seed=45)
        qs = synth.random_walks(5, 48, seed=45, stream=synth.STREAM_QUERY)
        w, p, k = 4, 2, 6
        a, b = shard.candidate_range(db.shape[0], world, rank)
        seeds = np.array([[oracle.dtw(db[a + c], q, w, p) for c in range(20)] for q in qs])
        kth = np.sort(seeds, axis=1)[:, k - 1]
        t32 = kth.astype(np.float32)
        t32 = np.where(t32.astype(np.float64) < kth, np.nextafter(t32, np.float32(np.inf)), t32)  # round up
        thr = torch.from_numpy(t32)
        mine = thr.clone()
        shard.exchange_thresholds(thr)
        li, ld = oracle.knn_bruteforce(db[a:b], qs, w, p, k)
        cut = ld > thr.numpy()[:, None].astype(np.float64)
        li = np.where(cut | (li < 0), -1, li + a)
        ld = np.where(cut, np.inf, ld)
        mi, md = shard.gather_merge(torch.from_numpy(li), torch.from_numpy(ld.astype(np.float32)), k)
        if rank == 0:
            np.savez(out_path, idx=mi.numpy(), dist=md.numpy(), thr=thr.numpy(), mine=mine.numpy())
    finally:
        dist.destroy_process_group()


def test_threshold_exchange_over_two_gloo_ranks_keeps_the_exact_result():
    import torch.multiprocessing as mp

    port = 31500 + (os.getpid() % 2000)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "merged.npz")
        mp.spawn(_rank_exchange_main, args=(2, port, out), nprocs=2, join=True)
        r = np.load(out)
    db = synth.random_walks(601, 48, seed=45)
    qs = synth.random_walks(5, 48, seed=45, stream=synth.STREAM_QUERY)
    ri, rd = oracle.knn_bruteforce(db, qs, 4, 2, 6)
    np.testing.assert_array_equal(r["idx"], ri)
    np.testing.assert_allclose(r["dist"], rd.astype(np.float32), rtol=0, atol=0)
    # the exchanged threshold is the smaller one, and bounds the true k-th
    assert (r["thr"] <= r["mine"]).all()
    assert (r["thr"].astype(np.float64) >= rd[:, -1].astype(np.float32)).all()
