"""Parity with the FP64 oracle at the sizes of the benchmark's workloads.

The other parity tests run small databases; these run the configurations
the benchmark times, where other code paths take over: long rows streamed
through the filter (n > 256), candidate segments of 1,024, the warp-per-pair
DTW for bands wider than 208 slots, the multi-length index with graphs and
autotuning, and the request server with a resident database of 100,000
series.  Every launch covers the whole workload; the oracle checks a sample
of its queries (the oracle's Algorithm 3 scan, which equals brute-force
k-NN, on all host cores).  Tolerances as in test_gpu_parity.py.
"""

import math
import os
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

REL = 1e-5
ABS = 1e-5
THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def api():
    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import api as a

    return a


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def check_rows(db, queries, w, p, k, gidx, gdist):
    """The GPU's top-k rows of `queries` against the oracle's: distances
    within REL, indices equal except at near-ties fp32 cannot order."""
    gidx = np.asarray(gidx)
    gdist = np.asarray(gdist, dtype=np.float64)
    ri, rd, _ = oracle.knn_cascade(db, queries, w, p, k, mode=1, threads=THREADS)
    for q in range(queries.shape[0]):
        for r in range(k):
            oi, od = int(ri[q, r]), float(rd[q, r])
            gi, gd = int(gidx[q, r]), float(gdist[q, r])
            if oi < 0:
                assert gi == -1 and math.isinf(gd), (q, r, gi, gd)
                continue
            assert abs(gd - od) <= REL * od + ABS, (q, r, gd, od)
            if gi != oi:
                d_gi = oracle.dtw(db[gi], queries[q], w, p)
                assert abs(d_gi - od) <= REL * od + ABS, (q, r, gi, oi, d_gi, od)


def test_shape_like_full_size_wide_band(api):
    # 50,000 shape-like series of length 1,024, band 204 (20 %), 500 queries,
    # DTW_1, 1-NN: streamed filter rows and the warp-per-pair DTW
    db = synth.shapes(50_000, 1024, seed=2)
    qs = synth.shapes(500, 1024, seed=2, stream=synth.STREAM_QUERY)
    idx, dist = api.knn_search(cuda(db), cuda(qs), 204, 1, 1)
    sample = np.array([0, 1, 2, 3, 4, 250, 496, 497, 498, 499])
    check_rows(db, qs[sample], 204, 1, 1, idx.cpu().numpy()[sample], dist.cpu().numpy()[sample])


def test_random_walk_full_size_ten_neighbours(api):
    # 100,000 random walks of length 256, band 25, 1,000 queries, 10-NN
    db = synth.random_walks(100_000, 256, seed=2)
    qs = synth.random_walks(1000, 256, seed=2, stream=synth.STREAM_QUERY)
    for p in (1, 2):
        idx, dist = api.knn_search(cuda(db), cuda(qs), 25, p, 10)
        sample = np.array([0, 1, 500, 998, 999])
        check_rows(db, qs[sample], 25, p, 10, idx.cpu().numpy()[sample], dist.cpu().numpy()[sample])
        # at this size the main DTW stage runs in row phases; every query's
        # answer equals the one-launch thread path's bit for bit
        ti, td = api.knn_search(cuda(db), cuda(qs), 25, p, 10, dtw_path=1)
        assert torch.equal(idx, ti) and torch.equal(dist, td), p


def test_index_long_buckets_graph_autotune(api):
    # buckets of 20,000 random walks of lengths 1,448 and 2,048 (the longest
    # of the batched workload), w = floor(n / 10), DTW_2, k = 10, the batch
    # captured as a CUDA graph with autotuned parameters; equal to knn_search
    # per bucket bit for bit, and to the oracle on a sample
    p, k = 2, 10
    buckets = [1448, 2048]
    dbs = {n: synth.random_walks(20_000, n, seed=1000 + n) for n in buckets}
    lens = np.array([buckets[i % 2] for i in range(40)])
    qs = synth.mixed_queries(lens, seed=77)
    ws = lens // 10
    with api.DtwIndex(p) as ix:
        for n in buckets:
            ix.add_bucket(cuda(dbs[n]))
        flat = cuda(np.concatenate(qs))
        gi, gd = ix.search_flat(flat, lens, ws, k, graph=True, autotune=True)
        gi2, gd2 = ix.search_flat(flat, lens, ws, k, graph=True)
        assert torch.equal(gi, gi2) and torch.equal(gd, gd2)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    for n in buckets:
        pos = np.flatnonzero(lens == n)
        ri, rd = api.knn_search(cuda(dbs[n]), cuda(np.stack([qs[i] for i in pos])), n // 10, p, k)
        np.testing.assert_array_equal(gi[pos], ri.cpu().numpy())
        np.testing.assert_array_equal(gd[pos], rd.cpu().numpy())
        sample = pos[:3]
        check_rows(dbs[n], np.stack([qs[i] for i in sample]), n // 10, p, k, gi[sample], gd[sample])


def test_server_large_resident_database(api):
    # resident buckets of 100,000 random walks of length 1,024 and 50,000 of
    # length 256, 1-NN and 10-NN mixed, requests in bursts so that batches
    # overlap; each result equal to knn_search on the query alone, and to the
    # oracle on a sample
    p = 1
    sizes = {256: 50_000, 1024: 100_000}
    dbs = {n: synth.random_walks(N, n, seed=3000 + n) for n, N in sizes.items()}
    g = np.random.default_rng(31)
    lens = g.choice(sorted(sizes), size=48)
    ks = g.choice([1, 10], size=48)
    qs = synth.mixed_queries(lens, seed=32)
    with api.DtwIndex(p) as ix:
        for n in sorted(sizes):
            ix.add_bucket(cuda(dbs[n]))
        with api.DtwServer(ix, slots=4, max_batch=16, slot_bytes=2 << 30) as srv:
            tickets = []
            for i in range(len(lens)):
                tickets.append(srv.submit(qs[i], int(lens[i]) // 10, int(ks[i])))
                if i % 8 == 7:
                    time.sleep(0.003)
            got = {}
            t_end = time.time() + 300
            while len(got) < len(tickets) and time.time() < t_end:
                for c in srv.poll(wait_ms=50):
                    got[c["ticket"]] = c
            info = srv.info()
    assert len(got) == len(tickets)
    assert info["max_batch_seen"] > 1, info
    res = [got[t] for t in tickets]
    for i, c in enumerate(res):
        assert c["status"] == 0
        n, k = int(lens[i]), int(ks[i])
        ri, rd = api.knn_search(cuda(dbs[n]), cuda(qs[i][None, :]), n // 10, p, k)
        np.testing.assert_array_equal(c["idx"], ri.cpu().numpy()[0])
        np.testing.assert_array_equal(c["dist"], rd.cpu().numpy()[0])
    for n in sorted(sizes):
        sel = [i for i in range(len(lens)) if lens[i] == n][:4]
        for i in sel:
            k = int(ks[i])
            check_rows(dbs[n], qs[i][None, :], n // 10, p, k, res[i]["idx"][None, :k], res[i]["dist"][None, :k])
