"""Batched multi-length search (dtw_index_*) through the C ABI.

A batch mixes query lengths (snapped to the length buckets), bands
w = floor(n/10) and k in {1, 5}.  Every query must get exactly what
knn_search gives it against its bucket (same indices, same fp32 distances:
the same kernels compute the same pair distances), whatever the execution
flags (concurrent groups, serial groups, one query per launch, CUDA graph
capture and replay, autotuned parameters); and, on a subset, the oracle's
neighbours within the tolerance of the other parity tests.
"""

import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

REL = 1e-5
ABS = 1e-5
P = 2
BUCKETS = [64, 91, 128, 181, 256]
NB = 1200


@pytest.fixture(scope="module")
def api():
    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import api as a

    return a


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def dbs():
    return {n: synth.random_walks(NB, n, seed=400 + n) for n in BUCKETS}


@pytest.fixture(scope="module")
def index(api, dbs):
    ix = api.DtwIndex(P)
    for n in BUCKETS:
        ix.add_bucket(cuda(dbs[n]))
    yield ix
    ix.close()


def make_batch(seed, Q):
    lens = synth.snap_to_buckets(synth.log_uniform_lengths(Q, 64, 256, seed=seed), BUCKETS)
    qs = synth.mixed_queries(lens, seed=seed)
    ws = lens // 10
    ks = np.where(np.arange(Q) % 3 == 0, 5, 1)
    return lens, qs, ws, ks


def flat_of(qs):
    return np.concatenate(qs).astype(np.float32)


def per_group_reference(api, dbs, lens, qs, ws, ks, k_stride):
    """knn_search on each (n, w, k) group; rows scattered back to batch order."""
    Q = len(lens)
    idx = np.full((Q, k_stride), -1, np.int64)
    dist = np.full((Q, k_stride), np.inf, np.float32)
    keys = sorted({(int(lens[i]), int(ws[i]), int(ks[i])) for i in range(Q)})
    for n, w, k in keys:
        pos = [i for i in range(Q) if (lens[i], ws[i], ks[i]) == (n, w, k)]
        qg = cuda(np.stack([qs[i] for i in pos]))
        gi, gd = api.knn_search(cuda(dbs[n]), qg, w, P, k)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        for r, i in enumerate(pos):
            idx[i, :k] = gi[r]
            dist[i, :k] = gd[r]
    return idx, dist


@pytest.fixture(scope="module")
def batch():
    return make_batch(seed=11, Q=90)


@pytest.fixture(scope="module")
def reference(api, dbs, batch):
    lens, qs, ws, ks = batch
    return per_group_reference(api, dbs, lens, qs, ws, ks, 5)


@pytest.mark.parametrize("mode", ["concurrent", "serial", "per_query", "graph", "persistent", "persistent_graph"])
def test_batched_equals_knn_search_per_group(api, index, batch, reference, mode):
    lens, qs, ws, ks = batch
    kw = {"serial": mode == "serial", "per_query": mode == "per_query", "graph": mode in ("graph", "persistent_graph"),
          "persistent": mode.startswith("persistent")}
    gi, gd = index.search_flat(cuda(flat_of(qs)), lens, ws, ks, **kw)
    ri, rd = reference
    np.testing.assert_array_equal(gi.cpu().numpy(), ri)
    np.testing.assert_array_equal(gd.cpu().numpy(), rd)


@pytest.mark.parametrize("persistent", [False, True])
def test_batched_matches_oracle_on_a_subset(index, dbs, batch, persistent):
    lens, qs, ws, ks = batch
    gi, gd = index.search_flat(cuda(flat_of(qs)), lens, ws, ks, persistent=persistent)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy().astype(np.float64)
    for i in range(0, len(lens), 6):  # 15 queries across all buckets
        n, w, k = int(lens[i]), int(ws[i]), int(ks[i])
        oi, od = oracle.knn_bruteforce(dbs[n], qs[i][None, :], w, P, k, threads=8)
        for r in range(k):
            assert abs(gd[i, r] - od[0, r]) <= REL * od[0, r] + ABS, (i, r, gd[i, r], od[0, r])
            if gi[i, r] != oi[0, r]:
                d_g = oracle.dtw(dbs[n][gi[i, r]], qs[i], w, P)
                assert abs(d_g - od[0, r]) <= REL * od[0, r] + ABS, (i, r)
        assert np.all(gi[i, k:] == -1) and np.all(np.isinf(gd[i, k:]))


def test_graph_replay_with_new_values_same_shapes(api, index, dbs, batch):
    lens, qs, ws, ks = batch
    qs2 = synth.mixed_queries(lens, seed=12)  # new values, same lengths
    ref_i, ref_d = per_group_reference(api, dbs, lens, qs2, ws, ks, 5)
    before = index.info()
    gi, gd = index.search_flat(cuda(flat_of(qs2)), lens, ws, ks, graph=True)
    gi2, gd2 = index.search_flat(cuda(flat_of(qs2)), lens, ws, ks, graph=True)
    after = index.info()
    assert after["graph_replays"] >= before["graph_replays"] + 2
    assert after["graph_captures"] <= before["graph_captures"] + 1
    for a, b in ((gi, gi2), (gd, gd2)):
        assert torch.equal(a, b)
    np.testing.assert_array_equal(gi.cpu().numpy(), ref_i)
    np.testing.assert_array_equal(gd.cpu().numpy(), ref_d)


def test_autotune_changes_speed_not_results(api, dbs, batch, reference):
    lens, qs, ws, ks = batch
    with api.DtwIndex(P) as ix:
        for n in BUCKETS:
            ix.add_bucket(cuda(dbs[n]))
        gi, gd = ix.search_flat(cuda(flat_of(qs)), lens, ws, ks, autotune=True)
        np.testing.assert_array_equal(gi.cpu().numpy(), reference[0])
        np.testing.assert_array_equal(gd.cpu().numpy(), reference[1])
        for n in BUCKETS:
            t = ix.get_tuning(n, n // 10, 1)
            assert t["ms"] > 0 and t["seg_len"] in (0, 512, 1024, 2048, 4096)
            assert t["parts"] == -1 or 1 <= t["parts"] <= n
        # explicit tuning: every parameter set gives the same answer
        n = 128
        sel = np.flatnonzero(lens == n)
        for parts, seeds, seg in ((-1, 4, 512), (n // 4, 32, 2048), (n // 16, 8, 1024)):
            for k in (1, 5):
                ix.set_tuning(n, n // 10, k, parts=parts, seeds=seeds, seg_len=seg)
            gi, gd = ix.search_flat(cuda(flat_of([qs[i] for i in sel])), lens[sel], ws[sel], ks[sel], k_stride=5)
            np.testing.assert_array_equal(gi.cpu().numpy(), reference[0][sel])
            np.testing.assert_array_equal(gd.cpu().numpy(), reference[1][sel])


def test_host_inputs_and_outputs_and_k_stride_padding(index, batch, reference):
    lens, qs, ws, ks = batch
    flat = torch.from_numpy(flat_of(qs))  # host
    gi, gd = index.search_flat(flat, lens, ws, ks, k_stride=8)
    assert not gi.is_cuda and gi.shape == (len(lens), 8)
    np.testing.assert_array_equal(gi[:, :5].numpy(), reference[0])
    np.testing.assert_array_equal(gd[:, :5].numpy(), reference[1])
    assert np.all(gi[:, 5:].numpy() == -1) and np.all(np.isinf(gd[:, 5:].numpy()))


def test_stats_count_every_pair(index, batch):
    lens, qs, ws, ks = batch
    _, _, st = index.search_flat(cuda(flat_of(qs)), lens, ws, ks, return_stats=True)
    assert st["candidates"] == len(lens) * NB
    pruned = st["pruned_summary"] + st["pruned_keogh"] + st["pruned_improved"]
    assert st["seeds"] + pruned + st["dtw_computed"] == st["candidates"]


def test_query_without_bucket_fails_before_any_work(api, index):
    q = np.zeros(100, np.float32)
    with pytest.raises(api.DtwError) as e:
        index.search_flat(cuda(q), [100], 10, 1)
    assert e.value.status == 5  # DTW_ERR_NO_BUCKET


def test_bucket_smaller_than_k_pads_the_tail(api):
    db = synth.random_walks(3, 32, seed=9)
    q = synth.random_walks(2, 32, seed=9, stream=synth.STREAM_QUERY)
    with api.DtwIndex(1) as ix:
        ix.add_bucket(cuda(db))
        gi, gd = ix.search_flat(cuda(q.reshape(-1)), [32, 32], 3, 5)
    oi, od = oracle.knn_bruteforce(db, q, 3, 1, 5)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    np.testing.assert_array_equal(gi, oi)
    for a, b in zip(gd.ravel(), od.ravel()):
        assert (math.isinf(a) and math.isinf(b)) or abs(a - b) <= REL * b + ABS


def test_empty_batch(index):
    gi, gd = index.search_flat(cuda(np.zeros(0, np.float32)), np.zeros(0, np.int64), 1, 1)
    assert gi.shape == (0, 1)


def test_persistent_arm_tuned_and_replayed(api, dbs, batch, reference):
    # the persistent launch over every group's (query, chunk) items, with its
    # chunk length autotuned on the batch, captured as a graph and replayed
    # with new query values; stats count every pair once
    lens, qs, ws, ks = batch
    with api.DtwIndex(P) as ix:
        for n in BUCKETS:
            ix.add_bucket(cuda(dbs[n]))
        gi, gd = ix.search_flat(cuda(flat_of(qs)), lens, ws, ks, persistent=True, autotune=True, graph=True)
        np.testing.assert_array_equal(gi.cpu().numpy(), reference[0])
        np.testing.assert_array_equal(gd.cpu().numpy(), reference[1])
        qs2 = synth.mixed_queries(lens, seed=13)
        ref2 = per_group_reference(api, dbs, lens, qs2, ws, ks, 5)
        for _ in range(2):
            gi, gd = ix.search_flat(cuda(flat_of(qs2)), lens, ws, ks, persistent=True, graph=True)
            np.testing.assert_array_equal(gi.cpu().numpy(), ref2[0])
            np.testing.assert_array_equal(gd.cpu().numpy(), ref2[1])
        assert ix.info()["graph_replays"] >= 2
        _, _, st = ix.search_flat(cuda(flat_of(qs2)), lens, ws, ks, persistent=True, return_stats=True)
        pruned = st["pruned_summary"] + st["pruned_keogh"] + st["pruned_improved"]
        assert st["seeds"] + pruned + st["dtw_computed"] == st["candidates"] == len(lens) * NB


def test_persistent_arm_rejects_what_it_does_not_serve(api, index, batch):
    lens, qs, ws, ks = batch
    with pytest.raises(api.DtwError) as e:
        index.search_flat(cuda(flat_of(qs)), lens, ws, ks, persistent=True, serial=True)
    assert e.value.status == 1
    with api.DtwIndex(P) as ix:  # band 2 * 300 + 1 = 601 > 512
        ix.add_bucket(cuda(synth.random_walks(50, 400, seed=4)))
        q = synth.random_walks(1, 400, seed=3, stream=synth.STREAM_QUERY).reshape(-1)
        with pytest.raises(api.DtwError) as e:
            ix.search_flat(cuda(q), [400], 300, 1, persistent=True)
        assert e.value.status == 1
        ix.search_flat(cuda(q), [400], 255, 1, persistent=True)  # band 511 is served
