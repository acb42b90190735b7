"""Candidate sharding on one GPU: the database split into shards searched one
after the other (no ranks wait on one another), with the thresholds of the
shards' seeds exchanged (their minimum) before the bounds, and the shards'
lists merged by the library's merge kernel.  The merged result must be the
single search's over the whole database (and the oracle's on a sample), and
the exchanged threshold must bound the true k-th distance."""


import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import api as a

    return a


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _sharded(api, db, qs, w, p, k, cuts, exchange=True):
    shards = list(zip([0] + cuts, cuts + [db.shape[0]]))
    thr = None
    if exchange:
        ts = [api.knn_seed_thresholds(cuda(db[a:b]), cuda(qs), w, p, k) for a, b in shards]
        thr = torch.stack(ts).min(dim=0).values
    lists_i, lists_d, stats = [], [], []
    for a, b in shards:
        i, d, st = (api.knn_search_bounded(cuda(db[a:b]), cuda(qs), w, p, k, thr, return_stats=True) if exchange
                     else api.knn_search(cuda(db[a:b]), cuda(qs), w, p, k, return_stats=True))
        lists_i.append(torch.where(i >= 0, i + a, i))
        lists_d.append(d)
        stats.append(st)
    mi, md = api.knn_merge_topk(torch.stack(lists_i), torch.stack(lists_d), k)
    return mi, md, thr, stats


def _same_topk(mi, md, ri, rd):
    # distances bit-equal; an index may differ only between equal distances
    assert torch.equal(md, rd)
    mi, ri, md = mi.cpu().numpy(), ri.cpu().numpy(), md.cpu().numpy()
    for q in range(mi.shape[0]):
        for r in range(mi.shape[1]):
            if mi[q, r] != ri[q, r]:
                assert np.sum(md[q] == md[q, r]) > 1, (q, r)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("k", [1, 5])
def test_two_and_three_shards_equal_the_whole_search(api, p, k):
    db = synth.random_walks(9_000, 128, seed=70 + p)
    qs = synth.random_walks(24, 128, seed=71 + p, stream=synth.STREAM_QUERY)
    w = 12
    ri, rd = api.knn_search(cuda(db), cuda(qs), w, p, k)
    for cuts in ([4_100], [2_000, 6_500]):
        mi, md, thr, _ = _sharded(api, db, qs, w, p, k, cuts)
        _same_topk(mi, md, ri, rd)
        # the exchanged threshold (power units) is at least the true k-th
        kth = rd[:, -1].double() ** p
        assert bool((thr.double() >= kth * (1 - 1e-6)).all())
    oi, od, _ = oracle.knn_cascade(db, qs[:5], w, p, k, mode=1, threads=8)
    mi, md, _, _ = _sharded(api, db, qs[:5], w, p, k, [4_100])
    for q in range(5):
        for r in range(k):
            assert abs(float(md[q, r]) - od[q, r]) <= 1e-5 * od[q, r] + 1e-5


def test_exchange_prunes_at_least_as_much(api):
    db = synth.random_walks(12_000, 256, seed=74)
    qs = synth.random_walks(30, 256, seed=75, stream=synth.STREAM_QUERY)
    w, p, k = 25, 1, 3
    _, _, _, with_x = _sharded(api, db, qs, w, p, k, [3_000, 6_000, 9_000])
    mi, md, _, without = _sharded(api, db, qs, w, p, k, [3_000, 6_000, 9_000], exchange=False)
    ri, rd = api.knn_search(cuda(db), cuda(qs), w, p, k)
    _same_topk(mi, md, ri, rd)
    assert sum(s["dtw_computed"] for s in with_x) <= sum(s["dtw_computed"] for s in without)


def test_merge_kernel_matches_the_host_merge(api):
    from paper_0811_3301_gb300 import shard

    rng = np.random.default_rng(76)
    R, Q, kin, k = 3, 40, 7, 9
    dist = rng.integers(0, 12, size=(R, Q, kin)).astype(np.float32) / 4  # many ties
    idx = rng.permutation(R * Q * kin).reshape(R, Q, kin).astype(np.int64) % 500
    empty = rng.random((R, Q, kin)) < 0.2
    idx[empty] = -1
    dist[empty] = np.inf
    hi, hd = shard.merge_topk(idx, dist, k)
    gi, gd = api.knn_merge_topk(torch.from_numpy(idx).cuda(), torch.from_numpy(dist).cuda(), k)
    np.testing.assert_array_equal(gi.cpu().numpy(), hi)
    np.testing.assert_array_equal(gd.cpu().numpy(), hd)


def test_thresholds_of_an_empty_shard_and_host_buffers(api):
    qs = synth.random_walks(6, 64, seed=77, stream=synth.STREAM_QUERY)
    t = api.knn_seed_thresholds(cuda(np.zeros((0, 64))), cuda(qs), 6, 2, 2)
    assert bool(torch.isinf(t).all())
    db = synth.random_walks(3_000, 64, seed=78)
    td = api.knn_seed_thresholds(cuda(db), cuda(qs), 6, 2, 2)
    th = api.knn_seed_thresholds(torch.from_numpy(db), torch.from_numpy(qs), 6, 2, 2)  # host in, host out
    assert not th.is_cuda and torch.equal(th, td.cpu())
    # a host thr_in, NaN and negative entries ignored (the query's own threshold stays)
    tin = th.clone()
    tin[0] = float("nan")
    tin[1] = -1.0
    ri, rd = api.knn_search(cuda(db), cuda(qs), 6, 2, 2)
    bi, bd = api.knn_search_bounded(cuda(db), cuda(qs), 6, 2, 2, tin)
    assert torch.equal(bi, ri) and torch.equal(bd, rd)
    # a threshold below every distance leaves nothing to list
    zi, zd = api.knn_search_bounded(cuda(db), cuda(qs), 6, 2, 2, torch.zeros(6).cuda())
    assert bool((zi == -1).all()) and bool(torch.isinf(zd).all())


def test_sharded_search_in_one_process(api):
    from paper_0811_3301_gb300 import shard

    db = synth.random_walks(5_000, 96, seed=79)
    qs = synth.random_walks(12, 96, seed=80, stream=synth.STREAM_QUERY)
    ri, rd = api.knn_search(cuda(db), cuda(qs), 9, 2, 4)
    for exchange in (True, False):
        mi, md = shard.sharded_knn_search(cuda(db), 0, cuda(qs), 9, 2, 4, exchange=exchange)
        _same_topk(mi, md, ri, rd)
