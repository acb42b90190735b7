"""Continuous-batching request server (dtw_server_*) through the C ABI.

Requests of mixed length (length buckets 64, 128, 256), band w = floor(n/10)
and k in {1, 10} are served alone (one request in flight at a time) and in a
mix (bursts of arrivals, several batches on the device at once).  Each
request's result must be the same in both cases and equal to knn_search on
that query alone (same indices, same fp32 distances), and on a subset the
oracle's neighbours within the parity tolerance.
"""

import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

REL = 1e-5
ABS = 1e-5
P = 1
BUCKETS = [64, 128, 256]
NB = 1500


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
    return {n: synth.random_walks(NB, n, seed=700 + n) for n in BUCKETS}


@pytest.fixture(scope="module")
def index(api, dbs):
    ix = api.DtwIndex(P)
    for n in BUCKETS:
        ix.add_bucket(cuda(dbs[n]))
    yield ix
    ix.close()


def make_requests(seed, count):
    g = np.random.default_rng(seed)
    lens = g.choice(BUCKETS, size=count)
    ks = g.choice([1, 10], size=count)
    qs = synth.mixed_queries(lens, seed=seed)
    return [(qs[i], int(lens[i]) // 10, int(ks[i])) for i in range(count)]


def collect(srv, tickets, timeout_s=60.0):
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < len(tickets) and time.time() < t_end:
        for c in srv.poll(wait_ms=50):
            got[c["ticket"]] = c
    assert len(got) == len(tickets), "requests did not complete"
    return [got[t] for t in tickets]


@pytest.fixture(scope="module")
def requests():
    return make_requests(seed=21, count=150)


@pytest.fixture(scope="module")
def alone(api, index, requests):
    out = []
    with api.DtwServer(index, slots=1, max_batch=1) as srv:
        for q, w, k in requests:
            t = srv.submit(q, w, k)
            out.append(collect(srv, [t])[0])
    return out


def test_alone_equals_knn_search(api, dbs, requests, alone):
    for (q, w, k), c in zip(requests, alone):
        assert c["status"] == 0
        gi, gd = api.knn_search(cuda(dbs[q.shape[0]]), cuda(q[None, :]), w, P, k)
        np.testing.assert_array_equal(c["idx"], gi.cpu().numpy()[0])
        np.testing.assert_array_equal(c["dist"], gd.cpu().numpy()[0])


def test_results_in_the_mix_equal_results_alone(api, index, requests, alone):
    with api.DtwServer(index, slots=4, max_batch=32) as srv:
        tickets = []
        g = np.random.default_rng(5)
        for i, (q, w, k) in enumerate(requests):
            tickets.append(srv.submit(q, w, k))
            if g.random() < 0.1:
                time.sleep(0.002)  # bursts separated by short gaps
        mixed = collect(srv, tickets)
        info = srv.info()
    for a, b in zip(alone, mixed):
        assert b["status"] == 0
        np.testing.assert_array_equal(a["idx"], b["idx"])
        np.testing.assert_array_equal(a["dist"], b["dist"])
        assert b["arrival_ns"] <= b["admit_ns"] <= b["done_ns"]
    assert info["completed"] == len(requests) and info["failed"] == 0
    # requests were batched, and batches overlapped on the device
    assert info["max_batch_seen"] > 1, info
    assert info["max_inflight_batches"] >= 2, info
    assert info["batches"] < len(requests), info


def test_served_results_match_the_oracle(dbs, requests, alone):
    for i in range(0, len(requests), 10):
        q, w, k = requests[i]
        oi, od = oracle.knn_bruteforce(dbs[q.shape[0]], q[None, :], w, P, k, threads=8)
        gd = alone[i]["dist"].astype(np.float64)
        for r in range(k):
            assert abs(gd[r] - od[0, r]) <= REL * od[0, r] + ABS, (i, r)
            if alone[i]["idx"][r] != oi[0, r]:
                d_g = oracle.dtw(dbs[q.shape[0]][alone[i]["idx"][r]], q, w, P)
                assert abs(d_g - od[0, r]) <= REL * od[0, r] + ABS, (i, r)


def test_memory_admission_bounds_the_batch(api, index, requests, alone):
    # a 2 MiB arena holds a few dozen of these queries' buffers (about 50 KB each)
    with api.DtwServer(index, slots=2, max_batch=64, slot_bytes=2 << 20) as srv:
        tickets = [srv.submit(q, w, k) for q, w, k in requests]
        res = collect(srv, tickets)
        info = srv.info()
    for a, b in zip(alone, res):
        np.testing.assert_array_equal(a["idx"], b["idx"])
        np.testing.assert_array_equal(a["dist"], b["dist"])
    assert info["max_batch_seen"] < 64, info
    # a slot too small for even one query rejects it at submission
    with api.DtwServer(index, slots=1, max_batch=4, slot_bytes=4096) as srv:
        with pytest.raises(api.DtwError) as e:
            srv.submit(requests[0][0], requests[0][1], requests[0][2])
        assert e.value.status == 3  # DTW_ERR_OOM


def test_query_without_bucket_is_rejected(api, index):
    with api.DtwServer(index, slots=1, max_batch=4) as srv:
        with pytest.raises(api.DtwError) as e:
            srv.submit(np.zeros(100, np.float32), 10, 1)
        assert e.value.status == 5  # DTW_ERR_NO_BUCKET


def test_poisoned_request_is_rejected_at_admission(api, index, requests):
    q = requests[0][0].copy()
    q[5] = np.nan
    with api.DtwServer(index, slots=1, max_batch=4) as srv:
        with pytest.raises(api.DtwError) as e:
            srv.submit(q, requests[0][1], requests[0][2])
        assert e.value.status == 1  # DTW_ERR_INVALID_ARG
        q[5] = np.inf
        with pytest.raises(api.DtwError):
            srv.submit(q, requests[0][1], requests[0][2])
        # the server keeps serving
        t = srv.submit(requests[1][0], requests[1][1], requests[1][2])
        assert collect(srv, [t])[0]["status"] == 0


def test_watchdog_completes_overdue_batches_with_timeout(api, index, requests, alone):
    # one query per launch makes a batch of many requests take milliseconds;
    # with a 1 ms deadline the watchdog completes them with DTW_ERR_TIMEOUT
    # (their buffers untouched) while the device finishes, and the slot is
    # reused once it has
    with api.DtwServer(index, slots=1, max_batch=64, per_query=True, batch_timeout_ms=1) as srv:
        tickets = [srv.submit(q, w, k) for q, w, k in requests[:80]]
        res = collect(srv, tickets)
        info = srv.info()
    timed = [r for r in res if r["status"] == 4]  # DTW_ERR_TIMEOUT
    assert len(timed) >= 1 and info["timed_out"] == len(timed), info
    assert info["completed"] == len(tickets)
    for a, b in zip(alone, res):
        if b["status"] == 0:
            np.testing.assert_array_equal(a["idx"], b["idx"])
            np.testing.assert_array_equal(a["dist"], b["dist"])
