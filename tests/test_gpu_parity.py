"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: envelopes are compared bit for bit (min/max do not round).
Bounds and DTW distances are fp32 sums of up to 2n terms; they must match
the oracle within REL = 1e-5 relative (plus a tiny absolute floor for values
near zero).  Neighbour indices must equal the oracle's exactly, except where
the oracle's own distances of the two candidates differ by less than REL
(a near-tie that fp32 cannot order); there the GPU's choice must still be a
candidate whose oracle distance equals the reported one within REL.
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


@pytest.fixture(scope="module")
def api():
    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import api as a

    return a


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def close(gpu, ref, rel=REL, abs_=ABS):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    both_inf = np.isinf(gpu) & np.isinf(ref)
    ok = both_inf | (np.abs(gpu - ref) <= rel * np.abs(ref) + abs_)
    return ok


def assert_knn(db, queries, w, p, k, gidx, gdist, ref_idx, ref_dist):
    gidx = gidx.cpu().numpy()
    gdist = gdist.cpu().numpy().astype(np.float64)
    Q = queries.shape[0]
    for q in range(Q):
        for r in range(k):
            oi, od = int(ref_idx[q, r]), float(ref_dist[q, r])
            gi, gd = int(gidx[q, r]), float(gdist[q, r])
            if oi < 0:
                assert gi == -1 and math.isinf(gd), (q, r, gi, gd)
                continue
            assert close(gd, od), (q, r, gd, od)
            if gi != oi:
                # accepted only as a near-tie: the oracle's distance of the GPU's
                # candidate equals the rank-r distance within REL
                d_gi = oracle.dtw(db[gi], queries[q], w, p)
                assert abs(d_gi - od) <= REL * od + ABS, (q, r, gi, oi, d_gi, od)


# ---------------------------------------------------------------------------
# envelope
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 7, 64, 129, 256, 1000, 2048, 4096])
def test_envelope_bit_exact(api, n):
    rng = np.random.default_rng(n)
    Y = np.concatenate([synth.random_walks(3, n, seed=n),
                        rng.integers(-2, 3, size=(2, n)).astype(np.float32)])  # ties
    for w in sorted({0, 1, 3, n // 10, n // 2, n - 1, n, n + 5}):
        U, L = api.dtw_envelope(cuda(Y), w)
        U, L = U.cpu().numpy(), L.cpu().numpy()
        for r in range(Y.shape[0]):
            Ur, Lr = oracle.envelope(Y[r], w)
            assert np.array_equal(U[r].astype(np.float64), Ur), (n, w, r)
            assert np.array_equal(L[r].astype(np.float64), Lr), (n, w, r)


@pytest.mark.parametrize("n", [33, 97, 256, 724, 1000, 1024])
def test_envelope_many_rows_bit_exact(api, n):
    # 4,096 rows or more take the warp-per-row kernels (the database rows'
    # envelopes of every knn_search call): lanes over runs of outputs when
    # 2w + 1 covers a lane's run (w >= 4 at n = 256, >= 16 at n = 1,000),
    # else the doubling table; sampled rows against the oracle
    count = 4500
    rng = np.random.default_rng(n + 1)
    Y = synth.random_walks(count, n, seed=n + 3)
    Y[::7] = rng.integers(-2, 3, size=Y[::7].shape).astype(np.float32)  # ties
    for w in sorted({0, 2, 3, 4, 15, 16, n // 10, n // 2, n - 1}):
        U, L = api.dtw_envelope(cuda(Y), w)
        U, L = U.cpu().numpy(), L.cpu().numpy()
        for r in list(range(0, count, 97)) + [count - 1]:
            Ur, Lr = oracle.envelope(Y[r], w)
            assert np.array_equal(U[r].astype(np.float64), Ur), (n, w, r)
            assert np.array_equal(L[r].astype(np.float64), Lr), (n, w, r)


# ---------------------------------------------------------------------------
# LB_Keogh and LB_Improved
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("n,w", [(1, 0), (5, 1), (128, 12), (131, 13), (256, 25), (1024, 102), (2048, 204)])
def test_lb_keogh_and_improved(api, p, n, w):
    N = 300
    X = synth.random_walks(N, n, seed=7 + n)
    y = synth.random_walks(1, n, seed=8 + n, stream=synth.STREAM_QUERY)[0]
    U, L = api.dtw_envelope(cuda(y), w)
    lbk = api.lb_keogh(cuda(X), U, L, p).cpu().numpy()
    lbi = api.lb_improved(cuda(X), cuda(y), U, L, w, p).cpu().numpy()
    for c in range(N):
        ri, rk = oracle.lb_improved_pow(X[c], y, w, p, with_first=True)
        assert close(lbk[c], rk ** (1.0 / p)), (c, lbk[c], rk)
        assert close(lbi[c], ri ** (1.0 / p)), (c, lbi[c], ri)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("n,d", [(1, 1), (37, 5), (128, 16), (181, 22), (256, 32), (256, 256), (1024, 128)])
def test_lb_piecewise(api, p, n, d):
    N = 200
    X = synth.random_walks(N, n, seed=11 + n)
    y = synth.random_walks(1, n, seed=12 + n, stream=synth.STREAM_QUERY)[0]
    w = max(1, n // 10)
    U, L = api.dtw_envelope(cuda(y), w)
    got = api.lb_piecewise(cuda(X), U, L, d, p).cpu().numpy().astype(np.float64)
    Uo, Lo = oracle.envelope(y, w)
    for c in range(N):
        ref = oracle.lb_piecewise_pow(X[c], y, w, d, p) ** (1.0 / p)
        # fp32 part sums cancel: allow the absolute rounding of sums of |values|
        scale = np.abs(X[c]).sum() + np.abs(Uo).sum() + np.abs(Lo).sum()
        tol = REL * ref + 4 * (n // d + 1) * 6e-8 * scale + ABS
        assert abs(got[c] - ref) <= tol, (c, got[c], ref)
        assert got[c] <= oracle.lb_keogh_pow(X[c], y, w, p) ** (1.0 / p) * (1 + 1e-5) + tol


# ---------------------------------------------------------------------------
# DTW
# ---------------------------------------------------------------------------

DTW_CASES = [(1, 0), (2, 1), (8, 3), (33, 0), (64, 6), (128, 12), (181, 18), (256, 25), (257, 51),
             (512, 51), (1024, 102), (400, 103), (300, 104), (1024, 150), (1024, 204), (600, 599)]


# p = 4 and p = infinity (App. C's other measures) through dtw_band; the
# oracle takes p = 0 for infinity
P_ALL = [1, 2, 4, math.inf]


def oracle_p(p):
    return 0 if p == math.inf else p


@pytest.mark.parametrize("p", P_ALL)
@pytest.mark.parametrize("n,w", DTW_CASES)
def test_dtw_band_shared_query(api, p, n, w):
    N = 70  # two full warps and a ragged tail
    X = synth.random_walks(N, n, seed=100 + n)
    y = synth.random_walks(1, n, seed=200 + n, stream=synth.STREAM_QUERY)[0]
    d = api.dtw_band(cuda(X), cuda(y), w, p).cpu().numpy()
    for c in range(N):
        ref = oracle.dtw(X[c], y, w, oracle_p(p))
        assert close(d[c], ref), (n, w, c, d[c], ref)


@pytest.mark.parametrize("p", P_ALL)
@pytest.mark.parametrize("n,w", [(16, 2), (256, 25), (1024, 204)])
def test_dtw_band_per_pair_query(api, p, n, w):
    N = 40
    X = synth.random_walks(N, n, seed=300 + n)
    Y = synth.random_walks(N, n, seed=301 + n, stream=synth.STREAM_QUERY)
    d = api.dtw_band(cuda(X), cuda(Y), w, p).cpu().numpy()
    for c in range(N):
        assert close(d[c], oracle.dtw(X[c], Y[c], w, oracle_p(p))), (c,)


@pytest.mark.parametrize("p", [4, math.inf])
def test_dtw_band_p4_and_inf_special_cases(api, p):
    # Sec. 4 / App. A facts that hold for every p: with w = 0 DTW_p is the l_p
    # distance; against a constant series DTW_p is the l_p distance too; and
    # DTW_inf(x, x + c) = |c| for a shift c
    g = np.random.default_rng(5)
    X = synth.random_walks(8, 64, seed=55)
    y = synth.random_walks(1, 64, seed=56, stream=synth.STREAM_QUERY)[0]
    d0 = api.dtw_band(cuda(X), cuda(y), 0, p).cpu().numpy()
    diff = np.abs(X.astype(np.float64) - y.astype(np.float64))
    lp = diff.max(axis=1) if p == math.inf else (diff ** 4).sum(axis=1) ** 0.25
    np.testing.assert_allclose(d0, lp, rtol=1e-5)
    cst = np.full(64, 1.5, np.float32)
    dc = api.dtw_band(cuda(X), cuda(cst), 10, p).cpu().numpy()
    dfc = np.abs(X.astype(np.float64) - 1.5)
    lpc = dfc.max(axis=1) if p == math.inf else (dfc ** 4).sum(axis=1) ** 0.25
    np.testing.assert_allclose(dc, lpc, rtol=1e-5)
    if p == math.inf:
        shift = np.float32(g.uniform(0.5, 2.0))
        Y = X + shift  # fp32: the per-element shifts differ by rounding
        ds = api.dtw_band(cuda(X), cuda(Y), 6, p).cpu().numpy()
        np.testing.assert_allclose(ds, np.abs(Y.astype(np.float64) - X).max(axis=1), rtol=2e-5)
        for c in range(len(X)):
            assert close(ds[c], oracle.dtw(X[c], Y[c], 6, 0)), c


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("n,w", [(64, 20), (128, 60), (100, 99)])
def test_dtw_band_per_pair_many_pairs(api, p, n, w):
    # 70,000 pairs with one query each: the warp path with two 16-lane groups
    # per warp; a short launch of the same pairs takes the 32-lane groups, and
    # both evaluate the same cells with the same fp32 operations
    N = 70_000
    X = synth.random_walks(N, n, seed=500 + n)
    Y = synth.random_walks(N, n, seed=600 + n, stream=synth.STREAM_QUERY)
    d = api.dtw_band(cuda(X), cuda(Y), w, p).cpu().numpy()
    head = api.dtw_band(cuda(X[:300]), cuda(Y[:300]), w, p).cpu().numpy()
    np.testing.assert_array_equal(d[:300], head)
    for c in list(range(0, N, 1400)) + [N - 1]:
        ref = oracle.dtw(X[c], Y[c], w, p)
        assert close(d[c], ref), (n, w, c, d[c], ref)


@pytest.mark.parametrize("p", P_ALL)
@pytest.mark.parametrize("n,w", [(128, 12), (1024, 204)])
def test_dtw_band_threshold(api, p, n, w):
    N = 64
    X = synth.random_walks(N, n, seed=400 + n)
    y = synth.random_walks(1, n, seed=401 + n, stream=synth.STREAM_QUERY)[0]
    ref = np.array([oracle.dtw(X[c], y, w, oracle_p(p)) for c in range(N)])
    thr = float(np.median(ref))
    d = api.dtw_band(cuda(X), cuda(y), w, p, threshold=thr).cpu().numpy()
    for c in range(N):
        if ref[c] > thr * (1 + 1e-4):
            assert math.isinf(d[c]), (c, d[c], ref[c], thr)
        elif ref[c] < thr * (1 - 1e-4):
            assert close(d[c], ref[c]), (c, d[c], ref[c])


def test_dtw_worked_examples(api):
    # Sec. 4 and App. A examples through the GPU path
    cases = [([0, 0, 1, 0], [2, 3, 2, 2], 1, 2, 17.0 ** 0.5), ([0, 0, 1, 0], [2, 3, 2, 2], 0, 2, 18.0 ** 0.5),
             ([0, 1, 2], [1, 2, 3], 1, 1, 2.0), ([0, 1, 2], [1, 2, 3], 0, 1, 3.0)]
    for x, y, w, p, v in cases:
        d = api.dtw_band(cuda(np.array([x])), cuda(np.array(y)), w, p).cpu().numpy()
        assert close(d[0], v)


# ---------------------------------------------------------------------------
# k nearest neighbours
# ---------------------------------------------------------------------------

def _knn_case(api, db, queries, w, p, k, mode="improved", **kw):
    idx, dist, st = api.knn_search(cuda(db), cuda(queries), w, p, k, mode=mode, return_stats=True, **kw)
    ri, rd, _ = oracle.knn_cascade(db, queries, w, p, k, mode=1, threads=8)
    assert_knn(db, queries, w, p, k, idx, dist, ri, rd)
    Q, N = queries.shape[0], db.shape[0]
    assert st["candidates"] == Q * N
    assert (st["seeds"] + st["pruned_summary"] + st["pruned_keogh"] + st["pruned_improved"] + st["dtw_computed"]
            == Q * N)
    return idx, dist, st


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("k", [1, 3, 10])
def test_knn_plain_cascade_small(api, p, k):
    # 1,000 random walks of length 128, band 12, 10 queries (the small plain case)
    db = synth.random_walks(1000, 128, seed=1)
    qs = synth.random_walks(10, 128, seed=1, stream=synth.STREAM_QUERY)
    _knn_case(api, db, qs, 12, p, k)


@pytest.mark.parametrize("mode", ["improved", "keogh", "noprune"])
def test_knn_modes_agree(api, mode):
    db = synth.random_walks(700, 96, seed=2)
    qs = synth.random_walks(9, 96, seed=2, stream=synth.STREAM_QUERY)
    _knn_case(api, db, qs, 9, 1, 4, mode=mode)


def test_knn_pruning_never_loses_the_neighbour(api):
    db = synth.random_walks(3000, 64, seed=3)
    qs = synth.random_walks(20, 64, seed=3, stream=synth.STREAM_QUERY)
    a = api.knn_search(cuda(db), cuda(qs), 6, 2, 5)
    b = api.knn_search(cuda(db), cuda(qs), 6, 2, 5, mode="noprune")
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    # an extreme slack prunes almost nothing and must give the same answer
    c = api.knn_search(cuda(db), cuda(qs), 6, 2, 5, slack=10.0)
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])


@pytest.mark.parametrize("parts", [-1, 0, 1, 8, 64])
@pytest.mark.parametrize("mode", ["improved", "keogh"])
def test_knn_piecewise_prefilter(api, parts, mode):
    # the piecewise-sum pass before LB_Keogh changes no result
    db = synth.random_walks(2500, 64, seed=13)
    qs = synth.random_walks(8, 64, seed=13, stream=synth.STREAM_QUERY)
    for p in (1, 2):
        idx, dist, st = _knn_case(api, db, qs, 6, p, 2, mode=mode, parts=parts)
        if parts == -1:
            assert st["pruned_summary"] == 0


@pytest.mark.parametrize("seeds", [1, 2, 32])
def test_knn_seed_count(api, seeds):
    db = synth.random_walks(900, 64, seed=4)
    qs = synth.random_walks(7, 64, seed=4, stream=synth.STREAM_QUERY)
    _knn_case(api, db, qs, 6, 1, 3, seeds=seeds)


WARP_CASES = [(1, 0, 3), (33, 0, 1), (40, 3, 2), (96, 9, 1), (128, 12, 10), (256, 25, 1), (512, 51, 3),
              (1024, 102, 1), (700, 150, 2), (1024, 204, 1), (900, 400, 1),
              # the one-row-per-step wavefront's bands (409 and 289 slots)
              (2048, 204, 3), (1448, 144, 2), (300, 144, 1), (230, 204, 4)]


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("n,w,k", WARP_CASES)
def test_knn_warp_dtw_path(api, p, n, w, k):
    # one warp per pair (the one-row-per-step wavefront for bands of 409 and
    # 289 slots, else two pairs per warp; wavefront abandoning) for every
    # DTW stage; the thread-per-pair kernels evaluate the same cells with the
    # same fp32 operations, so both paths give identical results (bands
    # wider than 208 slots: the wavefront against the two-steps-per-row
    # kernel of dtw_path 3)
    N = 400 if n >= 512 else 900
    db = synth.random_walks(N, n, seed=30 + n)
    qs = synth.random_walks(4, n, seed=30 + n, stream=synth.STREAM_QUERY)
    wi, wd, _ = _knn_case(api, db, qs, w, p, k, dtw_path=2)
    ti, td = api.knn_search(cuda(db), cuda(qs), w, p, k, dtw_path=1)
    assert torch.equal(wi, ti) and torch.equal(wd, td)
    if 2 * min(w, n - 1) + 1 <= 512:
        # the main stage on two 16-lane groups per warp
        gi, gd = api.knn_search(cuda(db), cuda(qs), w, p, k, dtw_path=3)
        assert torch.equal(gi, ti) and torch.equal(gd, td)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("n,w,k", [(256, 25, 1), (256, 25, 10), (200, 6, 3), (301, 30, 1), (130, 12, 2),
                                   (300, 40, 1), (517, 51, 3), (400, 102, 1), (260, 100, 5)])
def test_dtw_row_phases_equal_thread_path(api, p, n, w, k):
    # the main DTW stage in row phases of 64 rows (pairs alive at a phase's
    # end resumed by the next launch) gives the thread path's results bit
    # for bit; compile-time and runtime band paddings, n % 4 != 0 and n not a
    # multiple of the phase, bands of 4-rows-per-load kernels (up to 64
    # slots) and of the wider register kernels (96 to 208 slots); counters
    # still add up
    db = synth.random_walks(6_000, n, seed=60 + n)
    qs = synth.random_walks(40, n, seed=61 + n, stream=synth.STREAM_QUERY)
    ti, td = api.knn_search(cuda(db), cuda(qs), w, p, k, dtw_path=1)
    ri, rd, st = api.knn_search(cuda(db), cuda(qs), w, p, k, dtw_path=4, return_stats=True)
    assert torch.equal(ri, ti) and torch.equal(rd, td)
    pruned = st["pruned_summary"] + st["pruned_keogh"] + st["pruned_improved"]
    assert st["seeds"] + pruned + st["dtw_computed"] == st["candidates"]
    assert 0 < st["dtw_rows"] <= st["dtw_lane_rows"]
    oi, od, _ = oracle.knn_cascade(db, qs[:6], w, p, k, mode=1, threads=8)
    assert_knn(db, qs[:6], w, p, k, ti[:6], td[:6], oi, od)


def test_knn_edge_cases(api):
    # k > N pads with -1 / +inf; N = 1; n = 1; odd n (scalar load path); w = 0; w >= n
    db = synth.random_walks(5, 33, seed=5)
    qs = synth.random_walks(3, 33, seed=5, stream=synth.STREAM_QUERY)
    for w in (0, 4, 32, 100):
        for k in (1, 5, 8):
            _knn_case(api, db, qs, w, 1, k)
    _knn_case(api, db[:1], qs, 3, 2, 2)
    one = np.arange(12, dtype=np.float32).reshape(12, 1)
    _knn_case(api, one, one[[3, 7]] + 0.25, 0, 1, 3)


def test_knn_ties_go_to_lower_index(api):
    db = synth.random_walks(300, 40, seed=6)
    db[250] = db[17]
    db[260] = db[17]
    db[120] = db[200]
    qs = db[[17, 200]].copy()
    idx, dist = api.knn_search(cuda(db), cuda(qs), 4, 1, 3)
    idx = idx.cpu().numpy()
    assert list(idx[0]) == [17, 250, 260]
    assert list(idx[1][:2]) == [120, 200]
    assert float(dist[0, 0]) == 0.0


def test_knn_host_buffers(api):
    db = synth.random_walks(800, 64, seed=8)
    qs = synth.random_walks(6, 64, seed=8, stream=synth.STREAM_QUERY)
    dev = api.knn_search(cuda(db), cuda(qs), 6, 1, 2)
    host_q = torch.from_numpy(qs).pin_memory()
    host = api.knn_search(cuda(db), host_q, 6, 1, 2)
    assert not host[0].is_cuda
    assert torch.equal(dev[0].cpu(), host[0]) and torch.equal(dev[1].cpu(), host[1])
    allhost = api.knn_search(torch.from_numpy(db), torch.from_numpy(qs), 6, 1, 2)
    assert torch.equal(dev[0].cpu(), allhost[0])


def test_knn_shapes_long_series_wide_band(api):
    # shape-like series of length 1024 with w = 5 %, 10 %, 20 % (register and wide DTW paths)
    db = synth.shapes(1500, 1024, seed=9)
    qs = synth.shapes(3, 1024, seed=9, stream=synth.STREAM_QUERY)
    for w in (51, 102, 204):
        _knn_case(api, db, qs, w, 1, 1)


@pytest.mark.parametrize("p", [1, 2])
def test_knn_full_size_sampled(api, p):
    # 100,000 random walks of length 256, band 25, 1,000 queries, in the
    # launch configuration the benchmark times; a sample of queries is
    # checked against the oracle.
    db = synth.random_walks(100_000, 256, seed=2)
    qs = synth.random_walks(1000, 256, seed=2, stream=synth.STREAM_QUERY)
    idx, dist = api.knn_search(cuda(db), cuda(qs), 25, p, 1)
    sample = np.array([0, 1, 2, 3, 500, 997, 998, 999])
    ri, rd, _ = oracle.knn_cascade(db, qs[sample], 25, p, 1, mode=1, threads=16)
    assert_knn(db, qs[sample], 25, p, 1, idx[sample], dist[sample], ri, rd)


@pytest.mark.parametrize("p", P_ALL)
def test_classification_nearest_neighbours_match_the_oracle(api, p):
    # App. C: every test series against a small labelled database, all pairs
    # in one dtw_band launch, nearest neighbour by first minimum
    labels = np.repeat(np.arange(synth.SHAPE_CLASSES), 3)
    db = synth.shape_classes(labels, 128, seed=71)
    tl = np.random.default_rng(72).integers(0, synth.SHAPE_CLASSES, size=40)
    ts = synth.shape_classes(tl, 128, seed=71, stream=synth.STREAM_QUERY)
    k, T, w = len(labels), len(tl), 12
    X = np.ascontiguousarray(np.tile(db, (T, 1)))
    Y = np.ascontiguousarray(np.repeat(ts, k, axis=0))
    d = api.dtw_band(cuda(X), cuda(Y), w, p).cpu().numpy().reshape(T, k)
    nn = d.argmin(axis=1)
    for t in range(T):
        oi, od = oracle.knn_bruteforce(db, ts[t][None, :], w, oracle_p(p), 1)
        if nn[t] != oi[0, 0]:  # a near-tie fp32 cannot order: same distance
            assert close(oracle.dtw(db[nn[t]], ts[t], w, oracle_p(p)), od[0, 0]), (t, nn[t], oi[0, 0])
        assert close(d[t, nn[t]], od[0, 0]), t


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("n,w", [(200, 20), (201, 20), (301, 30), (1002, 100)])
def test_knn_filter_layouts(api, p, n, w):
    # the filter's row layouts besides the compiled fast one: 8 elements per
    # lane with rows shorter than 256 (16-byte pieces, then 4-byte copies when
    # n % 4 != 0) and streamed long rows with 4-byte loads (n % 4 != 0)
    db = synth.random_walks(600, n, seed=90 + n)
    qs = synth.random_walks(5, n, seed=91 + n, stream=synth.STREAM_QUERY)
    _knn_case(api, db, qs, w, p, 2)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("n,w", [(256, 25), (128, 12)])
def test_filter_paths_agree(api, p, n, w):
    # one warp per pair (1) and batches of eight pairs per warp (2) give the
    # same neighbours; with more queries
    # than one CTA wave and segments with ragged tails
    db = synth.random_walks(9_000, n, seed=150 + n)
    qs = synth.random_walks(70, n, seed=151 + n, stream=synth.STREAM_QUERY)
    out = {}
    for path in (1, 2):
        for k in (1, 7):
            out[path, k] = api.knn_search(cuda(db), cuda(qs), w, p, k, filter_path=path)
    for k in (1, 7):
        for path in (2,):
            assert torch.equal(out[path, k][0], out[1, k][0]) and torch.equal(out[path, k][1], out[1, k][1])
    ri, rd, _ = oracle.knn_cascade(db, qs[:12], w, p, 7, mode=1, threads=8)
    assert_knn(db, qs[:12], w, p, 7, out[2, 7][0][:12], out[2, 7][1][:12], ri, rd)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("n,w,k", [(1024, 102, 1), (600, 60, 5), (1002, 204, 1)])
def test_lb_early_abandon_same_result(api, p, n, w, k):
    # early abandoning inside the bound sums (streamed long rows) changes
    # which work is done, not the neighbours; the counters still add up
    db = synth.shapes(3_000, n, seed=80 + n)
    qs = synth.shapes(12, n, seed=81 + n, stream=synth.STREAM_QUERY)
    ri, rd, r_st = api.knn_search(cuda(db), cuda(qs), w, p, k, return_stats=True)
    ai, ad, a_st = api.knn_search(cuda(db), cuda(qs), w, p, k, lb_abandon=1, return_stats=True)
    assert torch.equal(ai, ri) and torch.equal(ad, rd)
    for st in (r_st, a_st):
        pruned = st["pruned_summary"] + st["pruned_keogh"] + st["pruned_improved"]
        assert st["seeds"] + pruned + st["dtw_computed"] == st["candidates"]
    oi, od, _ = oracle.knn_cascade(db, qs[:4], w, p, k, mode=1, threads=8)
    assert_knn(db, qs[:4], w, p, k, ai[:4], ad[:4], oi, od)
