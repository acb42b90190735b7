"""Pins of the FP64 oracle to what the paper and the mathematics fix.

None of these compare the oracle with itself: each check is a value the
paper prints (tests/golden), a closed form, an invariant the paper proves,
a special case that reduces to a library routine (numpy / scipy.ndimage),
or brute force over all warping paths on tiny inputs.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "worked_examples.json")))


def _p_code(p):
    return 0 if p == "inf" else int(p)


# ---------------------------------------------------------------------------
# brute force over warping paths (Sec. 4: a warping path is a monotone set
# of matches (i, j) from (1,1) to (n,n) with |i - j| <= w)
# ---------------------------------------------------------------------------

def brute_dtw_pow(x, y, w, p, count=False):
    n = len(x)
    best = [math.inf]
    npaths = [0]

    def cost(i, j):
        d = abs(float(x[i]) - float(y[j]))
        return d if p in (0, 1) else d ** p

    def rec(i, j, acc):
        if abs(i - j) > w:
            return
        c = cost(i, j)
        acc = max(acc, c) if p == 0 else acc + c
        if i == n - 1 and j == n - 1:
            npaths[0] += 1
            best[0] = min(best[0], acc)
            return
        if i + 1 < n:
            rec(i + 1, j, acc)
        if j + 1 < n:
            rec(i, j + 1, acc)
        if i + 1 < n and j + 1 < n:
            rec(i + 1, j + 1, acc)

    rec(0, 0, 0.0)
    return (best[0], npaths[0]) if count else best[0]


def test_bruteforce_enumerator_counts_delannoy():
    # The number of monotone paths with unit and diagonal steps on an 8x8
    # grid is the central Delannoy number D(7,7) = 48639.
    x = np.zeros(8)
    _, cnt = brute_dtw_pow(x, x, 7, 1, count=True)
    assert cnt == 48639


@pytest.mark.parametrize("p", [1, 2, 4, 0])
def test_dtw_matches_bruteforce_integer_series(p):
    rng = np.random.default_rng(11)
    for n in range(1, 8):
        for trial in range(6):
            x = rng.integers(-4, 5, size=n).astype(np.float32)
            y = rng.integers(-4, 5, size=n).astype(np.float32)
            for w in range(0, n + 1):
                assert oracle.dtw_pow(x, y, w, p) == brute_dtw_pow(x, y, w, p), (n, w, x, y)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_dtw_matches_bruteforce_real_series(p):
    rng = np.random.default_rng(12)
    for n in (5, 8):
        for trial in range(3):
            x = rng.standard_normal(n).astype(np.float32)
            y = rng.standard_normal(n).astype(np.float32)
            for w in (0, 1, 2, n):
                a = oracle.dtw_pow(x, y, w, p)
                b = brute_dtw_pow(x, y, w, p)
                assert a == pytest.approx(b, rel=1e-12, abs=1e-12)


# ---------------------------------------------------------------------------
# worked examples printed in the paper
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_worked_examples(case):
    x = np.array(case["x"], np.float32)
    y = np.array(case["y"], np.float32)
    p = _p_code(case["p"])
    n = len(x)
    for w in range(case["w_min"], n + 3):
        assert oracle.dtw_pow(x, y, w, p) == case["dtw_pow"], w
    if "lp_pow" in case:
        assert oracle.dtw_pow(x, y, 0, p) == case["lp_pow"]
    if case["w_min"] > 0:
        assert oracle.dtw_pow(x, y, case["w_min"] - 1, p) != case["dtw_pow"]


def test_xyz_family_appendix_b():
    fam = GOLD["xyz_family"]
    for m in fam["m_values"]:
        for eps in fam["eps_values"]:
            n = 2 * m + 1
            X = np.zeros(n, np.float32)
            Y = np.zeros(n, np.float32)
            Y[m] = eps
            Z = np.zeros(n, np.float32)
            Z[1:-1] = eps
            w = m - 1
            for p in (1, 2):
                e = abs(eps) ** p
                assert oracle.dtw_pow(X, Y, w, p) == e
                assert oracle.dtw_pow(Y, Z, w, p) == 0.0
                assert oracle.dtw_pow(X, Z, w, p) == (2 * m - 1) * e
                # the weak triangle inequality of App. B is tight here
                lhs = oracle.dtw(X, Y, w, p) + oracle.dtw(Y, Z, w, p)
                rhs = oracle.dtw(X, Z, w, p) / min(2 * w + 1, n) ** (1.0 / p)
                assert lhs == pytest.approx(rhs, rel=1e-12)


# ---------------------------------------------------------------------------
# closed forms and invariants of Sec. 4 and App. A/B
# ---------------------------------------------------------------------------

def _walks(count, n, seed):
    return synth.random_walks(count, n, seed=seed)


@pytest.mark.parametrize("p", [1, 2, 4, 0])
def test_w0_is_lp_distance(p):
    for x, y in zip(_walks(5, 40, 1), _walks(5, 40, 2)):
        d = np.abs(x.astype(np.float64) - y.astype(np.float64))
        ref = d.max() if p == 0 else np.sum(d ** p)
        assert oracle.dtw_pow(x, y, 0, p) == pytest.approx(ref, rel=1e-13)


def test_prop1_value_separated_dtw1_is_l1():
    rng = np.random.default_rng(5)
    for trial in range(10):
        n = int(rng.integers(2, 60))
        c = float(rng.standard_normal())
        x = (c + np.abs(rng.standard_normal(n))).astype(np.float32)
        y = (c - np.abs(rng.standard_normal(n))).astype(np.float32)
        l1 = np.sum(np.abs(x.astype(np.float64) - y))
        for w in (0, 1, n // 10, n):
            assert oracle.dtw_pow(x, y, w, 1) == pytest.approx(l1, rel=1e-12)
            assert oracle.dtw_pow(y, x, w, 1) == pytest.approx(l1, rel=1e-12)


@pytest.mark.parametrize("p", [1, 2, 4, 0])
def test_constant_series_lemma(p):
    rng = np.random.default_rng(6)
    for trial in range(6):
        n = int(rng.integers(1, 50))
        x = rng.standard_normal(n).astype(np.float32)
        y = np.full(n, np.float32(rng.standard_normal()))
        d = np.abs(x.astype(np.float64) - y)
        ref = d.max() if p == 0 else np.sum(d ** p)
        for w in (0, 2, n):
            assert oracle.dtw_pow(x, y, w, p) == pytest.approx(ref, rel=1e-12)


def test_dtw_nonincreasing_in_p():
    # App. A: DTW_p (root taken) does not increase with p, DTW_inf the smallest
    for x, y in zip(_walks(6, 30, 7), _walks(6, 30, 8)):
        for w in (0, 3, 30):
            vals = [oracle.dtw(x, y, w, p) for p in (1, 2, 4, 0)]
            for a, b in zip(vals, vals[1:]):
                assert a >= b * (1 - 1e-12), (w, vals)


@pytest.mark.parametrize("p", [1, 2])
def test_dtw_nonincreasing_in_w(p):
    for x, y in zip(_walks(4, 30, 3), _walks(4, 30, 4)):
        vals = [oracle.dtw_pow(x, y, w, p) for w in range(0, 31)]
        assert all(b <= a for a, b in zip(vals, vals[1:]))
        assert oracle.dtw_pow(x, y, 29, p) == oracle.dtw_pow(x, y, 1000, p)


@pytest.mark.parametrize("p", [1, 2])
def test_translation_invariance_dyadic(p):
    for x, y in zip(_walks(4, 33, 7), _walks(4, 33, 8)):
        for b in (0.5, -4.0, 2.25):
            xb = (x.astype(np.float64) + b).astype(np.float32)
            yb = (y.astype(np.float64) + b).astype(np.float32)
            if not (np.all(xb - b == x) and np.all(yb - b == y)):
                continue
            for w in (0, 3, 33):
                assert oracle.dtw_pow(xb, yb, w, p) == oracle.dtw_pow(x, y, w, p)


def test_p_monotonicity_proposition():
    for x, y in zip(_walks(5, 25, 9), _walks(5, 25, 10)):
        n = len(x)
        for w in (1, 4, 25):
            d1 = oracle.dtw(x, y, w, 1)
            d2 = oracle.dtw(x, y, w, 2)
            di = oracle.dtw(x, y, w, 0)
            assert (2 * n - 2) ** (1 - 0.5) * d2 >= d1 * (1 - 1e-12)
            assert (2 * n - 2) ** 1.0 * di >= d1 * (1 - 1e-12)
            assert (2 * n - 2) ** 0.5 * di >= d2 * (1 - 1e-12)
            assert d1 >= d2 >= di  # DTW_p decreases as p increases


@pytest.mark.parametrize("p", [1, 2])
def test_weak_triangle_inequality(p):
    X, Y, Z = _walks(6, 20, 11), _walks(6, 20, 12), _walks(6, 20, 13)
    for x, y, z in zip(X, Y, Z):
        for w in (0, 2, 20):
            lhs = oracle.dtw(x, y, w, p) + oracle.dtw(y, z, w, p)
            rhs = oracle.dtw(x, z, w, p) / min(2 * w + 1, 20) ** (1.0 / p)
            assert lhs >= rhs * (1 - 1e-12)


# ---------------------------------------------------------------------------
# envelope (Sec. 5) and projection (Eq. 1)
# ---------------------------------------------------------------------------

def test_envelope_equals_library_window_filters():
    rng = np.random.default_rng(21)
    for n in (1, 2, 7, 64, 257):
        y = rng.integers(-3, 4, size=n).astype(np.float32)  # many ties
        z = rng.standard_normal(n).astype(np.float32)
        for s in (y, z):
            for w in (0, 1, 3, n // 2, n - 1, n, n + 7):
                U, L = oracle.envelope(s, w)
                size = 2 * w + 1
                Ur = ndimage.maximum_filter1d(s.astype(np.float64), size=size, mode="nearest")
                Lr = ndimage.minimum_filter1d(s.astype(np.float64), size=size, mode="nearest")
                assert np.array_equal(U, Ur) and np.array_equal(L, Lr), (n, w)


def test_envelope_special_cases():
    y = _walks(1, 50, 22)[0]
    U, L = oracle.envelope(y, 0)
    assert np.array_equal(U, y.astype(np.float64)) and np.array_equal(L, y.astype(np.float64))
    U, L = oracle.envelope(y, 49)
    assert np.all(U == y.max()) and np.all(L == y.min())


def test_projection_is_clip():
    rng = np.random.default_rng(23)
    y = rng.standard_normal(100).astype(np.float32)
    x = (2 * rng.standard_normal(100)).astype(np.float32)
    U, L = oracle.envelope(y, 5)
    H = oracle.projection(x.astype(np.float64), U, L)
    assert np.array_equal(H, np.clip(x.astype(np.float64), L, U))
    # H lies in the envelope of y (Sec. 7)
    assert np.all(H <= U) and np.all(H >= L)


# ---------------------------------------------------------------------------
# LB_Keogh (Sec. 7) and LB_Improved (Sec. 8)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2])
def test_bounds_at_w0_equal_lp(p):
    # w = 0: U = L = y, so H(x, y) = y, LB_Keogh is the l_p distance, the
    # second LB_Improved term vanishes, and DTW is the l_p distance too.
    for x, y in zip(_walks(4, 64, 31), _walks(4, 64, 32)):
        lp = np.sum(np.abs(x.astype(np.float64) - y) ** p)
        assert oracle.lb_keogh_pow(x, y, 0, p) == pytest.approx(lp, rel=1e-13)
        lbi, lbk = oracle.lb_improved_pow(x, y, 0, p, with_first=True)
        assert lbk == pytest.approx(lp, rel=1e-13)
        assert lbi == pytest.approx(lp, rel=1e-13)


@pytest.mark.parametrize("p", [1, 2])
def test_lb_improved_constant_candidate_closed_form(p):
    # x = c >= max(y): H(x, y) = U(y) (grey dilation of y); the envelope of
    # U(y) has lower side erosion(dilation(y)) = closing(y) >= y, so the second
    # term is sum (closing(y) - y)^p.  Symmetrically for c <= min(y) with the
    # grey opening.  DTW_p is then ||c - y||_p (constant-series lemma).
    rng = np.random.default_rng(33)
    for trial in range(6):
        n = int(rng.integers(3, 80))
        w = int(rng.integers(0, n))
        y = rng.standard_normal(n).astype(np.float32)
        yd = y.astype(np.float64)
        size = 2 * w + 1
        dil = ndimage.grey_dilation(yd, size=size, mode="nearest")
        ero = ndimage.grey_erosion(yd, size=size, mode="nearest")
        clo = ndimage.grey_closing(yd, size=size, mode="nearest")
        opn = ndimage.grey_opening(yd, size=size, mode="nearest")
        c_hi = np.float32(y.max() + 1.5)
        x = np.full(n, c_hi, np.float32)
        ref_k = np.sum((c_hi - dil) ** p)
        ref_i = ref_k + np.sum((clo - yd) ** p)
        lbi, lbk = oracle.lb_improved_pow(x, y, w, p, with_first=True)
        assert lbk == pytest.approx(ref_k, rel=1e-12)
        assert lbi == pytest.approx(ref_i, rel=1e-12)
        assert oracle.dtw_pow(x, y, w, p) == pytest.approx(np.sum((c_hi - yd) ** p), rel=1e-12)
        c_lo = np.float32(y.min() - 0.75)
        x = np.full(n, c_lo, np.float32)
        ref_k = np.sum((ero - c_lo) ** p)
        ref_i = ref_k + np.sum((yd - opn) ** p)
        lbi, lbk = oracle.lb_improved_pow(x, y, w, p, with_first=True)
        assert lbk == pytest.approx(ref_k, rel=1e-12)
        assert lbi == pytest.approx(ref_i, rel=1e-12)


def test_lb_improved_small_hand_case():
    # n = 5, w = 1, y = (0,2,0,0,1), x = 3: U(y) = (2,2,2,1,1) so LB_Keogh_1 = 7;
    # the envelope of H = U(y) is U' = (2,2,2,2,1), L' = (2,2,1,1,1), and y lies
    # below it by (2,0,1,1,0): LB_Improved_1 = 11; DTW_1 = sum(3 - y) = 12.
    x = np.full(5, 3, np.float32)
    y = np.array([0, 2, 0, 0, 1], np.float32)
    lbi, lbk = oracle.lb_improved_pow(x, y, 1, 1, with_first=True)
    assert (lbk, lbi) == (7.0, 11.0)
    assert oracle.dtw_pow(x, y, 1, 1) == 12.0


@pytest.mark.parametrize("p", [1, 2])
def test_lb_improved_through_library_routines(p):
    # The whole second pass written with np.clip and scipy window filters.
    rng = np.random.default_rng(34)
    for trial in range(8):
        n = int(rng.integers(2, 120))
        w = int(rng.integers(0, n + 2))
        x = (rng.standard_normal(n) * 3).astype(np.float32)
        y = (rng.standard_normal(n) * 3).astype(np.float32)
        xd, yd = x.astype(np.float64), y.astype(np.float64)
        size = 2 * w + 1
        U = ndimage.maximum_filter1d(yd, size=size, mode="nearest")
        L = ndimage.minimum_filter1d(yd, size=size, mode="nearest")
        h = np.clip(xd, L, U)
        Uh = ndimage.maximum_filter1d(h, size=size, mode="nearest")
        Lh = ndimage.minimum_filter1d(h, size=size, mode="nearest")
        ref = np.sum(np.abs(xd - h) ** p) + np.sum(np.abs(yd - np.clip(yd, Lh, Uh)) ** p)
        assert oracle.lb_improved_pow(x, y, w, p) == pytest.approx(ref, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("p", [1, 2])
def test_bound_ordering_and_error_bounds(p):
    # LB_Keogh <= LB_Improved <= DTW <= l_p (Corollaries 1 and 2, Sec. 4);
    # DTW - LB_Keogh <= ||max(U - y, y - L)||_p (Corollary 1);
    # |DTW - ||x - h||| <= ||h - y|| with h = H(x, y) (Proposition 2).
    X = synth.random_walks(12, 96, seed=41)
    Y = synth.random_walks(12, 96, seed=42)
    for x, y in zip(X, Y):
        xd, yd = x.astype(np.float64), y.astype(np.float64)
        for w in (1, 9, 30):
            lbi, lbk = oracle.lb_improved_pow(x, y, w, p, with_first=True)
            d = oracle.dtw_pow(x, y, w, p)
            lp = np.sum(np.abs(xd - yd) ** p)
            tol = 1e-12 * max(1.0, d)
            assert lbk <= lbi + tol and lbi <= d + tol and d <= lp + tol
            U, L = oracle.envelope(y, w)
            width = np.sum(np.maximum(U - yd, yd - L) ** p) ** (1.0 / p)
            assert d ** (1.0 / p) - lbk ** (1.0 / p) <= width + 1e-9
            h = oracle.projection(xd, U, L)
            xh = np.sum(np.abs(xd - h) ** p) ** (1.0 / p)
            hy = np.sum(np.abs(h - yd) ** p) ** (1.0 / p)
            assert abs(d ** (1.0 / p) - xh) <= hy + 1e-9


# ---------------------------------------------------------------------------
# k nearest neighbours
# ---------------------------------------------------------------------------

def test_knn_bruteforce_against_path_enumeration():
    rng = np.random.default_rng(51)
    n, N = 5, 25
    db = rng.integers(-2, 3, size=(N, n)).astype(np.float32)  # ties in distance
    qs = rng.integers(-2, 3, size=(3, n)).astype(np.float32)
    for p in (1, 2):
        for w in (0, 1, 4):
            for k in (1, 4, 30):
                idx, dist = oracle.knn_bruteforce(db, qs, w, p, k)
                for qi, q in enumerate(qs):
                    d = [brute_dtw_pow(db[c], q, w, p) for c in range(N)]
                    order = sorted(range(N), key=lambda c: (d[c], c))[:k]
                    exp_idx = order + [-1] * (k - len(order))
                    assert list(idx[qi]) == exp_idx
                    for j, c in enumerate(order):
                        assert dist[qi, j] == pytest.approx(d[c] ** (1.0 / p), rel=1e-14)
                    assert np.all(np.isinf(dist[qi, len(order):]))


def test_knn_query_in_database_is_found():
    db = synth.random_walks(200, 48, seed=52)
    db[117] = db[40]  # duplicate: ties go to the lower index
    idx, dist = oracle.knn_bruteforce(db, db[[40, 3]], 4, 1, 2)
    assert list(idx[0]) == [40, 117] and dist[0, 0] == 0.0 and dist[0, 1] == 0.0
    assert idx[1, 0] == 3 and dist[1, 0] == 0.0


@pytest.mark.parametrize("p", [1, 2])
def test_cascades_equal_bruteforce(p):
    db = synth.random_walks(400, 40, seed=61)
    qs = synth.random_walks(6, 40, seed=61, stream=synth.STREAM_QUERY)
    for w in (0, 4, 39):
        for k in (1, 3, 7):
            bi, bd = oracle.knn_bruteforce(db, qs, w, p, k)
            i0, d0, s0 = oracle.knn_cascade(db, qs, w, p, k, mode=0)
            i1, d1, s1 = oracle.knn_cascade(db, qs, w, p, k, mode=1)
            assert np.array_equal(bi, i0) and np.array_equal(bi, i1)
            assert np.array_equal(bd, d0) and np.array_equal(bd, d1)
            assert np.all(s0[:, 0] == 400) and np.all(s1[:, 0] == 400)
            assert np.all(s0[:, 1] + s0[:, 2] + s0[:, 3] == 400) and np.all(s0[:, 2] == 0)
            assert np.all(s1[:, 1] + s1[:, 2] + s1[:, 3] == 400)
            # same threshold trajectory, so LB_Improved never computes more DTWs
            assert np.all(s1[:, 1] == s0[:, 1]) and np.all(s1[:, 3] <= s0[:, 3])


# ---------------------------------------------------------------------------
# piecewise-sum bound (Sec. 9)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2])
def test_piecewise_with_unit_parts_is_lb_keogh(p):
    # d = n: every part is one index, so the bound is LB_Keogh itself
    for x, y in zip(_walks(4, 37, 71), _walks(4, 37, 72)):
        for w in (0, 3, 37):
            assert oracle.lb_piecewise_pow(x, y, w, 37, p) == pytest.approx(oracle.lb_keogh_pow(x, y, w, p), rel=1e-13)


@pytest.mark.parametrize("p", [1, 2])
def test_piecewise_single_part_closed_form(p):
    # d = 1: |sum x - clip(sum x, sum L, sum U)|^p / n^(p-1)
    for x, y in zip(_walks(4, 50, 73), _walks(4, 50, 74)):
        U, L = oracle.envelope(y, 5)
        sx = np.sum(x.astype(np.float64))
        dd = abs(sx - np.clip(sx, L.sum(), U.sum()))
        ref = dd if p == 1 else dd * dd / 50
        assert oracle.lb_piecewise_pow(x, y, 5, 1, p) == pytest.approx(ref, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("p", [1, 2])
def test_piecewise_is_below_lb_keogh_and_cover(p):
    # the bound never exceeds LB_Keogh (Sec. 9 chain of inequalities); the
    # cover: floor(n/d) per part, the last part takes the rest (checked with
    # numpy sums over explicit index sets)
    X, Y = _walks(10, 61, 75), _walks(10, 61, 76)
    for x, y in zip(X, Y):
        for w in (2, 6, 20):
            U, L = oracle.envelope(y, w)
            lbk = oracle.lb_keogh_pow(x, y, w, p)
            for d in (1, 2, 7, 8, 30, 61):
                v = oracle.lb_piecewise_pow(x, y, w, d, p)
                assert v <= lbk * (1 + 1e-12) + 1e-12
                s = 61 // d
                parts = [list(range(j * s, (j + 1) * s)) for j in range(d - 1)] + [list(range((d - 1) * s, 61))]
                smax = max(len(c) for c in parts)
                tot = 0.0
                for c in parts:
                    px, pu, pl = x[c].astype(np.float64).sum(), U[c].sum(), L[c].sum()
                    dj = max(px - pu, pl - px, 0.0)
                    tot += dj if p == 1 else dj * dj
                assert v == pytest.approx(tot if p == 1 else tot / smax, rel=1e-12, abs=1e-12)
