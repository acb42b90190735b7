"""The second term of LB_Improved (Sec. 8) from envelopes alone.

LB_Improved_p(x, y)^p = LB_Keogh_p(x, y)^p + sum_i d(y_i, [L(H)_i, U(H)_i])^p
with H = H(x, y) the projection of x onto the envelope of y (Eq. 1) and
U(H), L(H) its envelope.  The GPU filter evaluates the second sum as

    sum_i d(y_i, [min(L(x)_i, L(U)_i), max(U(x)_i, U(L)_i)])^p

where U(x), L(x) is the candidate's own envelope (computed once per database
row and band) and U(L), L(U) are envelopes of the query's envelope (once per
query).  The two sums are equal term by term:

- U(H)_i <= max(U(x)_i, U(L)_i), since H_j = min(max(x_j, L_j), U_j) <=
  max(x_j, L_j); so when y_i <= U(H)_i both upper terms are 0.
- When y_i > U(H)_i: every j in the window of i has i in its own window, so
  U_j >= y_i > U(H)_i >= H_j; H_j is then never clipped at U_j, H_j =
  max(x_j, L_j) over the whole window, and U(H)_i = max(U(x)_i, U(L)_i).

The lower terms follow by symmetry.  These tests check the equality against
the oracle's direct evaluation (the projection and its envelope, as the paper
defines them) on series with ties, plateaus and clamped ends.
"""

import numpy as np
import pytest

import oracle
import synth


def second_from_envelopes(x, y, w, p):
    U, L = oracle.envelope(y, w)
    Ux, Lx = oracle.envelope(x, w)
    UL, _ = oracle.envelope_f64(L, w)
    _, LU = oracle.envelope_f64(U, w)
    y = np.asarray(y, np.float64)
    up = np.maximum(y - np.maximum(Ux, UL), 0.0)
    lo = np.maximum(np.minimum(Lx, LU) - y, 0.0)
    assert not np.any((up > 0) & (lo > 0))  # at most one side per index
    return float(np.sum((up + lo) ** p))


def second_direct(x, y, w, p):
    lbi, first = oracle.lb_improved_pow(x, y, w, p, with_first=True)
    return lbi - first


def cases():
    g = np.random.default_rng(2024)
    out = []
    for n in (1, 2, 3, 7, 32, 100, 257):
        for w in sorted({0, 1, n // 10, n // 3, n - 1, n + 5}):
            for kind in ("walk", "noise", "ints", "steps"):
                if kind == "walk":
                    x, y = synth.random_walks(2, n, seed=int(g.integers(1 << 30)))
                elif kind == "noise":
                    x, y = synth.white_noise(2, n, seed=int(g.integers(1 << 30)))
                elif kind == "ints":  # many ties
                    x, y = g.integers(-3, 4, size=(2, n)).astype(np.float32)
                else:  # plateaus
                    lv = g.integers(-5, 6, size=(2, 4)).astype(np.float32)
                    cut = np.sort(g.integers(0, n + 1, size=3))
                    x, y = (np.repeat(row, np.diff(np.r_[0, cut, n])) for row in lv)
                out.append((kind, n, w, np.ascontiguousarray(x, np.float32), np.ascontiguousarray(y, np.float32)))
    return out


@pytest.mark.parametrize("p", [1, 2])
def test_second_term_equals_the_envelope_form(p):
    for kind, n, w, x, y in cases():
        a = second_direct(x, y, w, p)
        b = second_from_envelopes(x, y, w, p)
        assert abs(a - b) <= 1e-12 * max(1.0, abs(a)), (kind, n, w, a, b)


def test_shape_like_series_long_band():
    db = synth.shapes(6, 512, seed=77)
    q = synth.shapes(1, 512, seed=77, stream=synth.STREAM_QUERY)[0]
    for w in (25, 51, 204):
        for x in db:
            for p in (1, 2):
                a = second_direct(x, q, w, p)
                b = second_from_envelopes(x, q, w, p)
                assert abs(a - b) <= 1e-12 * max(1.0, abs(a)), (w, p, a, b)


def test_the_query_side_envelope_is_needed():
    # x far below y's envelope: H = L there, so U(H) comes from U(L), not from
    # U(x); a form that dropped U(L) would give a different (wrong) sum, so
    # the equality above is a real check of that term
    x = np.full(6, -10.0, np.float32)
    y = np.array([0, 5, 0, 0, 0, 0], np.float32)
    w = 1
    Ux, _ = oracle.envelope(x, w)
    wrong = float(np.sum(np.maximum(y - Ux, 0.0)))
    assert second_direct(x, y, w, 1) == pytest.approx(second_from_envelopes(x, y, w, 1))
    assert abs(second_direct(x, y, w, 1) - wrong) > 1.0
