"""Triangle-inequality ratios of App. B (dtw_triangle) against the oracle.

For triples of white-noise, random-walk and shape-like series of 100 samples,
with no time constraint (w = n - 1, the paper's setting) and with a band,
the three DTW_p distances must match the oracle within 1e-5 relative and the
ratio DTW_p(x,z) / (DTW_p(x,y) + DTW_p(y,z)) within 3e-5 relative.
"""

import math

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


GENS = {
    "white_noise": synth.white_noise,
    "random_walk": synth.random_walks,
    "shapes": synth.shapes,
}


@pytest.mark.parametrize("kind", sorted(GENS))
@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("w", [99, 10])
def test_triangle_ratio_matches_oracle(api, kind, p, w):
    N, n = 150, 100
    g = GENS[kind]
    x, y, z = (g(N, n, seed=60 + s) for s in range(3))
    ratio, d3 = api.dtw_triangle(cuda(x), cuda(y), cuda(z), w, p, with_distances=True)
    ratio, d3 = ratio.cpu().numpy().astype(np.float64), d3.cpu().numpy().astype(np.float64)
    for i in range(N):
        dxy = oracle.dtw(x[i], y[i], w, p)
        dyz = oracle.dtw(y[i], z[i], w, p)
        dxz = oracle.dtw(x[i], z[i], w, p)
        for got, ref in ((d3[0, i], dxy), (d3[1, i], dyz), (d3[2, i], dxz)):
            assert abs(got - ref) <= 1e-5 * ref + 1e-5, (i, got, ref)
        r = dxz / (dxy + dyz)
        assert abs(ratio[i] - r) <= 3e-5 * r + 1e-6, (i, ratio[i], r)


def test_triangle_degenerate_triples(api):
    n = 20
    x = synth.random_walks(3, n, seed=3)
    # identical triples: 0 / 0 -> 0; x = y != z: ratio exactly 1
    ratio = api.dtw_triangle(cuda(x), cuda(x), cuda(x), n - 1, 1).cpu().numpy()
    assert (ratio == 0).all()
    z = x + 1.0
    ratio = api.dtw_triangle(cuda(x), cuda(x), cuda(z), n - 1, 2).cpu().numpy()
    assert np.allclose(ratio, 1.0, rtol=1e-6)
    assert math.isfinite(float(ratio.max()))
