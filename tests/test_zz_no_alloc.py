"""dtw_band_noalloc, the DTW entry point for callers that cannot allocate
device memory (for example a service whose GPU memory belongs to another
allocator, or a loop that must not stall on cudaFree).  It takes its scratch
from a fixed array inside the library instead of the growable workspace.

This file is collected last, so that a run stopping at the first failure has
already run every other test.  The test also passes on its own in a fresh
process.
"""

import ctypes
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

REL = 1e-5
ABS = 1e-5


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _call(fn, x, y, n, w, p, thr, per_pair):
    out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    st = fn(x.data_ptr(), y.data_ptr(), x.shape[0], n if per_pair else 0, n, w, p, ctypes.c_float(thr),
            out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st, out


def test_noalloc_matches_dtw_band_on_two_calls_in_a_row():
    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import _native as N

    lib = N.lib
    n, w, p = 256, 25, 1
    X = _cuda(synth.random_walks(70, n, seed=901))
    y = _cuda(synth.random_walks(1, n, seed=902, stream=synth.STREAM_QUERY)[0])
    Y = _cuda(synth.random_walks(70, n, seed=903, stream=synth.STREAM_QUERY))
    # first call: one shared query; second call: one query per pair, p = 2,
    # and a finite threshold, on the same (reused) scratch
    calls = [(y, False, 1, math.inf), (Y, True, 2, 0.0)]
    for yy, per_pair, pp, thr in calls:
        st_ref, ref = _call(lib.dtw_band, X, yy, n, w, pp, thr if thr else math.inf, per_pair)
        assert st_ref == 0
        if not thr:
            thr = float(torch.median(ref).item())
            st_ref, ref = _call(lib.dtw_band, X, yy, n, w, pp, thr, per_pair)
            assert st_ref == 0
        st, got = _call(lib.dtw_band_noalloc, X, yy, n, w, pp, thr, per_pair)
        assert st == 0, lib.dtw_last_error().decode()
        torch.cuda.synchronize()
        a, b = got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        both_inf = np.isinf(a) & np.isinf(b)
        with np.errstate(invalid="ignore"):
            near = np.abs(a - b) <= REL * np.abs(b) + ABS
        assert np.all(both_inf | near)


def test_noalloc_rejects_scratch_beyond_its_limit():
    from paper_0811_3301_gb300 import _native as N

    n, w = 1024, 100
    X = torch.zeros((2000, n), dtype=torch.float32, device="cuda")
    st, _ = _call(N.lib.dtw_band_noalloc, X, X, n, w, 1, math.inf, True)
    assert st == 1  # DTW_ERR_INVALID_ARG
    assert "scratch" in N.lib.dtw_last_error().decode()
