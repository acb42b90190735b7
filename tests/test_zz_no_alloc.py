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
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

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


def _close(got, ref):
    a, b = got.cpu().numpy().astype(np.float64), np.asarray(ref, dtype=np.float64)
    both_inf = np.isinf(a) & np.isinf(b)
    with np.errstate(invalid="ignore"):
        near = np.abs(a - b) <= REL * np.abs(b) + ABS
    return bool(np.all(both_inf | near))


@pytest.mark.parametrize("n,w,p", [(512, 150, 1), (512, 150, 4), (2048, 600, 2), (300, 40, 0)])
def test_noalloc_matches_the_oracle_and_dtw_band(n, w, p):
    """Bands wider than one thread's registers (2w + 1 > 208: the warp path,
    and > 1024: the wide path), p = 4 and p = infinity (0), one shared query,
    against the FP64 oracle and against dtw_band."""
    import oracle
    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import _native as N

    xs = synth.random_walks(12, n, seed=911 + n + p)
    y = synth.random_walks(1, n, seed=912 + n, stream=synth.STREAM_QUERY)[0]
    X, Y = _cuda(xs), _cuda(y)
    st, got = _call(N.lib.dtw_band_noalloc, X, Y, n, w, p, math.inf, False)
    assert st == 0, N.lib.dtw_last_error().decode()
    st_ref, ref = _call(N.lib.dtw_band, X, Y, n, w, p, math.inf, False)
    assert st_ref == 0
    torch.cuda.synchronize()
    assert _close(got, ref.cpu().numpy())
    assert _close(got, [oracle.dtw(xs[c], y, w, p) for c in range(len(xs))])


_FRESH = r"""
import ctypes, math, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import synth
from paper_0811_3301_gb300 import _native as N
n, w = 256, 25
X = torch.from_numpy(synth.random_walks(500, n, seed=921)).cuda()
Y = torch.from_numpy(synth.random_walks(500, n, seed=922, stream=synth.STREAM_QUERY)).cuda()
out = torch.empty(500, dtype=torch.float32, device="cuda")
s = torch.cuda.current_stream().cuda_stream
def call(N_, stride, p):
    st = N.lib.dtw_band_noalloc(X.data_ptr(), Y.data_ptr(), N_, stride, n, w, p, ctypes.c_float(math.inf),
                                out.data_ptr(), s)
    assert st == 0, N.lib.dtw_last_error().decode()
calls = [(500, n, 1), (500, n, 2), (500, 0, 1), (37, n, 0), (500, n, 4)]
# warm-up: loads each kernel's code and looks up the scratch address once
for c in calls:
    call(*c)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
for _ in range(2):
    for c in calls:
        call(*c)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
assert free1 == free0, (free0, free1)
print("noalloc-free-unchanged", free0)
"""


def test_noalloc_allocates_nothing_in_a_fresh_process():
    """In a fresh process where dtw_band never ran (so the library's growable
    workspace was never allocated), the device's free memory is the same
    before and after two more rounds of calls, once a warm-up round has
    loaded the kernels' code."""
    from paper_0811_3301_gb300 import build

    build.build()
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "noalloc-free-unchanged" in r.stdout
