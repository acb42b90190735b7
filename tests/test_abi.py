"""The C-ABI library builds, loads and exports every symbol the header
declares; argument checks run on the host (no GPU needed)."""

import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dtwknn.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:dtw_status|const char\s*\*|int64_t)\s*(\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def native():
    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import _native

    return _native


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dtw_envelope", "lb_keogh", "lb_improved", "dtw_band", "knn_search", "knn_search_ex",
                     "dtw_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    missing = [name for name in _declared_functions() if not hasattr(lib, name)]
    assert missing == []


def test_binding_covers_every_declared_symbol(native):
    bound = set(native.SIGNATURES) | {"dtw_last_error", "dtw_version", "dtw_monotonic_ns"}
    assert set(_declared_functions()) <= bound


def test_library_is_built_for_sm103a(native):
    # the objects were produced with -gencode arch=compute_103a,code=sm_103a
    from paper_0811_3301_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def _status(native, call):
    st = call()
    msg = native.lib.dtw_last_error().decode()
    return st, msg


@pytest.mark.parametrize(
    "n,w,p,k,msg",
    [
        (0, 1, 1, 1, "n=0"),
        (5000, 1, 1, 1, "n=5000"),
        (16, -1, 1, 1, "w=-1"),
        (16, 1, 3, 1, "p=3"),
        (16, 1, 1, 0, "k=0"),
        (16, 1, 1, 1000, "k=1000"),
        (4000, 3000, 1, 1, "band"),
    ],
)
def test_knn_search_rejects_bad_arguments_on_host(native, n, w, p, k, msg):
    idx = (ctypes.c_int64 * 4)()
    dist = (ctypes.c_float * 4)()
    buf = (ctypes.c_float * 16)()
    st, text = _status(native, lambda: native.lib.knn_search(buf, 1, buf, 1, n, w, p, k, idx, dist, None, None))
    assert st == 1, text  # DTW_ERR_INVALID_ARG
    assert msg.split("=")[0] in text


def test_single_op_calls_validate_on_host(native):
    buf = (ctypes.c_float * 16)()
    assert native.lib.dtw_envelope(buf, 1, 0, 1, buf, buf, None) == 1
    assert native.lib.lb_keogh(buf, 1, buf, buf, 16, 5, buf, None) == 1
    assert native.lib.lb_improved(buf, -1, buf, buf, buf, 16, 1, 1, buf, None) == 1
    assert native.lib.dtw_band(buf, buf, 1, 7, 16, 1, 1, math.inf, buf, None) == 1  # bad y_stride
    assert native.lib.dtw_band(buf, buf, 1, 0, 16, 1, 1, float("nan"), buf, None) == 1
    # empty inputs are a no-op success
    assert native.lib.dtw_envelope(buf, 0, 16, 1, buf, buf, None) == 0
    assert native.lib.lb_keogh(buf, 0, buf, buf, 16, 1, buf, None) == 0


def test_p_values_per_entry_point(native):
    # dtw_band (and dtw_band_noalloc) take p = 1, 2, 4 and DTW_P_INF (0); the
    # bounds and the cascade take p = 1, 2 only
    buf = (ctypes.c_float * 16)()
    idx = (ctypes.c_int64 * 4)()
    for p in (1, 2, 4, 0):
        assert native.lib.dtw_band(buf, buf, 0, 0, 16, 1, p, math.inf, buf, None) == 0, p  # N = 0: no work
        assert native.lib.dtw_band_noalloc(buf, buf, 0, 0, 16, 1, p, math.inf, buf, None) == 0, p
    for p in (3, 5, -1):
        assert native.lib.dtw_band(buf, buf, 0, 0, 16, 1, p, math.inf, buf, None) == 1, p
        assert native.lib.dtw_band_noalloc(buf, buf, 0, 0, 16, 1, p, math.inf, buf, None) == 1, p
    for p in (4, 0):
        st, text = _status(native, lambda: native.lib.knn_search(buf, 1, buf, 1, 16, 1, p, 1, idx, buf, None, None))
        assert st == 1 and "p=" in text, text
        assert native.lib.lb_keogh(buf, 1, buf, buf, 16, p, buf, None) == 1


def test_bad_mode_and_slack_rejected(native):
    buf = (ctypes.c_float * 16)()
    idx = (ctypes.c_int64 * 4)()
    for opt in (native.Options(7, 1e-6, 0), native.Options(0, -1.0, 0), native.Options(0, 1e-6, -3)):
        st = native.lib.knn_search_ex(buf, 1, buf, 1, 16, 1, 1, 1, ctypes.byref(opt), idx, buf, None, None)
        assert st == 1


def test_profile_api_without_gpu(native):
    native.profile_enable(True)
    native.profile_enable(False)
    prof = native.profile_read(reset=True)
    assert set(prof) == set(native.STAGE_NAMES)


def test_index_rejects_bad_arguments_on_host(native):
    h = ctypes.c_void_p()
    st, text = _status(native, lambda: native.lib.dtw_index_create(3, None, ctypes.byref(h)))
    assert st == 1 and "p=3" in text
    opt = native.Options(7, 1e-6, 0, 0)
    st, text = _status(native, lambda: native.lib.dtw_index_create(1, ctypes.byref(opt), ctypes.byref(h)))
    assert st == 1 and "mode" in text
    st, text = _status(native, lambda: native.lib.dtw_index_search(None, None, 0, None, None, None, 1, 0, None, None,
                                                                   None, None))
    assert st == 1 and "null" in text
    st, text = _status(native, lambda: native.lib.dtw_index_destroy(None))
    assert st == 0


def test_server_rejects_bad_arguments_on_host(native):
    h = ctypes.c_void_p()
    st, text = _status(native, lambda: native.lib.dtw_server_create(None, None, ctypes.byref(h)))
    assert st == 1 and "null" in text
    st, text = _status(native, lambda: native.lib.dtw_server_submit(None, None, 8, 1, 1, None, None, 0, None))
    assert st == 1 and "null" in text
    cnt = ctypes.c_int32()
    st, text = _status(native, lambda: native.lib.dtw_server_poll(None, None, 0, ctypes.byref(cnt), 0))
    assert st == 1
    assert native.lib.dtw_server_destroy(None) == 0
    t0 = native.lib.dtw_monotonic_ns()
    assert native.lib.dtw_monotonic_ns() >= t0 > 0


def test_header_compiles_as_c99_and_cxx(tmp_path):
    # the C ABI must be usable from plain C (no C++ types in the signatures)
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use_abi.c"
    src.write_text('#include "dtwknn.h"\n'
                   "int main(void) { dtw_stats s; dtw_options o; dtw_tuning t; (void)s; (void)o; (void)t;\n"
                   "  return DTW_P_INF + DTW_OK; }\n")
    inc = os.path.join(ROOT, "include")
    for cmd in ([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, "-fsyntax-only", str(src)],
                [shutil.which("g++") or "g++", "-std=c++17", "-Wall", "-Werror", "-I", inc, "-fsyntax-only",
                 "-x", "c++", str(src)]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_shard_entry_points_validate_on_host(native):
    # candidate sharding: the threshold export / bounded search / merge calls
    # reject bad arguments before any device work
    buf = (ctypes.c_float * 16)()
    idx = (ctypes.c_int64 * 16)()
    lib = native.lib
    # merge: R, k_in, k out of range; host buffers refused; no queries is no work
    assert _status(native, lambda: lib.knn_merge_topk(idx, buf, 0, 1, 1, 1, idx, buf, None))[0] == 1
    assert _status(native, lambda: lib.knn_merge_topk(idx, buf, 2, 1, 0, 1, idx, buf, None))[0] == 1
    st, text = _status(native, lambda: lib.knn_merge_topk(idx, buf, 2, 1, 4, 1000, idx, buf, None))
    assert st == 1 and "k=1000" in text
    st, text = _status(native, lambda: lib.knn_merge_topk(idx, buf, 2, 1, 4, 4, idx, buf, None))
    assert st == 1 and "device" in text
    assert lib.knn_merge_topk(idx, buf, 2, 0, 4, 4, idx, buf, None) == 0
    # thresholds out: the usual argument checks, and an output buffer
    st, text = _status(native, lambda: lib.knn_seed_thresholds(buf, 1, buf, 1, 16, 1, 3, 1, None, buf, None))
    assert st == 1 and "p=3" in text
    st, text = _status(native, lambda: lib.knn_seed_thresholds(buf, 1, buf, 1, 16, 1, 1, 1, None, None, None))
    assert st == 1 and "null" in text
    assert lib.knn_seed_thresholds(buf, 1, buf, 0, 16, 1, 1, 1, None, buf, None) == 0  # Q = 0
    # bounded search: a threshold array is required when there are queries
    st, text = _status(native, lambda: lib.knn_search_bounded(buf, 1, buf, 1, 16, 1, 1, 1, None, None, idx, buf,
                                                              None, None))
    assert st == 1 and "null" in text
    st, text = _status(native, lambda: lib.knn_search_bounded(buf, 1, buf, 1, 16, 1, 1, 0, None, buf, idx, buf,
                                                              None, None))
    assert st == 1 and "k=0" in text
