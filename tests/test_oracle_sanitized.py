"""The oracle built with AddressSanitizer and UndefinedBehaviorSanitizer runs
every entry point on many sizes (tests/sanitize_oracle_driver.c) without a
report: no out-of-bounds access, leak or undefined operation."""

import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no host C compiler")
def test_oracle_under_address_and_undefined_behaviour_sanitizers():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "oracle_sanitized")
        cmd = ["gcc", "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
               "-fno-sanitize-recover=all", "-o", exe, os.path.join(ROOT, "oracle", "dtw_oracle.c"),
               os.path.join(ROOT, "tests", "sanitize_oracle_driver.c"), "-lm"]
        try:
            subprocess.run(cmd, check=True, capture_output=True, text=True)
        except subprocess.CalledProcessError as e:
            if "sanitize" in e.stderr and "not supported" in e.stderr:
                pytest.skip("sanitizers not supported by this compiler")
            raise
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300,
                           env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1"))
        assert r.returncode == 0, r.stderr[-4000:]
        assert "runtime error" not in r.stderr and "ERROR: AddressSanitizer" not in r.stderr, r.stderr[-4000:]
        assert r.stdout.startswith("ok")
