"""The host-side C and C++ code built with AddressSanitizer and
UndefinedBehaviorSanitizer and run on small exhaustive, periodic and seeded
cases.  The code is the oracle (oracle/oracle.c) and the library's DC3
construction (csrc/dc3_host.cpp).  The drivers are tests/sanitize/*.  The
device code has no such run: compute-sanitizer is closed on the GPU pool, so
its bounds are argued by reading and checked by the parity tests.  No GPU."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

SAN = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
CSRC = os.path.join(ROOT, "paper_1303_3692_gb300", "csrc")


def _build_and_run(tmp_path, compiler, name, args):
    cc = shutil.which(compiler)
    if cc is None:
        pytest.skip(f"{compiler} not installed")
    exe = str(tmp_path / name)
    r = subprocess.run([cc, *SAN, *args, "-o", exe], capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr or "ubsan" in r.stderr):
        pytest.skip("sanitizer runtime not available")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    return r.stdout


def test_oracle_under_sanitizers(tmp_path):
    out = _build_and_run(tmp_path, "gcc", "oracle_check",
                         ["-std=gnu11", "-pthread", os.path.join(ROOT, "oracle", "oracle.c"),
                          os.path.join(ROOT, "tests", "sanitize", "oracle_check.c")])
    assert "oracle checks passed" in out


def test_host_dc3_under_sanitizers(tmp_path):
    out = _build_and_run(tmp_path, "g++", "dc3_check",
                         ["-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                          os.path.join(CSRC, "dc3_host.cpp"), os.path.join(ROOT, "tests", "sanitize", "dc3_check.cpp")])
    assert "dc3 checks passed" in out
