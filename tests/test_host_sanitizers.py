"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU): the pass planner
(csrc/plan.cpp, every plan the library can ask for) and the oracle (every entry point on small
graphs) are compiled with -fsanitize=address,undefined and run through the drivers in
tests/native/, which also check the plans' and the oracle's consistency.  An out-of-bounds access,
a leak or undefined behaviour fails the test with the sanitizer's report."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NATIVE = os.path.join(ROOT, "tests", "native")
CSRC = os.path.join(ROOT, "paper_2312_03019_b300", "csrc")
SAN = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def _run(cmd, exe):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and "unrecognized" in r.stderr:
        pytest.skip("compiler without sanitizer support")
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-3000:])
    assert "0 failures" in r.stdout
    return r.stdout


def test_planner_under_sanitizers(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "plan_check")
    out = _run(["g++", "-std=c++17", *SAN, "-I", CSRC, os.path.join(NATIVE, "plan_check.cpp"),
                os.path.join(CSRC, "plan.cpp"), "-o", exe], exe)
    assert int(out.split()[0]) > 1000


def test_oracle_under_sanitizers(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "oracle_check")
    out = _run(["gcc", "-std=c11", *SAN, os.path.join(NATIVE, "oracle_check.c"),
                os.path.join(ROOT, "oracle", "qaoa_oracle.c"), "-o", exe, "-lm"], exe)
    assert int(out.split()[0]) > 50
