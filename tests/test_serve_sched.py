"""The service's scheduling policy (paper_1809_10585_gb300/csrc/serve_sched.h) on the CPU: a
small C++ driver is compiled with the host compiler and run; its fake device work records
what was started, so admission order, deferral of solves, slot reuse, the memory budget with
LRU eviction and the failure codes are checked without a GPU."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_scheduling_policy():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = os.path.join(ROOT, "tests", "native", "test_serve_sched.cpp")
    inc = os.path.join(ROOT, "paper_1809_10585_gb300", "csrc")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "test_serve_sched")
        r = subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-I" + inc, src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "all checks passed" in r.stdout
