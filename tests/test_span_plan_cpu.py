"""Host-side check of the staged kernels' bulk-copy plans (csrc/nasg_span.h):
alignment, buffer bounds, coverage and destination capacity of every tile's
copies over a sweep of N, L and element sizes (tests/span_plan_check.cpp,
compiled here with the host compiler; no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_09794_gb300", "csrc")


def test_span_plans(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "span_plan_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "span_plan_check.cpp"),
                    "-o", exe], check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert res.stdout.startswith("ok ")
