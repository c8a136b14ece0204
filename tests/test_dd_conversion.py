"""The double-float -> double conversion of the CUDA path (mf_dd.cuh) checked on the host:
tests/dd_conversion_check.cu compiled by nvcc as a host program over normalised pairs across
the float range, powers of two with lo on either side, and the edge cases (not normalised,
subnormal lo, zero, inf, nan)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_dd_to_double_rounds_to_nearest(tmp_path):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    exe = tmp_path / "dd_check"
    src = os.path.join(ROOT, "tests", "dd_conversion_check.cu")
    inc = os.path.join(ROOT, "paper_2609_04534_gb300", "csrc")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", inc, "-o", str(exe), src], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
