"""Host logic of the Gauss-Jordan panel's FP32 pivot choice, on the CPU: the
order of gj_pivot_key (sign-cleared magnitude bits) reduced as the register
panel reduces it must pick the same pivot as a float comparison, signed
zeros, denormals, infinities and ties included (tests/cpp/gj_pivot_key_test.cu,
compiled as host code by nvcc and run; it makes no CUDA call)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_pivot_key_order(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "gj_pivot_key_test")
    src = os.path.join(ROOT, "tests", "cpp", "gj_pivot_key_test.cu")
    csrc = os.path.join(ROOT, "paper_1604_00617_gb300", "csrc")
    cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", csrc, "-I", os.path.join(ROOT, "include"),
           src, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and "OK" in out.stdout, out.stdout + out.stderr
