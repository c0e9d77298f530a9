"""Host-side checks of the benchmark's bookkeeping: the DRAM traffic record
is used only for the kernel source it was taken from, its scaling to an
average launch, and the serving admission bound."""

import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _tree(tmp_path):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_1604_00617_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    shutil.copy(os.path.join(ROOT, "paper_1604_00617_gb300", "csrc", "k_tc.cu"), csrc / "k_tc.cu")
    return csrc / "k_tc.cu"


def test_committed_record_matches_current_kernel():
    rec = bench.traffic_record("gemm_tc")
    assert rec is not None, "profiles/traffic.json was taken from another k_tc.cu"
    assert rec["bytes_per_output_element"] > 0 and rec["blksz"] > 0


def test_record_dropped_when_kernel_changes(tmp_path):
    src = _tree(tmp_path)
    assert bench.traffic_record("gemm_tc", root=str(tmp_path)) is not None
    src.write_text(src.read_text() + "\n// changed\n")
    assert bench.traffic_record("gemm_tc", root=str(tmp_path)) is None


def test_missing_or_broken_record(tmp_path):
    _tree(tmp_path)
    (tmp_path / "profiles" / "traffic.json").write_text("not json")
    assert bench.traffic_record("gemm_tc", root=str(tmp_path)) is None
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({}))
    assert bench.traffic_record("gemm_tc", root=str(tmp_path)) is None


def test_scaled_traffic():
    rec = {"bytes_per_output_element": 10.0}
    b = 1024
    # three one-term b x b products in a launch: 3 b^2 output elements
    assert bench.scaled_traffic(rec, 3 * 2.0 * b ** 3, b) == pytest.approx(30.0 * b * b)
    assert bench.scaled_traffic(None, 1.0, b) is None


def test_peak_bytes_bounds_resident_bytes():
    from paper_1604_00617_gb300 import _lib as acr
    from paper_1604_00617_gb300 import serving
    import numpy as np
    prev = 0
    for n in (64, 128, 256):
        z = np.zeros(n * n)
        req = serving.SystemRequest(0, 0.0, n, n, z, np.zeros(3 * n * n), z, 1, 1e-6, 32)
        o = acr.acr_default_opts()
        o.precision = acr.ACR_FP32TC_IR
        o.input_kind = acr.ACR_BANDED
        pb = serving.peak_bytes(req, acr.ACR_FP32TC_IR)
        assert pb >= acr.acr_factor_bytes(n, n, 0.0, o)
        assert pb > prev
        prev = pb
