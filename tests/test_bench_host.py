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


def _stats(sweep_ms, gemm_ms):
    return {"gemm_flops": 2.0 * 1024 ** 3 * 100, "gemm_launches": 10, "gemm_ms": gemm_ms,
            "sweep_bytes": 2.0e9 * 21, "sweep_ms": sweep_ms, "sweep_passes": 21}


def test_roofline_reports_the_larger_class():
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops_sustained": 1700.0}
    clocks = {"sm_max_mhz": 2070.0}
    main, key, other = bench.rooflines(_stats(47.0, 9.3), "fp32tc", peaks, clocks, 170.0, 1024)
    assert main["bound"] == "hbm" and key == "roofline_products" and other["bound"] == "tensor"
    # 2 GB per application in 47 / 21 ms
    assert main["achieved"] == pytest.approx(2.0e9 * 21 / 47e-3 / 1e9)
    assert main["frac"] == pytest.approx(main["achieved"] / 6800.0)
    assert main["applications"] == 21 and main["application_ms"] == pytest.approx(47.0 / 21)
    assert other["peak"] == pytest.approx(850.0) and other["frac"] == pytest.approx(170.0 / 850.0)
    assert other["tensor_pipe_3xtf32"]["frac"] == pytest.approx(3 * 170.0 / 850.0)
    main2, key2, _ = bench.rooflines(_stats(5.0, 9.3), "fp32tc", peaks, clocks, 170.0, 1024)
    assert main2["bound"] == "tensor" and key2 == "roofline_sweep"


def test_roofline_fallback_peaks():
    main, _, other = bench.rooflines(_stats(47.0, 9.3), "fp32tc", None, {}, 170.0, 1024)
    assert main["peak"] == 6800.0 and "fallback" in main["peak_source"]
    assert "fallback" in other["peak_source"]
