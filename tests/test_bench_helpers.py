"""Host-side helpers of bench.py (no GPU)."""
import json

import bench


def test_tensor_roofline_uses_measured_peak(tmp_path):
    p = tmp_path / "peaks.json"
    p.write_text(json.dumps({"bf16_tflops": 2000.0}))
    r = bench.tensor_roofline(2.0 * 1000 ** 3, 1.0, str(p))  # 2e9 FLOP in 1 ms = 2 TFLOP/s
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 2.0) < 1e-9 and r["peak"] == 2000.0
    assert abs(r["frac"] - 1e-3) < 1e-12 and "measured" in r["peak_basis"]


def test_tensor_roofline_falls_back_without_peaks_file(tmp_path):
    r = bench.tensor_roofline(4.6e13, 230.0, str(tmp_path / "missing.json"))
    assert r["peak"] == 1900.0 and "fallback" in r["peak_basis"]
    assert abs(r["achieved"] - 200.0) < 1e-6
