"""Host-side arithmetic of the benchmark (no GPU): the paper's parameter set
(Sec. IV-A), the HBM fractions of the memory-bound stages, and the FP32 peak."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_paper_parameters_follow_sec_iv_a():
    # eps = 0.1 N^-0.26, dt_h = eps / sigma_v with sigma_v ~ 0.65, n = 4, R1 = 1.03 N^-1/3, R2 = 2 R1, a_err = 2^-8
    n = 1 << 20
    p = bench.paper_params(n)
    assert p["eps"] == pytest.approx(0.1 * 2.0 ** (-20 * 0.26), rel=1e-15)
    assert p["dt_h"] == pytest.approx(p["eps"] / 0.65, rel=1e-15)
    assert p["R1"] == pytest.approx(1.03 / 2.0 ** (20 / 3), rel=1e-14)
    assert p["R2"] == 2 * p["R1"] and p["n_hard"] == 4 and p["a_err"] == 2.0 ** -8
    # the split radius is a few softening lengths at the paper's sizes (256k to 4096k)
    for n in (1 << 18, 1 << 22):
        q = bench.paper_params(n)
        assert 3.0 < q["R1"] / q["eps"] < 6.0


def test_hbm_stage_fractions():
    # 2^24 particles, 8 builds per soft step taking 14.8 ms in all: 96 B per particle per build (sample sort)
    out = bench.hbm_stages(1 << 24, 8, {"sort": 14.8, "kick_drift": 6.75})
    gbs = (1 << 24) * 96 * 8 / 14.8e-3 / 1e9
    assert out["sort"]["GB/s"] == pytest.approx(gbs)
    assert out["sort"]["frac_of_measured_hbm"] == pytest.approx(gbs / float(bench.measured_peaks().get("hbm_gbs", 6655.6)))
    assert out["kick_drift"]["bytes_per_particle"] == 108 and out["kick_drift"]["bytes_per_node"] == 0
    assert "topology" not in out and bench.hbm_stages(10, 1, {}) == {}
    # with the node count: topology 8 B per particle + 24 B per node, moments 32 B per particle + 96 B per node
    out = bench.hbm_stages(1000, 2, {"topology": 1.0, "moments": 2.0}, nodes=300)
    assert out["topology"]["bytes_per_launch"] == 1000 * 8 + 300 * 24
    assert out["moments"]["bytes_per_launch"] == 1000 * 32 + 300 * 96
    assert out["moments"]["GB/s"] == pytest.approx((1000 * 32 + 300 * 96) * 2 / 2e-3 / 1e9)


def test_fp32_peak():
    # 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz
    assert bench.fp32_peak_tflops(152, 2070.0) == pytest.approx(80.54784)
