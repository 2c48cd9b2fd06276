"""Host-side arithmetic of bench.py (no GPU): the tensor-core synthesis
roofline and the guard on the recorded DRAM traffic."""
from __future__ import annotations

import pytest

import bench


def test_tc_roofline_of_the_default_job():
    """1024^2 pixels x 512 stations x 64 eigenvectors x 100 steps in 96.8 ms against
    a 1385.2 TFLOP/s tensor peak: the split GEMM's 3 x 8 P flops take 59.5 ms at
    peak, the 5.4e10 sincos pairs 24.1 ms at an SFU rate of 2.23e12 pairs/s, and the kernel's measured
    instructions per pair take their issue-slot time; frac is the larger of the first two over 96.8 ms."""
    P = 1048576 * 512 * 64 * 100
    pairs = 1048576 * 512 * 100
    r = bench.tc_roofline(8.0 * P, 96.8, pairs, {"bf16_tflops_sustained": 1385.2}, None, 2.23e12)
    t = r["t_roof_ms"]
    assert t["tensor_split"] == pytest.approx(3 * 8.0 * P / 1385.2e12 * 1e3)
    assert t["sfu_sincos"] == pytest.approx(pairs / 2.23e12 * 1e3)
    assert t["issue_slots"] == pytest.approx(bench.SYNTH_TC_INSTR_PER_PAIR * pairs / (148 * 4 * 32 * 2.032e9) * 1e3)
    assert r["frac"] == pytest.approx(t["tensor_split"] / 96.8)
    assert r["achieved"] == pytest.approx(3 * 8.0 * P / 96.8e-3 / 1e12)
    assert r["largest_bound"] == "tensor_split" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert 0.6 < r["frac"] < 0.63
    assert r["frac_issue"] == pytest.approx(t["issue_slots"] / 96.8)


def test_traffic_only_for_the_captured_workload(monkeypatch):
    """The recorded DRAM traffic is reported only while the kernel sources hash
    to those of the capture and the workload is the captured one."""
    import hashlib
    import os
    csrc = os.path.join(os.path.dirname(bench.__file__), "paper_2310_09200_b300", "csrc")
    now = {name: hashlib.sha256(open(os.path.join(csrc, name), "rb").read()).hexdigest()
           for name in bench.SYNTH_TC_TRAFFIC["sha256"]}
    rec = dict(bench.SYNTH_TC_TRAFFIC, sha256=now)
    monkeypatch.setattr(bench, "SYNTH_TC_TRAFFIC", rec)
    w = dict(rec["workload"])
    assert bench.synth_tc_traffic(w) == rec["bytes"]
    w["n_t"] = 10
    assert bench.synth_tc_traffic(w) is None
    stale = dict(rec, sha256={k: "0" * 64 for k in now})
    monkeypatch.setattr(bench, "SYNTH_TC_TRAFFIC", stale)
    assert bench.synth_tc_traffic(dict(rec["workload"])) is None


def test_eig_roofline_of_the_default_job():
    """512 stations, kp = 80, 100 steps: FP32 stage (16/3 n^3 + 12 n^2 kp flops per step)
    at the FP32 rate and two refinement passes of double-float products at half of it."""
    r = bench.eig_roofline(512, 80, 100, 50.0, 6.5e13)
    n, kp = 512, 80
    t32 = (16 / 3 * n ** 3 + 12 * n ** 2 * kp) * 100 / 6.5e13
    tdf = 2 * 12 * (6 * n ** 2 * kp + 20 * n * kp ** 2) * 100 / 3.25e13
    assert r["t_roof_ms"]["fp32_stage"] == pytest.approx(t32 * 1e3)
    assert r["t_roof_ms"]["df_refinement"] == pytest.approx(tdf * 1e3)
    assert r["frac"] == pytest.approx((t32 + tdf) / 50e-3)


def test_synth_shape_reader_never_raises():
    """The bench line's synthesis shape is optional: a failing read gives None."""
    def boom():
        raise RuntimeError("no handle")
    assert bench.synth_shape_of(boom) is None
    assert bench.synth_shape_of(lambda: {"stages": 3}) == {"stages": 3}
