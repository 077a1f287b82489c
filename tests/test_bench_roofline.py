"""bench.py's roofline arithmetic on CPU: the dominant launch's roofline and
the whole-step chain roofline, on a hand-made launch report with numbers
whose expected results are worked out below by hand."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2000.0}

# three steps' worth of launches, as codec.profile_report() returns them
REP = [
    # FP32 conv on the 3xTF32 tensor path: 2 launches, 1.2e12 FLOP, 1.2e9 bytes
    {"name": "g_a.conv1+gdn1:tc", "launches": 2, "ms": 4.0, "flop": 1.2e12, "bytes": 1.2e9},
    # memory-bound layout kernel: 3 launches, 6e9 bytes
    {"name": "patch_pack", "launches": 3, "ms": 1.5, "flop": 0.0, "bytes": 6.0e9},
    # a BF16 conv: 1.8e12 FLOP, 0.6e9 bytes
    {"name": "g_a.conv2+gdn2:bf16", "launches": 3, "ms": 3.0, "flop": 1.8e12, "bytes": 0.6e9},
]


def test_dominant_launch_roofline():
    r = bench.roofline(REP, PEAKS)
    assert r["kernel"] == "g_a.conv1+gdn1:tc"   # the largest total time
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    # TF32 peak = BF16 x 1.1 / 2.25 = 880 TFLOP/s; per launch 0.6e12 FLOP in 2 ms = 300 TFLOP/s
    assert r["peak"] == pytest.approx(880.0)
    assert r["achieved"] == pytest.approx(300.0)
    assert r["frac"] == pytest.approx(300.0 / 880.0)
    assert r["ceiling_3xtf32"] == pytest.approx(880.0 / 3)
    assert r["launch_ms"] == pytest.approx(2.0)


def test_chain_roofline():
    c = bench.chain_roofline(REP, PEAKS, measured_ms=10.0, steps=3)
    # conv1: compute 1.2e12 / (880e12 / 3) = 4.0909 ms, memory 1.2e9 / 6e12 = 0.2 ms -> 4.0909
    # patch_pack: no FLOP; memory 6e9 / 6e12 = 1.0 ms
    # conv2 (bf16): compute 1.8e12 / 1800e12 = 1.0 ms, memory 0.6e9 / 6e12 = 0.1 ms -> 1.0
    t_conv1 = 1.2e12 / (880e12 / 3) * 1e3
    roof = (t_conv1 + 1.0 + 1.0) / 3   # per step
    assert c["t_roof_ms"] == pytest.approx(roof)
    assert c["frac"] == pytest.approx(roof / 10.0)
    # compute and HBM sums over every launch, per step
    # (the layout kernel's FLOP time counts against the CUDA-core peak and is zero)
    assert c["t_compute_ms"] == pytest.approx((t_conv1 + 1.0) / 3)
    assert c["t_hbm_ms"] == pytest.approx((0.2 + 1.0 + 0.1) / 3)
    assert c["t_io_floor_ms"] is None
    # the I/O floor: bytes of one step over the measured HBM bandwidth
    c = bench.chain_roofline(REP, PEAKS, measured_ms=10.0, steps=3, floor_bytes=6e9)
    assert c["t_io_floor_ms"] == pytest.approx(1.0)


def test_e4m3_peak_is_twice_bf16():
    rep = [{"name": "g_s.deconv2.p0+igdn2:e4m3", "launches": 1, "ms": 1.0, "flop": 1.8e12, "bytes": 0.0}]
    r = bench.roofline(rep, PEAKS)
    assert r["peak"] == pytest.approx(3600.0) and r["achieved"] == pytest.approx(1800.0)
    c = bench.chain_roofline(rep, PEAKS, measured_ms=1.0, steps=1)
    assert c["t_roof_ms"] == pytest.approx(0.5)
