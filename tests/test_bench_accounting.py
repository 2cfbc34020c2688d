"""The bench's roofline arithmetic against hand-computed values (no GPU).

The algorithmic bytes of a launch are the samples the frames need, read once,
plus the features, written once (FP32); achieved = bytes / launch time, and
frac = achieved / the measured copy bandwidth.  The FP32 form is held to the
ALU peak derived from 152 SMs x 128 FP32 lanes x 2 FLOP x the SM clock.
"""
import types

import numpy as np
import pytest

import bench


def _w(n_clips=64, length=480000):
    return types.SimpleNamespace(lens=np.full(n_clips, length, dtype=np.int64), name="rich_64x30s")


CFG = dict(sr=16000.0, n_fft=400, hop=160, n_mels=80, fmin=0.0, fmax=8000.0)


def test_frames_and_algorithmic_bytes_of_the_64x30s_batch():
    W = _w()
    assert bench.frames_of(W.lens, 400, 160) == 64 * 2998 == 191872
    # a 30 s clip's 2998 frames need samples [0, 2997*160 + 400): 479,920 floats
    per_clip = 4 * (2997 * 160 + 400) + 4 * 2998 * 80
    assert bench.algorithmic_bytes(W.lens, 400, 160, 80) == 64 * per_clip == 184258560
    # clips shorter than a frame move nothing; a clip of exactly N moves N samples
    assert bench.algorithmic_bytes([399, 400], 400, 160, 80) == 4 * 400 + 4 * 80


def test_hbm_roofline_of_a_bf16_launch(monkeypatch):
    monkeypatch.setattr(bench, "measured_traffic", lambda key: None)
    W = _w()
    r = {"precision": "bf16", "T": 191872, "n_out": 80, "launch_ms": 0.040}
    peaks = {"hbm_gbs": 6789.6, "bf16_tflops": 1894.0}
    out = bench.roofline(CFG, W, r, peaks, "measured")
    assert out["bound"] == "hbm" and out["unit"] == "GB/s"
    assert out["achieved"] == pytest.approx(184258560 / 40e-6 / 1e9)
    assert out["frac"] == pytest.approx(184258560 / 40e-6 / 1e9 / 6789.6)
    assert out["traffic_key"] == "bf16/rich_64x30s/n_mels=80/n_out=80"
    flops = 2 * 400 * 160 * 191872
    assert out["tensor_tflops"] == pytest.approx(flops / 40e-6 / 1e12)
    assert out["tensor_frac_of_bf16_peak"] == pytest.approx(flops / 40e-6 / 1e12 / 1894.0)


def test_split_bf16_counts_three_products(monkeypatch):
    monkeypatch.setattr(bench, "measured_traffic", lambda key: None)
    r = {"precision": "bf16x3", "T": 191872, "n_out": 80, "launch_ms": 0.1}
    out = bench.roofline(CFG, _w(), r, {"hbm_gbs": 6789.6, "bf16_tflops": 1894.0}, "measured")
    assert out["tensor_tflops"] == pytest.approx(3 * 2 * 400 * 160 * 191872 / 1e-4 / 1e12)


def test_fp32_alu_roofline():
    r = {"precision": "fp32", "T": 191872, "n_out": 80, "launch_ms": 0.885}
    out = bench.roofline(CFG, _w(), r, {"hbm_gbs": 6789.6, "sm_max_mhz": 2070.0}, "measured")
    peak = 152 * 128 * 2 * 2070e6 / 1e12  # 80.5 TFLOP/s
    assert out["bound"] == "alu" and out["peak"] == pytest.approx(peak)
    assert out["frac"] == pytest.approx(2 * 400 * 160 * 191872 / 0.885e-3 / 1e12 / peak)


def test_clock_and_power_sample_parsing():
    text = "\n".join([
        "0, 2070, 2070, 612.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 905.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, [N/A], 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    ck = bench.ClockSampler.parse(text)
    assert ck["samples"] == 3 and ck["sm_mhz"] == 2070.0 and ck["sm_max_mhz"] == 2070.0
    assert ck["reasons"] == ["sw_power_cap"]
    assert ck["power_w_median"] == pytest.approx((612.5 + 905.0) / 2)


def test_energy_estimate():
    r = {"T": 191872, "launch_ms": 0.041, "clocks": {"power_w_median": 800.0, "samples": 9}}
    e = bench.energy_estimate(r)
    assert e["joules_per_frame"] == pytest.approx(800.0 * 41e-6 / 191872)
    assert e["frames_per_joule"] == pytest.approx(191872 / (800.0 * 41e-6))
    assert bench.energy_estimate({"T": 5, "launch_ms": 1.0, "clocks": {"power_w_median": None}}) is None


def test_energy_estimate_degenerate_inputs():
    assert bench.energy_estimate({"T": 5, "launch_ms": 0.0, "clocks": {"power_w_median": 500.0}}) is None
    assert bench.energy_estimate({"T": 0, "launch_ms": 1.0, "clocks": {"power_w_median": 500.0}}) is None
    assert bench.energy_estimate({"T": 5, "launch_ms": 1.0}) is None
