"""The benchmark's roofline arithmetic on the host: the dominant kernel is the
one with the largest share of device time, its bound is the one the method's
roofline gives it (HBM for the frame pass and the upsampling step, FP32 for
the transforms, tensor cores for the direct form), `achieved` is its
algorithmic work per second over the live duration, `frac` divides by that
bound's peak with the other fractions beside it, and the DRAM traffic
constants are reported only for the workload and form they were captured on."""
import math

import pytest

import bench
from paper_1506_06039_gb300 import XCORR_DIRECT_BF16X3, XCORR_FFT_FP32, synth

PEAKS = {"hbm_gbs": 6787.2, "bf16_tflops": 1942.7, "bf16_tflops_sustained": 1714.2}
INFO_288 = {"mc": 256, "nc": 256, "fft_rows": 288, "fft_cols": 288, "xcorr": XCORR_FFT_FP32}
# measured ALU peaks as moco_alu_peak would report them (T ops/s, source)
ALU = {"fp32": (71.5, "measured"), "int": (19.0, "measured")}


def _rf(profile, info, name="std512", frames=2000, steps=300):
    return bench.roofline(profile, info, synth.WORKLOADS[name], frames, steps, PEAKS, ALU)


def test_jitter_dominant_is_hbm_bound_with_the_integer_pipe_beside_it():
    # ms summed over 300 launches, as the library's profile returns them
    prof = {"k_frame_rows": (300, 137.0), "k_cols": (300, 125.0), "k_rows_inv": (300, 52.0),
            "k_jitter": (300, 144.0)}
    rf = _rf(prof, INFO_288)
    assert rf["kernel"] == "k_jitter" and rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    assert rf["avg_launch_ms"] == pytest.approx(144.0 / 300)
    # every full-resolution pixel of 2000 frames of 512 x 512 read once
    byts = 2.0 * 512 * 512 * 2000
    assert rf["algorithmic_per_launch"]["bytes"] == pytest.approx(byts)
    achieved = byts / (144.0 / 300 / 1e3) / 1e9
    assert rf["achieved"] == pytest.approx(achieved)
    assert rf["peak"] == PEAKS["hbm_gbs"]
    assert rf["frac"] == pytest.approx(achieved / PEAKS["hbm_gbs"])
    # nine exact products per pixel, against the measured dp2a rate, beside it
    mads = 9.0 * 512 * 512 * 2000
    assert rf["algorithmic_per_launch"]["int_mads"] == pytest.approx(mads)
    assert rf["fractions"]["int"] == pytest.approx(mads / (144.0 / 300 / 1e3) / 1e12 / ALU["int"][0])
    assert rf["share"] == pytest.approx(144.0 / (137.0 + 125.0 + 52.0 + 144.0))
    # the captured traffic, scaled from 512 frames to a 2000-frame launch
    assert rf["traffic"] == pytest.approx(bench.TRAFFIC_PER_FRAME["k_jitter"] * 2000)


def test_frame_pass_dominant_is_hbm_bound_with_its_algorithmic_bytes():
    prof = {"k_frame_rows": (10, 5.0), "k_cols": (10, 1.0)}
    rf = _rf(prof, INFO_288, frames=2000, steps=10)
    assert rf["kernel"] == "k_frame_rows" and rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    per_frame = 2 * 512 * 512 + 8 * (288 // 2 + 1) * 256  # frame in, row spectra out
    assert per_frame == 821248
    assert rf["algorithmic_per_launch"]["bytes"] == pytest.approx(per_frame * 2000)
    assert rf["achieved"] == pytest.approx(per_frame * 2000 / 0.5e-3 / 1e9)
    assert rf["frac"] == pytest.approx(rf["achieved"] / PEAKS["hbm_gbs"])


def test_traffic_only_for_the_captured_workload_and_form():
    prof = {"k_jitter": (1, 1.0)}
    assert _rf(prof, INFO_288)["traffic"] is not None
    direct = dict(INFO_288, xcorr=XCORR_DIRECT_BF16X3)
    assert _rf(prof, direct)["traffic"] is None
    assert _rf(prof, INFO_288, name="large512")["traffic"] is None
    assert _rf(prof, INFO_288, name="tiny128")["traffic"] is None


def test_direct_form_kernel_takes_the_sustained_bf16_peak():
    prof = {"k_direct": (20, 112.0), "k_jitter": (20, 9.6)}
    info = dict(INFO_288, xcorr=XCORR_DIRECT_BF16X3)
    rf = _rf(prof, info, frames=2000, steps=20)
    assert rf["kernel"] == "k_direct" and rf["bound"] == "tensor" and rf["unit"] == "TFLOP/s"
    W = 63
    flops = 3 * 2.0 * W * W * 256 * 256 * 2000
    assert rf["achieved"] == pytest.approx(flops / (112.0 / 20 / 1e3) / 1e12)
    assert rf["peak"] == PEAKS["bf16_tflops_sustained"]
    assert math.isclose(rf["frac"], rf["achieved"] / rf["peak"])


def test_transform_kernel_is_reported_against_the_measured_fp32_peak():
    prof = {"k_cols": (10, 4.0), "k_jitter": (10, 1.0)}
    rf = _rf(prof, INFO_288, frames=2000, steps=10)
    assert rf["kernel"] == "k_cols" and rf["bound"] == "alu" and rf["unit"] == "TFLOP/s"
    N = 288
    flops = (N // 2 + 1) * (2 * 5.0 * N * math.log2(N) + 6 * N) * 2000
    assert rf["achieved"] == pytest.approx(flops / 0.4e-3 / 1e12)
    assert rf["peak"] == ALU["fp32"][0]
    assert rf["frac"] == pytest.approx(rf["achieved"] / ALU["fp32"][0])
