"""The roofline arithmetic of bench.py on synthetic stage statistics (no GPU): the transform class
that takes the most time is the headline entry, the others sit under "others", and every
fraction is the achieved rate (algorithmic flops or bytes over the stage time) over its peak."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

STAGES = ("near", "gen", "fft", "pointwise", "out", "fft_df64", "fft_fp32")


def _stats(**over):
    st = {k: {"ms": 0.0, "flops": 0.0, "entries": 0.0, "bytes": 0.0, "launches": 0} for k in STAGES}
    for k, v in over.items():
        st[k].update(v)
    return st


def test_fft_roofline_picks_the_longest_class_and_divides_by_its_peak():
    # two plans' statistics over 2 steps: FP64 transforms 10 ms, FP32 transforms 4 ms in all
    stats = [_stats(fft={"ms": 6.0, "flops": 6e9, "bytes": 3e9, "launches": 5},
                    fft_fp32={"ms": 1.0, "flops": 1e9, "bytes": 2e9, "launches": 3}),
             _stats(fft={"ms": 4.0, "flops": 4e9, "bytes": 2e9, "launches": 4},
                    fft_fp32={"ms": 3.0, "flops": 1e9, "bytes": 8e9, "launches": 3})]
    r = bench.fft_roofline(stats, 2)
    assert r["bound"] == "alu" and r["unit"] == "GFLOP/s"
    assert r["achieved"] == pytest.approx(10e9 / 0.010 / 1e9)  # 1000 GFLOP/s
    assert r["frac"] == pytest.approx(1000.0 / bench.FP64_PEAK_GFLOPS)
    assert r["frac_of_measured_fp64"] == pytest.approx(1000.0 / bench.FP64_MEASURED_GFLOPS)
    assert r["fft_ms_per_step"] == pytest.approx(5.0)
    assert r["launches"] == 9
    # DRAM bytes per launch: the capture's ratio times the algorithmic bytes of a launch
    assert r["traffic"] == pytest.approx(bench.FFT_TRAFFIC_RATIO * 5e9 / 9)
    fp32 = r["others"]["fp32_transforms"]
    peak, _ = bench.hbm_peak()
    assert fp32["bound"] == "hbm" and fp32["unit"] == "GB/s"
    assert fp32["achieved"] == pytest.approx(10e9 / 0.004 / 1e9)  # 2500 GB/s
    assert fp32["frac"] == pytest.approx(2500.0 / peak)
    assert "df64_transforms" not in r["others"]
    json.dumps(r)  # the entry goes into the JSON line as it is


def test_fp32_class_leads_when_it_takes_the_most_time():
    stats = [_stats(fft={"ms": 1.0, "flops": 1e9, "bytes": 1e9, "launches": 1},
                    fft_fp32={"ms": 2.0, "flops": 1e9, "bytes": 9e9, "launches": 2})]
    r = bench.fft_roofline(stats, 1)
    assert r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(4500.0)
    assert set(r["others"]) == {"fp64_transforms"}


def test_stage_hbm_reports_both_bounds_per_step():
    # segment sums: 8 flop per point and segment; row sums: 4 flop per column and row
    stats = [_stats(pointwise={"ms": 3.0, "flops": 3.0e9, "bytes": 6e9, "launches": 20},
                    out={"ms": 2.0, "flops": 1e9, "bytes": 8e9, "launches": 40}),
             _stats(pointwise={"ms": 3.0, "flops": 3.0e9, "bytes": 6e9, "launches": 20},
                    out={"ms": 2.0, "flops": 1e9, "bytes": 8e9, "launches": 40})]
    h = bench.stage_hbm(stats, 2)
    peak, _ = bench.hbm_peak()
    seg, out = h["pointwise"], h["out"]
    assert seg["ms_per_step"] == pytest.approx(3.0) and seg["launches"] == 20
    assert seg["achieved"] == pytest.approx(12e9 / 0.006 / 1e9)  # 2000 GB/s
    assert seg["frac"] == pytest.approx(2000.0 / peak)
    assert seg["gflops"] == pytest.approx(6e9 / 0.006 / 1e9)  # 1000 GFLOP/s
    assert seg["frac_of_fp64_peak"] == pytest.approx(1000.0 / bench.FP64_PEAK_GFLOPS)
    assert out["gbytes_per_step"] == pytest.approx(8.0)
    assert out["frac_of_measured_fp64"] == pytest.approx(500.0 / bench.FP64_MEASURED_GFLOPS)


def test_stage_without_time_reports_no_rate():
    h = bench.stage_hbm([_stats()], 1)
    assert h["out"]["achieved"] is None and h["out"]["frac"] is None and h["out"]["gflops"] is None
