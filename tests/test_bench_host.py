"""Host-side contract of bench.py, without a GPU: the oracle (reference)
arm's JSON line, the workload configs both arms share, the multi-rank
value, the clock-record parser and the variant operation count."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["config"] == bench.video_config(600, 16)
    assert line["value"] > 0 and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_names_workloads_it_does_not_cover():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "sweep", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_workload_configs():
    c = bench.video_config(600, 16)
    assert c["workload"] == "video_yuv420_600x3840x2160_r16"
    assert c["samples_per_step"] == 600 * 12_441_600 == 7_464_960_000
    assert "larger than L2" in c["l2"] and "1800 planes" in c["launch"]
    small = bench.video_config(1, 16)
    assert small["samples_per_step"] == 12_441_600
    from paper_1402_6034_gb300 import synth
    planes = synth.video_yuv420(1, 2160, 3840, seed=0, device="cpu")  # what the GPU arm allocates per frame
    assert sum(p.numel() for p in planes) == small["samples_per_step"]
    b = bench.batch512_config(10)
    assert b["samples_per_step"] == 1024 * 512 * 512 and b["workload"] == "batch_1024x512x512_r10"


def test_weak_scaling_value():
    # two ranks, each 7.46e9 samples per step, 10 steps, slowest rank 25 ms -> whole-job Gsamples/s
    v = bench.weak_scaling_value(7_464_960_000, 10, 25.0, 2)
    assert v == pytest.approx(2 * 7.46496e9 * 10 / 0.025 / 1e9)


def test_clock_summary_flags_throttle_reasons():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = None
    s.lines = [
        (10.0, "2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active"),
        (10.2, "2070, 2070, 1000.0, 0x4, Not Active, Not Active, Not Active, Active"),
        (10.4, "1800, 2070, 1100.0, 0x8, Active, Not Active, Not Active, Not Active"),
        (99.0, "300, 2070, 90.0, 0x0, Not Active, Not Active, Not Active, Not Active"),  # outside the window
    ]
    r = s.summary(9.9, 10.5)
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]
    empty = s.summary(50.0, 51.0)  # no sample inside: the nearest ones are reported and labelled
    assert "nearest" in empty["note"]


def test_variant_ops_per_block_hand_count():
    # r = 10 ends on anti-diagonal 3: K = 4 kept columns, a zone of 10 coefficients
    assert bench.variant_ops_per_block(10) == 8 * 4 * 8 + 10 * 8 + 8 * 10 + 64 * 4 + 128
    assert bench.variant_ops_per_block(10) / 64.0 == 12.5
    # r = 64: every column and the whole block
    assert bench.variant_ops_per_block(64) == 8 * 8 * 8 + 64 * 8 + 8 * 64 + 64 * 8 + 128
