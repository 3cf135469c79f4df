"""Host-side logic of bench.py that needs no GPU: the clock-record parsing that decides whether a
run is rejected, the traffic lookup keyed by the kernel sources, the per-operation byte table, the
argument checks and the reference arm's JSON line (the oracle on one frame per step)."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

import bench
from paper_2505_12425_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sampler(tmp_path, lines):
    s = bench.ClockSampler(0, str(tmp_path))
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = object()   # as if nvidia-smi had run
    return s


def test_clock_summary_reports_throttle_reasons(tmp_path):
    ok = "0, 2070, 2070, 180.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    hot = "0, 1800, 2070, 900.0, 0x40, Not Active, Active, Not Active, Not Active"
    cap = "0, 1950, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active"
    s = _sampler(tmp_path, [ok, hot, cap, ok])
    d = s.summary()
    assert d["samples"] == 4
    assert d["sm_max_mhz"] == 2070.0
    assert d["sm_mhz"] == pytest.approx((1950 + 2070) / 2)
    assert d["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert d["power_w_max"] == 1399.0


def test_clock_summary_without_samples(tmp_path):
    assert _sampler(tmp_path, ["garbage"]).summary() is None
    s = bench.ClockSampler(0, str(tmp_path))
    assert s.summary() is None   # nvidia-smi never ran


def test_traffic_is_null_once_the_kernels_change(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"per_op": {"warp_f32": {"dram_bytes_per_launch": 123456}}}
    (prof / "ncu_traffic.json").write_text(json.dumps(dict(entry, kernel_source_sha=bench.kernel_source_sha())))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the source hash is read from the package sources, not from ROOT's copy of them
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: json.loads((prof / "ncu_traffic.json").read_text())
                        ["kernel_source_sha"])
    assert bench.load_traffic("warp_f32") == 123456
    assert bench.load_traffic("warp_u8") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.load_traffic("warp_f32") is None


def test_kernel_source_sha_tracks_the_tile_engine():
    sha = bench.kernel_source_sha()
    assert len(sha) == 16 and int(sha, 16) >= 0
    assert bench.kernel_source_sha() == sha


def test_op_table_output_bytes():
    ops = {name: (px, ob) for name, px, ob in bench.op_table()}
    rs = bench.RS_H * bench.RS_W
    full = inputs.BENCH_H * inputs.BENCH_W
    assert ops["resize_u8"] == (rs, 3 * rs)
    assert ops["resize_gray_u8"] == (rs, rs)
    assert ops["resize_f32"] == (rs, 12 * rs) and ops["resize_norm_f32_chw"] == (rs, 12 * rs)
    assert ops["warp_u8"] == (full, 3 * full) and ops["warp_gray_u8"] == (full, full)
    assert ops["warp_f32"] == (full, 12 * full) and ops["rgb_to_gray"] == (full, full)
    assert sum(px for px, _ in ops.values()) * inputs.BENCH_IMAGES == 383385600


@pytest.mark.parametrize("argv", [["--warmup", "2"], ["--images", "0"], ["--images", "33"], ["--next-reps", "0"]])
def test_bench_rejects_bad_arguments(argv):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 2 and "error" in r.stderr


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "Gpixel/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_two_stream_step_issues_every_operation_once():
    """The two-stream step (the default) splits the step's operations between the streams: each
    of the eight operations exactly once, the u8 kinds on the first stream."""
    names = [n for n, _, _ in bench.op_table()]
    first, second = bench.Step.SPLIT
    assert all(n.endswith("_u8") for n in first)
    for k, split in bench.Step.SPLITS.items():
        assert len(split) == k
        flat = [n for part in split for n in part]
        assert sorted(flat) == sorted(names) and len(set(flat)) == len(names)
