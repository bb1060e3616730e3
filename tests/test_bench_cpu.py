"""The benchmark script's CPU side: the reference arm's JSON line and the
roofline arithmetic it reports against (no GPU needed)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_peak_is_the_shared_memory_term():
    # 152 SMs x 2070 MHz x 128 B/clk / 16 B per edge-update.
    assert bench.roofline_peak_edge_updates(152, 2070.0) == pytest.approx(2.51712e12, rel=1e-9)
    # The ALU term (10 lane-ops per edge-update against 128 lanes/clk) is looser.
    assert bench.roofline_peak_edge_updates(1, 1000.0) == pytest.approx(1e9 * 128 / 16)


def test_dram_traffic_per_shot_is_below_the_shots_io():
    # 12 B of packed syndrome in and 24 B of results out per shot of [[144]].
    assert 0 < bench.DRAM_BYTES_PER_SHOT < 12 + 24


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-shots", "100"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "shots/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["sample_shots_per_p"] == 100
