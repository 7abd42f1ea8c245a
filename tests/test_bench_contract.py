"""The benchmark's host-side contract, without a GPU: the reference arm (the
kd-tree CPU oracle timed on the workload) prints one well-formed JSON line, and
the byte models of the streaming-phase rooflines are the documented ones."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c2",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    res = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in res, key
    assert res["impl"] == "reference" and res["value"] > 0 and res["unit"] == "points/s"
    assert res["cpu_baseline"]["kind"] == "oracle" and res["cpu_baseline"]["cores"] >= 1
    assert res["cpu_baseline"]["value"] == res["value"]
    assert res["e2e"]["h2d_bytes_per_step"] == 0 and res["e2e"]["d2h_bytes_per_step"] == 0
    assert res["config"]["workload"].startswith("c2_")
    assert 1 <= res["steps"] <= 2 and res["steps_requested"] == 2


def test_phase_roofline_byte_model():
    import bench

    class Job:
        sizes, dims, n_dcut, N = [1000], [3], 2, 1000
    out = bench.phase_rooflines(Job(), {"bits_per_axis": 15}, {"bin": 1.0, "labels": 0.5}, 1000.0, "measured")
    # 3-D: 12*3 + 48 + 24 * ceil(45 / 8) + 4 * 4 bytes per point; labels 20 per cutoff
    assert out["bin"]["bytes_per_point"] == 36 + 48 + 24 * 6 + 16
    assert out["bin"]["passes"] == 6
    assert out["labels"]["bytes_per_point"] == 40
    assert out["bin"]["achieved"] == pytest.approx(244 * 1000 / 1e-3 / 1e9)
    assert out["labels"]["frac"] == pytest.approx(out["labels"]["achieved"] / 1000.0)

    class Batch:
        sizes, dims, n_dcut, N = [10, 20], [2, 3], 1, 30
    assert bench.phase_rooflines(Batch(), {}, {"bin": 1.0}, 1000.0, "measured") is None
