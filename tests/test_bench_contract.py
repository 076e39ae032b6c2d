"""bench.py on CPU: the reference arm's JSON line carries the keys the harness reads, and the
work model of the sweep counts what the design says."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "water",
                          "--steps", "1", "--warmup", "0", "--ref-time-cap", "5"], capture_output=True, text=True,
                         timeout=600, env={**os.environ, "RANK": "0", "WORLD_SIZE": "1"})
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith("water:")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                         capture_output=True, text=True, timeout=120,
                         env={**os.environ, "RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_sweep_work_model():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1106_2456_gb300 import workloads as wl

    # k = 2: three FMA-corrected 2 x 2 determinants (18) + C det, C z (2 + 4) + the scaling (3)
    assert bench.exc_flops(1) == 4.0 and bench.exc_flops(2) == 27.0
    assert all(bench.exc_flops(k + 1) > bench.exc_flops(k) for k in range(1, 8))
    p = wl.make_workload("water", n_walkers=2).problem
    f, b = bench.sweep_work(p, 0, 10, True, 400)
    f2, b2 = bench.sweep_work(p, 0, 20, True, 400)
    assert f2 == 2 * f and b2 > b and b2 < 2 * b + 1  # records are read once per launch
    assert np.isfinite(f) and f > 0


def test_traffic_record_is_dropped_when_the_kernel_changed(tmp_path, monkeypatch):
    """The roofline's measured DRAM traffic comes from profiles/traffic.json only while the sweep
    kernel's sources hash to the value recorded with the capture."""
    sys.path.insert(0, ROOT)
    import bench

    path = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(path))
    assert bench.profiled_traffic(True) is None
    rec = {"dram_bytes_per_walker": 250000.0, "walkers": 1024, "source_hash": bench.sweep_source_hash()}
    path.write_text(json.dumps({"k_ratio_mixed": rec}))
    got = bench.profiled_traffic(True)
    assert got["dram_bytes_per_walker"] == 250000.0 and got["walkers"] == 1024
    assert bench.profiled_traffic(False) is None
    path.write_text(json.dumps({"k_ratio_mixed": dict(rec, source_hash="0" * 16)}))
    assert bench.profiled_traffic(True) is None
