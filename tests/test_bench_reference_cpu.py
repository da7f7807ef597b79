"""The benchmark's reference arm (the oracle timed on the host cores) keeps
the line contract: one JSON line with the metric, unit, value and the
cpu_baseline / e2e objects.  CPU only, on the small 2D Stokes workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(workload, extra=()):
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--steps", "1",
           "--warmup", "1", *extra]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


def test_reference_line_contract():
    d = run_reference("stokes2d_32", ["--ref-iters", "5"])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_bench_workloads_build_on_the_host():
    # every named workload's generator and settings are consistent (no GPU needed)
    sys.path.insert(0, ROOT)
    import bench

    for name, wl in bench.WORKLOADS.items():
        assert {"make", "levels", "max_coarse", "restart", "prec", "desc"} <= set(wl), name
        assert wl["prec"] in (32, 64) and wl["restart"] > 0 and wl["levels"] >= 1
        if wl.get("coarse_prec") == 32:
            assert wl["prec"] == 32, name
