"""The benchmark's JSON line keeps its contract: one line on stdout with the metric, the value,
the timing keys, the end-to-end measurement through host buffers, the launch count, the clock
record and the roofline object (a small run: 2^20 blocks, three timed steps)."""
import json
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]


def test_bench_line_has_the_contract_keys(aes_lib_ready):
    cmd = [sys.executable, str(ROOT / "bench.py"), "--steps", "3", "--warmup", "3", "--nblocks", str(1 << 20),
           "--no-cpu-baseline", "--no-batched", "--no-served", "--no-cbc", "--no-followons"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "clocks", "roofline"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0 and d["higher_is_better"]
    assert d["unit"] == "GB/s" and d["scaling"] == "weak" and d["config"]["workload"]
    assert d["gpu_launches"] == 2 * d["steps"]  # one encryption and one decryption per step
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    r = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(r)
    assert r["bound"] == "alu" and r["unit"] == "GB/s" and 0 < r["frac"] < 1.5
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-9)
    assert r["traffic"] is None  # the committed traffic figure is for 2^26 blocks only
