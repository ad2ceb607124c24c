"""bench.py as the full test run calls it (--steps 20 --warmup 5), with the
long secondary legs switched off: it must exit 0 and print one JSON line with
every key the benchmark contract asks for, an RSR step inside the timed
window, and the roofline, end-to-end, clock and oracle-baseline fields."""
import json
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

ROOT = Path(__file__).resolve().parents[1]


def test_bench_line_at_twenty_steps():
    cmd = [sys.executable, str(ROOT / "bench.py"), "--gpus", "1", "--steps", "20", "--warmup", "5",
           "--no-mixed", "--no-batched", "--no-reindex", "--no-next-rows", "--no-ceiling", "--no-secondary",
           "--cpu-seconds", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches",
              "p10_ms", "p50_ms", "p90_ms"):
        assert k in d, k
    assert d["steps"] == 20 and d["warmup"] == 5 and d["n_gpus"] == 1 and d["gpu_launches"] == 20
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["rsr_steps_timed"], "no RSR step inside the timed window"
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0 < rf["frac"] < 1.5
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["d2h_bytes_per_step"] == 8 and e["h2d_bytes_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    v = d["visibility_vs_oracle"]
    assert v["differing_beyond_1e-6"] == 0
