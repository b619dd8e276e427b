"""bench.py's output line: both arms print one JSON object with the keys and
types of the benchmark contract (small sizes, so the test takes seconds)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_gpu_arm_line():
    d = run_bench("--steps", "3", "--warmup", "3", "--replicas", "304", "--steps-per-replica", "2000")
    for k, t in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                 ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                 ("dtype", str), ("data", str), ("config", dict), ("roofline", dict), ("e2e", dict),
                 ("gpu_launches", int), ("cpu_baseline", dict)):
        assert isinstance(d[k], t), k
    assert d["metric"] == d["unit"] == "flip-evals/s" and d["n_gpus"] == 1 and d["steps"] == 3
    assert d["vs_baseline"] is None and d["scaling"] == "weak" and d["higher_is_better"] is True
    assert "workload" in d["config"] and d["value"] > 0
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "Gop/s" and 0 < r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    e = d["e2e"]
    assert e["unit"] == d["unit"] and e["value"] > 0 and e["h2d_bytes_per_step"] > 0
    assert e["d2h_bytes_per_step"] == 304 * 64
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and c["sample"]
    assert d["gpu_launches"] == 3
    assert "clocks" in d
    # the other configurations, measured in the same run
    assert set(d["tts_p50_s"]) == set(d["tts_p99_s"]) == {str(n) for n in range(92, 121, 4)}
    b = d["batch_uneven_512"]
    assert b["ms_per_batch"] > 0 and b["flip_evals_per_s"] > 0 and b["speedup_vs_plain"] > 1
    s = d["serve_poisson"]
    assert 0 < s["latency_s"]["p50_cap_mode"] <= s["latency_s"]["p99_cap_mode"]
    assert s["plain_one_launch_per_request"]["requests"] == 200 and s["flip_evals_per_s"] > 0


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--steps-per-replica", "2000")
    assert d["impl"] == "reference" and d["metric"] == "flip-evals/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
