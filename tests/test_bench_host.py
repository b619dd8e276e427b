"""Host logic of bench.py that needs no GPU: the a * b^N fit of median
times (Table III) and the summary of sampled clocks and throttle reasons."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def bench():
    import bench

    return bench


def test_fit_exponential_recovers_a_and_b(bench):
    Ns = list(range(20, 41, 2))
    a, b = 3e-6, 1.27
    exact = bench.fit_exponential(Ns, [a * b**n for n in Ns])
    assert exact["a"] == pytest.approx(a, rel=1e-9) and exact["b"] == pytest.approx(b, rel=1e-12)
    rng = np.random.default_rng(0)
    noisy = [a * b**n * math.exp(rng.normal(0, 0.05)) for n in Ns]
    f = bench.fit_exponential(Ns, noisy)
    assert f["b_ci"][0] < b < f["b_ci"][1] and f["a_ci"][0] < a < f["a_ci"][1]
    # the same slope as an ordinary least-squares line through (N, log t)
    slope = np.polyfit(Ns, np.log(noisy), 1)[0]
    assert math.log(f["b"]) == pytest.approx(slope, rel=1e-9)
    assert (f["N_min_fit"], f["N_max_fit"]) == (20, 40)


def test_median_fit_skips_unreached_and_short_lists(bench):
    rows = [{"N": n, "p50_s": 2.0**n if n != 30 else float("inf"), "p50_steps": 3.0**n} for n in (28, 29, 30, 31)]
    f = bench.median_fit(rows)
    assert f["b"] == pytest.approx(2.0) and f["N_max_fit"] == 31
    assert bench.median_fit(rows, "p50_steps")["b"] == pytest.approx(3.0)
    assert bench.median_fit(rows[:2]) is None


def test_clock_summary_from_samples(bench, tmp_path):
    s = bench.ClockSampler("00000000:01:00.0")
    s.proc = object()  # sampled already: only the file is read
    s.path = str(tmp_path / "clocks.csv")
    lines = [
        "0, 00000000:01:00.0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 00000000:01:00.0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 00000000:01:00.0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, 00000000:02:00.0, 1000, 2070, 500.0, 0x8, Active, Not Active, Not Active, Not Active",
    ]
    open(s.path, "w").write("\n".join(lines) + "\n")
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]  # the other GPU's slowdown is not ours


def test_kernel_hash_ignores_comments_not_code(bench, tmp_path, monkeypatch):
    """The DRAM traffic record is keyed by this hash: a comment edit keeps
    it, any change of code orphans it (the bench line then reports null)."""
    import os
    import shutil

    src = os.path.join(bench.ROOT, "paper_2504_00987_gb300", "csrc")
    dst = tmp_path / "paper_2504_00987_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.kernel_hash()
    core = dst / "tabu_core.cuh"
    text = core.read_text()
    core.write_text("// a new comment line\n" + text.replace("#pragma once", "/* block\n comment */ #pragma once", 1))
    assert bench.kernel_hash() == base
    core.write_text(text.replace("kRecompute = NW <= 4", "kRecompute = NW <= 3", 1))
    assert bench.kernel_hash() != base


def test_traffic_record_matches_the_kernel(bench):
    """profiles/ holds the DRAM traffic of the current MTS kernel."""
    import json

    rec = json.load(open(bench.TRAFFIC_FILE))
    assert rec["kernel_hash"] == bench.kernel_hash()
    assert 0 < rec["bytes_per_launch"] < 1 << 20
