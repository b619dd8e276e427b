#!/usr/bin/env python3
"""Throughput benchmark of the GB300 memetic tabu search (flip-evals/s).

One step = one launch of the whole hot path over the workload: N=64, K=100,
1,024 independent MTS replicas (Philox streams 0..1023), each running
exactly 10^5 tabu steps (every step scores all N one-bit-flip neighbours).
flip-evals = tabu steps x N; pair-terms = flip-evals x (N-1).

    python bench.py [--gpus G] [--steps S] [--warmup W] [--impl gpu|reference]

The same line carries the N = 92..120 configuration as extra keys: its
throughput per N and its time to target (p50/p99 per N over 50 seeds).

Under torchrun each rank runs its own 1,024 replicas (instances offset by
rank x 1,024; weak scaling, no collective on the data path); for time to
target the ranks share the stop flag between slices of generations.  Rank 0
prints one JSON line.  `--impl reference` times the CPU oracle (test
infrastructure) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_00987_gb300 import parallel  # noqa: E402  (host logic only; no CUDA at import)

N, K, REPLICAS, STEPS_PER_REPLICA = 64, 100, 1024, 100_000
WORKLOAD = "replicas_n64"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
SM_COUNT_GB300 = 152
INT32_LANES_PER_SM = 128  # 4 SM sub-partitions x 32 lanes
SM_MAX_MHZ_GB300 = 2070.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "mts_kernel_n64_traffic.json")
KERNEL_SOURCES = ["tabu_core.cuh", "tabu_skew.cuh", "replica.cuh", "mts_kernels.cuh", "mts.cu", "labs_device.cuh",
                  "kernels.h"]


def kernel_hash() -> str:
    """Hash of the code the MTS kernel is compiled from: comments and blank
    space are left out, so that an edit of a comment does not orphan the
    recorded DRAM traffic of an unchanged kernel."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2504_00987_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)  # block comments
        text = re.sub(r"//[^\n]*", " ", text)                # line comments
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def workload_config(extra: dict | None = None) -> dict:
    cfg = {
        "workload": f"{WORKLOAD}: N={N}, K={K}, {REPLICAS} replicas x {STEPS_PER_REPLICA} tabu steps",
        "N": N, "K": K, "replicas_per_gpu": REPLICAS, "steps_per_replica": STEPS_PER_REPLICA,
        "p_comb": 0.9, "p_mut": "1/N", "replace": "random", "seed": 0,
    }
    if extra:
        cfg.update(extra)
    return cfg


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi sampling (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile

            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict | None:
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.bus_id and self.bus_id not in parts[1].lower():
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle


def cpu_baseline_run(replicas: int, threads: int, steps: int, n: int | None = None) -> dict:
    import oracle

    n = N if n is None else n
    oracle.build()
    P = oracle.make_params(n, K, max_steps=steps)
    t0 = time.perf_counter()
    res = oracle.mts_run_many(P, 0, 0, replicas, threads)
    dt = time.perf_counter() - t0
    total = sum(r["steps"] for r in res) * n
    return {"value": total / dt, "unit": "flip-evals/s", "cores": threads, "kind": "oracle",
            "sample": f"{replicas} of the {REPLICAS} replicas (instances 0..{replicas - 1}), "
                      f"{steps} tabu steps each, one replica per thread, {dt:.1f} s wall"}


def apply_overrides(args) -> None:
    """--n, --replicas and --steps-per-replica resize the default workload (both arms)."""
    global N, WORKLOAD, REPLICAS, STEPS_PER_REPLICA
    if args.n:
        N, WORKLOAD = args.n, f"replicas_n{args.n}"
    if args.replicas:
        REPLICAS = args.replicas
    if args.steps_per_replica:
        STEPS_PER_REPLICA = args.steps_per_replica


def run_reference(args) -> None:
    world, rank, _ = dist_env()
    if rank != 0:
        return
    apply_overrides(args)
    cores = cpu_cores()
    for _ in range(args.warmup):
        cpu_baseline_run(cores, cores, STEPS_PER_REPLICA // 10)
    times, total = [], 0
    for _ in range(args.steps):
        cb = cpu_baseline_run(cores, cores, STEPS_PER_REPLICA)
        times.append(cores * STEPS_PER_REPLICA * N / cb["value"])
        total += cores * STEPS_PER_REPLICA * N
    value = total / sum(times)
    line = {
        "impl": "reference", "metric": "flip-evals/s", "value": value, "unit": "flip-evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config({"reference_sample": f"{cores} replicas per step (one per host core)"}),
        "cpu_baseline": {"value": value, "unit": "flip-evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: {cores} of the {REPLICAS} replicas x {STEPS_PER_REPLICA} steps"},
        "e2e": {"value": value, "unit": "flip-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm


def run_gpu(args) -> None:
    import torch

    import paper_2504_00987_gb300 as labs
    from paper_2504_00987_gb300 import _build

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    apply_overrides(args)
    first, _ = parallel.shard(world, rank, REPLICAS)
    P = labs.make_params(N, K, max_steps=STEPS_PER_REPLICA)
    out = torch.empty((REPLICAS, 8), dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        labs.mts_launch(P, 0, first, REPLICAS, out=out)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    props = torch.cuda.get_device_properties(dev)
    try:  # nvidia-smi prints the bus id as DDDDDDDD:BB:DD.F
        bus = "{:02x}:{:02x}.".format(int(props.pci_bus_id), int(props.pci_device_id))
    except (AttributeError, TypeError, ValueError):
        bus = None
    barrier()
    with ClockSampler(bus) as clocks:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)  # evict L2 between timed steps (untimed)
            starts[i].record(stream)
            labs.mts_launch(P, 0, first, REPLICAS, out=out, stream=stream)
            ends[i].record(stream)
        barrier()
        wall = time.perf_counter() - wall0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    res = labs.decode_results(out, N, first)
    steps_done = sum(r["steps"] for r in res)
    assert steps_done == REPLICAS * STEPS_PER_REPLICA, "every replica must use its full step budget"
    local_ms = sum(step_ms)
    clock = clocks.summary()

    # e2e: the blocking C-ABI call with host results (allocation, launch, D2H)
    e2e_ms = []
    for _ in range(0 if args.no_e2e else max(1, args.steps // 3)):
        barrier()
        t0 = time.perf_counter()
        hres = labs.mts_run(P, 0, first, REPLICAS)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        assert sum(r["steps"] for r in hres) == REPLICAS * STEPS_PER_REPLICA
    if not e2e_ms:
        e2e_ms = [float("nan")]

    # max over ranks of the timed region; the best replica of the whole job
    total_ms, e2e_step_ms = parallel.max_over_ranks(pg, [local_ms, sum(e2e_ms) / len(e2e_ms)], dev)
    lbest = min(res, key=lambda r: (r["E"], r["instance"]))
    best_E, best_inst = parallel.best_over_ranks(pg, lbest["E"], lbest["instance"], dev)
    extras = None
    if not args.no_extras:
        extras = c2_extras(args, torch, labs, pg, dev, world, rank, stream)
        extras.update(c34_extras(args, torch, labs, pg, dev, world, rank))
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return

    flips_per_step_all = REPLICAS * STEPS_PER_REPLICA * N * world
    ms_per_step = total_ms / args.steps
    value = flips_per_step_all / (ms_per_step / 1e3)
    pair_terms_per_launch = REPLICAS * STEPS_PER_REPLICA * N * (N - 1)
    achieved = pair_terms_per_launch / (statistics.mean(step_ms) / 1e3) / 1e9  # Gop/s
    peak = SM_COUNT_GB300 * INT32_LANES_PER_SM * SM_MAX_MHZ_GB300 * 1e6 / 1e9  # Gop/s
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        rec = json.load(open(TRAFFIC_FILE))
        if rec.get("kernel_hash") == kernel_hash() and N == 64:  # captured on the N = 64 kernel
            traffic = rec.get("bytes_per_launch")
    line = {
        "metric": "flip-evals/s", "value": value, "unit": "flip-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": workload_config({"l2": "flushed between timed steps (256 MiB write, untimed)",
                                   "parallelism": f"replicas only, {REPLICAS} per GPU"}),
        "pair_terms_per_s": value * (N - 1),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "note": "achieved = pair-terms (one scalar int32 accumulate each) per launch / "
                             "mean launch time; peak = 152 SMs x 128 int32 lanes x 2070 MHz"},
        "e2e": None if args.no_e2e else {
            "value": flips_per_step_all / (e2e_step_ms / 1e3), "unit": "flip-evals/s",
            "h2d_bytes_per_step": ctypes.sizeof(P), "d2h_bytes_per_step": REPLICAS * 64,
            "call": "labs_mts_run (blocking; results copied to host)",
            "inputs": "the instance definition (labs_params) goes with the launch; each replica's "
                      "population is drawn on the device from (seed, instance), Algorithm 1"},
        "gpu_launches": args.steps,
        "best_E": best_E, "best_merit_factor": N * N / (2.0 * best_E), "best_instance": best_inst,
        "wall_s_timed": wall,
        "clocks": clock,
    }
    if extras is not None:
        line.update(extras)
    if world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        line["cpu_baseline"] = cpu_baseline_run(2 * cores, cores, STEPS_PER_REPLICA)
        if extras is not None:
            line["sweep_cpu_baseline"] = sweep_cpu_baseline(cores)
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def c2_extras(args, torch, labs, pg, dev, world, rank, stream) -> dict:
    """The N = 92..120 configuration beside the headline: its throughput sweep
    (16 replicas per SM x 10^6 tabu steps per N, one timed launch each) and its
    time to target (the oracle's one-minute best energy per N, the launch's
    replicas stopped by the global termination flag; p50/p99 over --tts-runs
    seeds per N)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    reps, steps = sms * 16, 1_000_000
    first, _ = parallel.shard(world, rank, reps)
    rows = sweep_rows(torch, labs, pg, dev, first, reps, steps, 1, 1, stream, world)
    targets = load_targets("sweep_n92_120")
    treps, cap = sms * TTS_REPLICAS_PER_SM, 10_000_000
    trows = tts_rows(torch, labs, SWEEP_NS, targets, treps, cap, args.tts_runs, stream, pg=pg, rank=rank)
    return {
        "sweep_n92_120": {"workload": f"N=92..120 step 4, K=100, {reps} replicas x {steps} tabu steps per N "
                                      f"per GPU, one timed launch per N",
                          "flip_evals_per_s": {str(r["N"]): r["flip_evals_per_s"] for r in rows},
                          "best_E": {str(r["N"]): r["best_E"] for r in rows},
                          "value": sum(r["flips"] for r in rows) / (sum(r["ms"] for r in rows) / 1e3)},
        "tts_n92_120": {"workload": f"{treps} replicas per GPU with the global termination flag, K=100, cap "
                                    f"{cap} steps per replica, seeds 1000..{999 + args.tts_runs}"
                                    + (", ranks stop together between slices of 100 generations"
                                       if world > 1 else ""),
                        "targets": "tests/golden/targets.json sweep_n92_120 (the oracle's one-minute best)",
                        "runs_per_N": args.tts_runs,
                        "reached": {str(r["N"]): r["reached"] for r in trows},
                        "target_E": {str(r["N"]): r["target_E"] for r in trows}},
        "tts_p50_s": {str(r["N"]): r["p50_s"] for r in trows},
        "tts_p99_s": {str(r["N"]): r["p99_s"] for r in trows},
    }


def c34_extras(args, torch, labs, pg, dev, world, rank) -> dict:
    """The batched and the served forms beside the headline, shortened so that
    the default run stays short: the 512-instance uneven batch (the autotuned
    graph launch, 10 timed launches, and every instance as its own launch) and
    the solve service on the first --extras-requests requests of the Poisson
    stream (the plain one-launch-per-request form on the first tenth)."""
    b = batch_measure(args, torch, labs, pg, dev, world, rank, steps=10, grid=False)
    nreq = args.extras_requests
    sv = serve_measure(args, torch, labs, world, rank, nreq, max(1, nreq // 10))
    return {
        "batch_uneven_512": {
            "workload": "512 instances, N~U{40..127}, K~U{50..200}, 10 N^2 steps, seed 7; one persistent "
                        "graph launch per batch, mean of 10",
            "ms_per_batch": b["ms_per_batch"], "flip_evals_per_s": b["flip_evals_per_s"],
            "mapping": b["mapping"],
            "plain_one_launch_per_instance": b["plain_one_launch_per_instance"],
            "speedup_vs_plain": b["speedup_vs_plain"]},
        "serve_poisson": {
            "workload": serve_config(args, nreq)["workload"] + " (the first requests of the 20,000-request stream)",
            **{k: sv[k] for k in ("flip_evals_per_s", "latency_s", "target_misses", "in_flight",
                                  "admission_held_back", "plain_one_launch_per_request")}},
    }


# ---------------------------------------------------------------- other workloads
# These print one JSON line each for the configurations beside the default
# one: the N = 92..120 sweep, time-to-target, the uneven batch and the solve
# service.  Each compares against the plain form where the contract names one.

TARGETS_FILE = os.path.join(ROOT, "tests", "golden", "targets.json")


def gpu_context(args):
    import torch

    from paper_2504_00987_gb300 import _build

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    return torch, dev, pg, world, rank


def load_targets(kind: str) -> dict:
    with open(TARGETS_FILE) as f:
        return {int(n): v["E"] for n, v in json.load(f)[kind]["targets"].items()}


def timed_launch(torch, fn, stream):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    out = fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e), out


SWEEP_NS = list(range(92, 121, 4))


def sweep_rows(torch, labs, pg, dev, first, reps, steps, timed, warmup, stream, world):
    """C2 throughput: per N = 92..120 step 4, `timed` launches of `reps` replicas x
    `steps` tabu steps (K=100) after `warmup` short ones; time = max over ranks."""
    rows = []
    for n in SWEEP_NS:
        P = labs.make_params(n, 100, max_steps=steps)
        warm = labs.make_params(n, 100, max_steps=max(1, steps // 100))
        for _ in range(warmup):
            labs.mts_launch(warm, 0, first, reps)
        ms_list = []
        for _ in range(timed):
            ms, out = timed_launch(torch, lambda: labs.mts_launch(P, 0, first, reps, stream=stream), stream)
            ms_list.append(ms)
        ms = parallel.max_over_ranks(pg, [statistics.mean(ms_list)], dev)[0]
        res = labs.decode_results(out, n, first)
        assert sum(r["steps"] for r in res) == reps * steps, "every replica must use its full step budget"
        lb = min(res, key=lambda r: (r["E"], r["instance"]))
        bE, bi = parallel.best_over_ranks(pg, lb["E"], lb["instance"], dev)
        flips = reps * steps * n * world
        rows.append({"N": n, "ms": ms, "flips": flips, "flip_evals_per_s": flips / (ms / 1e3),
                     "pair_terms_per_s": flips * (n - 1) / (ms / 1e3), "best_E": bE,
                     "best_merit_factor": n * n / (2.0 * bE), "best_instance": bi})
    return rows


def sweep_cpu_baseline(cores: int, steps: int = 10_000) -> dict:
    """The oracle on the sweep's N and parameters: one replica per host core."""
    per_n = {str(n): cpu_baseline_run(cores, cores, steps, n)["value"] for n in SWEEP_NS}
    return {"value": statistics.mean(per_n.values()), "unit": "flip-evals/s", "cores": cores,
            "kind": "oracle", "per_N": per_n,
            "sample": f"per N: {cores} replicas (instances 0..{cores - 1}) x {steps} tabu steps, "
                      f"one replica per thread; value = mean over N"}


def run_sweep(args) -> None:
    """N = 92, 96, ..., 120 (two words), one K=100 population per warp, 16 warps per SM
    (more warps hide the step's latencies)."""
    torch, dev, pg, world, rank = gpu_context(args)
    import paper_2504_00987_gb300 as labs

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    reps = args.replicas or sms * 16
    steps = args.steps_per_replica or 1_000_000
    first, _ = parallel.shard(world, rank, reps)
    stream = torch.cuda.current_stream()
    rows = sweep_rows(torch, labs, pg, dev, first, reps, steps, args.steps, args.warmup, stream, world)
    tot_flips, tot_ms = sum(r.pop("flips") for r in rows), sum(r["ms"] for r in rows)
    cpu = sweep_cpu_baseline(cpu_cores()) if world == 1 and not args.no_cpu_baseline else None
    if rank == 0:
        print(json.dumps({
            "cpu_baseline": cpu,
            "metric": "flip-evals/s", "value": tot_flips / (tot_ms / 1e3), "unit": "flip-evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"sweep_n92_120: N=92..120 step 4, K=100, {reps} replicas x {steps} steps per N",
                       "replicas_per_gpu": reps, "steps_per_replica": steps},
            "per_N": rows}), flush=True)


def fit_exponential(Ns, medians):
    """OLS of log(median) on N (Table III): a * b^N with 95 % intervals of a and b."""
    import numpy as np

    x = np.asarray(Ns, dtype=float)
    y = np.log(np.asarray(medians, dtype=float))
    A = np.vstack([np.ones_like(x), x]).T
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    resid = y - A @ coef
    dof = max(len(x) - 2, 1)
    s2 = float(resid @ resid) / dof
    cov = s2 * np.linalg.inv(A.T @ A)
    from scipy import stats

    tq = float(stats.t.ppf(0.975, dof))
    la, lb = coef
    sa, sb = np.sqrt(np.diag(cov))
    return {"a": float(np.exp(la)), "a_ci": [float(np.exp(la - tq * sa)), float(np.exp(la + tq * sa))],
            "b": float(np.exp(lb)), "b_ci": [float(np.exp(lb - tq * sb)), float(np.exp(lb + tq * sb))],
            "N_min_fit": int(min(Ns)), "N_max_fit": int(max(Ns))}


# Time to target runs 16 replicas per SM: measured against 8, 4 and 32 per SM on
# the N = 92..120 targets, 16 gave the lowest median p50 (3.0 ms against 3.3 ms at 8;
# 32 per SM cannot all be resident, so the flag stops the first wave's search).
TTS_REPLICAS_PER_SM = 16


def tts_run_ranks(torch, labs, pg, dev, n, target, seed, first, reps, cap, state, out, flag, stream,
                  slice_gens=100):
    """One time-to-target run on every rank: the rank's replicas advance in slices
    of `slice_gens` generations (labs_mts_resume), and after each slice the ranks
    OR their reached flags (parallel.run_until_any), so every GPU stops after the
    slice in which any replica of the job reached the target.  Returns (seconds,
    reached, tabu steps of this rank's replicas)."""
    gens = [0]

    def run_slice(i):
        gens[0] += slice_gens
        P = labs.make_params(n, 100, max_generations=gens[0], max_steps=cap, target_E=target, glf=True)
        labs.mts_resume(P, seed, first, reps, state, resume=i > 0, out=out, glf_flag=flag, stream=stream)
        return bool(((out[:, 4] >> 32) == labs.RUN_REACHED).any().item())

    flag.zero_()
    pg.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    max_slices = cap // (slice_gens * max(1, n // 2)) + 1  # a generation takes at least N/2 steps
    _, ok = parallel.run_until_any(pg, run_slice, max_slices, dev)
    torch.cuda.synchronize()
    dt = parallel.max_over_ranks(pg, [time.perf_counter() - t0], dev)[0]
    return dt, ok, int(out[:, 6].sum().item())


def tts_rows(torch, labs, Ns, targets, reps, cap, runs, stream, variant=0, replace_policy=0, pg=None,
             rank=0):
    """Per N: `runs` launches of `reps` replicas (seeds 1000, 1001, ...) that stop,
    all of them, as soon as one reaches targets[N]; seconds to target per run.
    Under torchrun (pg given) each rank runs its own `reps` replicas and the
    ranks share the stop flag between slices of generations (tts_run_ranks)."""
    import numpy as np

    if pg is not None:
        if variant or replace_policy:
            raise ValueError("variants run on one GPU")
        dev = stream.device
        rows = []
        for n in Ns:
            state = torch.empty(reps * labs.mts_state_bytes(n, 100), dtype=torch.uint8, device=dev)
            out = torch.empty((reps, 8), dtype=torch.int64, device=dev)
            flag = torch.zeros(1, dtype=torch.int32, device=dev)
            times, work, reached = [], [], 0
            for run in range(runs):
                dt, ok, st = tts_run_ranks(torch, labs, pg, dev, n, targets[n], 1000 + run, rank * reps, reps,
                                           cap, state, out, flag, stream)
                st = parallel.sum_over_ranks(pg, [float(st)], dev)[0]
                reached += ok
                times.append(dt if ok else float("inf"))
                work.append(st if ok else float("inf"))
            t, w = np.array(times), np.array(work)
            rows.append({"N": n, "target_E": targets[n], "runs": runs, "reached": reached,
                         "p50_s": float(np.percentile(t, 50)), "p99_s": float(np.percentile(t, 99)),
                         "q1_s": float(np.percentile(t, 25)), "q3_s": float(np.percentile(t, 75)),
                         "p50_steps": float(np.percentile(w, 50)), "times_s": [round(x, 6) for x in times]})
        return rows
    rows = []
    for n in Ns:
        target = targets[n]
        P = labs.make_params(n, 100, target_E=target, max_steps=cap, glf=True, variant=variant,
                             replace_policy=replace_policy)
        labs.mts_launch(labs.make_params(n, 100, max_steps=1000, variant=variant), 0, 0, reps)
        times, work, reached = [], [], 0
        for run in range(runs):
            flag = torch.zeros(1, dtype=torch.int32, device=stream.device)
            ms, out = timed_launch(torch, lambda: labs.mts_launch(P, 1000 + run, 0, reps, glf_flag=flag,
                                                                  stream=stream), stream)
            res = labs.decode_results(out, n)
            ok = any(r["status"] == labs.RUN_REACHED for r in res)
            reached += ok
            times.append(ms / 1e3 if ok else float("inf"))
            work.append(sum(r["steps"] for r in res) if ok else float("inf"))  # tabu steps, all replicas
        t, w = np.array(times), np.array(work)
        rows.append({"N": n, "target_E": target, "runs": runs, "reached": reached,
                     "p50_s": float(np.percentile(t, 50)), "p99_s": float(np.percentile(t, 99)),
                     "q1_s": float(np.percentile(t, 25)), "q3_s": float(np.percentile(t, 75)),
                     "p50_steps": float(np.percentile(w, 50)),
                     "times_s": [round(x, 6) for x in times]})
        print(json.dumps({k: v for k, v in rows[-1].items() if k != "times_s"}), file=sys.stderr, flush=True)
    return rows


def median_fit(rows, key="p50_s"):
    import numpy as np

    ok_rows = [r for r in rows if np.isfinite(r[key])]
    if len(ok_rows) < 3:
        return None
    return fit_exponential([r["N"] for r in ok_rows], [r[key] for r in ok_rows])


def run_tts(args) -> None:
    """Time to a target E with every replica of the launch stopped by the global
    termination flag; p50/p99 over runs with distinct seeds, and an a * b^N fit of the
    median (Table III).  Targets (tests/golden/targets.json): the oracle's one-minute
    best for N = 92..120, or the exact optimum (exhaustive search) for N = 16..36.
    Each N also reports the median tabu steps of all replicas to the target (the
    work, free of launch overhead), with the same fit."""
    torch, dev, pg, world, rank = gpu_context(args)
    import paper_2504_00987_gb300 as labs

    kind = "optimum_n16_36" if args.tts_targets == "optimum" else "sweep_n92_120"
    targets = load_targets(kind)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    reps = args.replicas or sms * TTS_REPLICAS_PER_SM
    cap = args.steps_per_replica or 10_000_000
    stream = torch.cuda.current_stream()
    Ns = [int(x) for x in args.tts_n.split(",")] if args.tts_n else sorted(targets)
    rows = tts_rows(torch, labs, Ns, targets, reps, cap, args.runs, stream, pg=pg, rank=rank)
    for r in rows:
        r.pop("times_s")
    if rank == 0:
        print(json.dumps({
            "metric": "time-to-target-E p50", "value": statistics.median(r["p50_s"] for r in rows),
            "unit": "s", "n_gpus": world, "higher_is_better": False, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"tts_{kind}: {reps} replicas with the global termination flag, K=100, "
                                   f"cap {cap} steps per replica", "runs_per_N": args.runs, "targets": kind},
            "per_N": rows, "fit_median_a_b_pow_N": median_fit(rows),
            "fit_median_steps_a_b_pow_N": median_fit(rows, "p50_steps"),
            f"fit_median_steps_a_b_pow_N_from_{args.fit_min_n}":
                median_fit([r for r in rows if r["N"] >= args.fit_min_n], "p50_steps")}), flush=True)


# Policies compared by the A/B time-to-target workload: the default reading of
# Algorithm 1 and one change each (replace-worst, uniform crossover, s_1 = +1).
AB_POLICIES = [
    ("one_point+replace_random", 0, 0),
    ("one_point+replace_worst", 0, 1),
    ("uniform+replace_random", 1, 0),
    ("one_point+replace_random+s1_fixed", 2, 0),
    ("uniform+replace_worst+s1_fixed", 3, 1),
]


def run_tts_ab(args) -> None:
    """A/B time to target of the population policies, same N, targets, seeds and
    replica count for each; per N the Mann-Whitney U test of each policy's run
    times against the default's (two-sided; runs that miss count as +inf)."""
    torch, dev, pg, world, rank = gpu_context(args)
    import numpy as np
    from scipy import stats

    import paper_2504_00987_gb300 as labs

    kind = "optimum_n16_36" if args.tts_targets == "optimum" else "sweep_n92_120"
    targets = load_targets(kind)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    reps = args.replicas or sms * 8
    cap = args.steps_per_replica or 10_000_000
    stream = torch.cuda.current_stream()
    Ns = [int(x) for x in args.tts_n.split(",")] if args.tts_n else sorted(targets)[:5]
    out = {}
    for name, variant, policy in AB_POLICIES:
        print(f"# {name}", file=sys.stderr, flush=True)
        out[name] = tts_rows(torch, labs, Ns, targets, reps, cap, args.runs, stream, variant=variant,
                             replace_policy=policy)
    base = out[AB_POLICIES[0][0]]
    summary = []
    for name, variant, policy in AB_POLICIES:
        rows = out[name]
        per_n = []
        for r, b in zip(rows, base):
            big = 1e9  # a run that missed ranks after every run that reached
            x = np.minimum(np.array(r["times_s"]), big)
            y = np.minimum(np.array(b["times_s"]), big)
            p = float(stats.mannwhitneyu(x, y, alternative="two-sided").pvalue) if name != AB_POLICIES[0][0] else None
            per_n.append({"N": r["N"], "reached": r["reached"], "p50_s": r["p50_s"], "q1_s": r["q1_s"],
                          "q3_s": r["q3_s"], "p50_ratio_vs_default": r["p50_s"] / b["p50_s"],
                          "mannwhitney_p_vs_default": p})
        summary.append({"policy": name, "variant": variant, "replace_policy": policy,
                        "per_N": per_n, "fit_median_a_b_pow_N": median_fit(rows),
                        "geomean_p50_ratio_vs_default": float(np.exp(np.mean(np.log(
                            [q["p50_ratio_vs_default"] for q in per_n]))))})
    if rank == 0:
        print(json.dumps({
            "metric": "time-to-target-E p50 ratio vs default policy (geomean over N)",
            "value": min(s["geomean_p50_ratio_vs_default"] for s in summary[1:]),
            "unit": "ratio", "n_gpus": world, "higher_is_better": False, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"tts_ab_{kind}: {len(AB_POLICIES)} policies, N={Ns}, {reps} replicas with "
                                   f"the global termination flag, K=100, cap {cap} steps per replica",
                       "runs_per_N": args.runs, "targets": kind},
            "policies": summary}), flush=True)


def run_skew_ab(args) -> None:
    """Unrestricted search against the search restricted to skew-symmetric
    sequences (Sec. II.C), odd N = 17..45.  Both race to the exhaustive
    skew-symmetric optimum (reachable by both); where the exhaustive optimum
    over all sequences is known (N <= 31) the unrestricted search also races
    to it (the restricted one reaches it only if it is skew-symmetric).  Per
    N: median time and median tabu steps (all replicas) to target, and an
    a * b^N fit of each median."""
    torch, dev, pg, world, rank = gpu_context(args)
    import paper_2504_00987_gb300 as labs

    skew_opt = load_targets("skew_optimum_odd_n17_45")
    all_opt = load_targets("optimum_n16_36")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    reps = args.replicas or sms * 8
    cap = args.steps_per_replica or 2_000_000
    stream = torch.cuda.current_stream()
    Ns = [int(x) for x in args.tts_n.split(",")] if args.tts_n else sorted(skew_opt)
    runs = args.runs
    rows_u = tts_rows(torch, labs, Ns, skew_opt, reps, cap, runs, stream)
    rows_s = tts_rows(torch, labs, Ns, skew_opt, reps, cap, runs, stream, variant=labs.VARIANT_SKEW)
    Ns_all = [n for n in Ns if n in all_opt and all_opt[n] < skew_opt[n]]
    rows_o = tts_rows(torch, labs, Ns_all, all_opt, reps, cap, runs, stream) if Ns_all else []
    per_n = []
    for u, k in zip(rows_u, rows_s):
        n = u["N"]
        o = next((x for x in rows_o if x["N"] == n), None)
        per_n.append({
            "N": n, "E_skew_opt": skew_opt[n], "E_opt": all_opt.get(n),
            "unrestricted_to_skew_opt": {x: u[x] for x in ("reached", "p50_s", "q1_s", "q3_s", "p50_steps")},
            "restricted_to_skew_opt": {x: k[x] for x in ("reached", "p50_s", "q1_s", "q3_s", "p50_steps")},
            "p50_steps_ratio_restricted_vs_unrestricted": k["p50_steps"] / u["p50_steps"],
            "unrestricted_to_opt": ({x: o[x] for x in ("reached", "p50_s", "p50_steps")} if o else None),
        })
    if rank == 0:
        ratios = [r["p50_steps_ratio_restricted_vs_unrestricted"] for r in per_n]
        print(json.dumps({
            "metric": "tabu steps to the skew-symmetric optimum, restricted / unrestricted (geomean over N)",
            "value": statistics.geometric_mean(ratios), "unit": "ratio", "n_gpus": world,
            "higher_is_better": False, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"skew_ab: odd N={Ns}, {reps} replicas with the global termination flag, "
                                   f"K=100, cap {cap} steps per replica", "runs_per_N": runs,
                       "targets": "skew_optimum_odd_n17_45, optimum_n16_36"},
            "fit_unrestricted_p50_steps": median_fit(rows_u, "p50_steps"),
            "fit_restricted_p50_steps": median_fit(rows_s, "p50_steps"),
            "fit_unrestricted_p50_s": median_fit(rows_u), "fit_restricted_p50_s": median_fit(rows_s),
            "per_N": per_n}), flush=True)


def batch_measure(args, torch, labs, pg, dev, world, rank, steps, grid=True) -> dict:
    """512 uneven instances (N ~ U{40..127}, K ~ U{50..200}, 10 N^2 steps): the autotuned,
    graph-captured persistent launch (mean of `steps` timed launches, max over ranks),
    optionally a grid of other mappings, and the plain form (one launch per instance)."""
    from paper_2504_00987_gb300 import workloads

    wl = workloads.uneven_batch(512, seed=7, steps_per_n2=10)
    lo, cnt = parallel.split_range(len(wl), world, rank)
    wl = wl[lo:lo + cnt]
    inst = [labs.make_instance(x.N, x.K, seed=x.seed, instance=x.instance, max_steps=x.max_steps) for x in wl]
    flips = sum(x.max_steps * x.N for x in wl)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    if args.batch_mapping:  # profiling: this mapping only (no tuning, grid or plain form)
        wpb, bps, wps = (int(v) for v in args.batch_mapping.split(","))
        mapping = {"warps_per_block": wpb, "blocks_per_sm": bps, "order": 0, "warps_per_seq": wps}
    else:
        mapping = labs.autotune(inst)
    tune_s = time.perf_counter() - t0

    def makespan(m, n):
        with labs.Batch(inst, mapping=m) as b:
            for _ in range(args.warmup):
                b.launch()
            torch.cuda.synchronize()
            return statistics.mean(timed_launch(torch, lambda: b.launch(stream), stream)[0] for _ in range(n))

    ms = parallel.max_over_ranks(pg, [makespan(mapping, steps)], dev)[0]
    total_flips = parallel.sum_over_ranks(pg, [float(flips)], dev)[0]
    out = {"ms_per_batch": ms, "flip_evals_per_s": total_flips / (ms / 1e3), "mapping": mapping,
           "autotune_s": tune_s, "instances": len(wl)}
    if args.batch_mapping:
        return out
    if grid:  # other mappings, for the record: one and two warps per replica
        out["mappings_ms"] = []
        for wps in (1, 2):
            for wpb, bps in ((wps, 1), (wps, 2), (4, 1), (4, 2)):
                m = {"warps_per_block": wpb, "blocks_per_sm": bps, "order": 0, "warps_per_seq": wps}
                out["mappings_ms"].append({**m, "ms": parallel.max_over_ranks(pg, [makespan(m, 3)], dev)[0]})
    # plain form: one launch per instance, round robin over 128 streams (the
    # kernels a GPU runs at once), every instance of the batch
    streams = [torch.cuda.Stream() for _ in range(128)]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for i, x in enumerate(wl):
        labs.mts_launch(labs.make_params(x.N, x.K, max_steps=x.max_steps), x.seed, x.instance, 1,
                        stream=streams[i % len(streams)])
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t1
    out["plain_one_launch_per_instance"] = {"flip_evals_per_s": flips / plain_s, "instances": len(wl),
                                            "streams": len(streams), "wall_s": plain_s}
    out["speedup_vs_plain"] = out["flip_evals_per_s"] / (flips / plain_s)
    return out


def run_batch(args) -> None:
    """The uneven batch as its own JSON line (`--workload batch`)."""
    torch, dev, pg, world, rank = gpu_context(args)
    import paper_2504_00987_gb300 as labs

    r = batch_measure(args, torch, labs, pg, dev, world, rank, args.steps)
    if rank != 0:
        return
    line = {"metric": "flip-evals/s", "value": r["flip_evals_per_s"], "unit": "flip-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_batch"],
            "higher_is_better": True, "dtype": "int32", "data": "synthetic"}
    if args.batch_mapping:
        line["config"] = {"workload": "batch_uneven_512 (profiling: fixed mapping)", "mapping": r["mapping"]}
    else:
        line.update({"scaling": "strong",
                     "config": {"workload": "batch_uneven_512: N~U{40..127}, K~U{50..200}, 10 N^2 steps, seed 7",
                                "mapping": r["mapping"], "autotune_s": r["autotune_s"]},
                     "mappings_ms": r["mappings_ms"],
                     "plain_one_launch_per_instance": r["plain_one_launch_per_instance"],
                     "speedup_vs_plain": r["speedup_vs_plain"]})
    print(json.dumps(line), flush=True)


def serve_measure(args, torch, labs, world, rank, requests, baseline_requests) -> dict:
    """Poisson solve requests (mean 200/s, N ~ U{32..160}, K=100, half with a target E = the
    oracle's ten-second best, half capped at 10^5 steps) through the continuous-batching
    service, and a prefix of the same stream as one launch per request on a pool of streams."""
    import numpy as np

    from paper_2504_00987_gb300 import workloads

    targets = load_targets("serve_n32_160")
    reqs = workloads.poisson_requests(requests, 200.0, seed=11)
    lo, cnt = parallel.split_range(len(reqs), world, rank)
    reqs = reqs[lo:lo + cnt]

    def instance(i, r):
        if r.target_mode:
            return labs.make_instance(r.N, r.K, seed=11, instance=lo + i, target_E=targets[r.N],
                                      max_steps=r.max_steps)
        return labs.make_instance(r.N, r.K, seed=11, instance=lo + i, max_steps=r.max_steps)

    insts = [instance(i, r) for i, r in enumerate(reqs)]

    def drive(submit, poll, running=None):
        done, pending, i = {}, [], 0
        t0 = time.perf_counter()
        samples, t_sample = [], 0.0
        while len(done) < len(reqs):
            if running is not None and time.perf_counter() - t_sample > 0.01:
                t_sample = time.perf_counter()
                samples.append(running())
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival_s <= now:
                pending.append((i, submit(i), t0 + reqs[i].arrival_s))
                i += 1
            keep = []
            for k, h, t_arr in pending:
                res = poll(h)
                if res is None:
                    keep.append((k, h, t_arr))
                else:
                    done[k] = (res, time.perf_counter() - t_arr)
            pending = keep
            time.sleep(0.0002)
        drive.in_flight = samples
        return done, time.perf_counter() - t0

    qsteps = args.quantum_steps if args.quantum_us == 0 else (1 << 40)
    with labs.Server(max_slots=args.slots or 4096, max_N=160, max_K=100, quantum_steps=qsteps,
                     quantum_us=args.quantum_us, warps_per_request=args.warps_per_request) as srv:
        done, wall = drive(lambda i: srv.submit(insts[i]), srv.poll, lambda: srv.stats()["running"])
        st = srv.stats()
    in_flight = drive.in_flight
    lat = np.array([done[k][1] for k in range(len(reqs))])
    tmode = np.array([r.target_mode for r in reqs])
    missed = sum(1 for k, r in enumerate(reqs) if r.target_mode and done[k][0]["status"] != labs.RUN_REACHED)
    served_rate = st["flip_evals"] / wall
    # one launch per request on a prefix of the same stream, round robin over as many
    # streams as the service had requests in flight on average (at most 128, the
    # number of kernels a GPU runs concurrently)
    nb = min(len(reqs), baseline_requests)
    mean_in_flight = float(np.mean(in_flight)) if in_flight else 1.0
    n_streams = int(min(128, max(1, round(mean_in_flight))))
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    outs, evs = {}, {}

    def submit_plain(i):
        x = insts[i]
        st_ = streams[i % len(streams)]
        P = labs.make_params(x.N, x.K, max_steps=x.max_steps, target_E=x.target_E)
        outs[i] = labs.mts_launch(P, x.seed, x.instance, 1, stream=st_)
        ev = torch.cuda.Event()
        ev.record(st_)
        evs[i] = ev
        return i

    def poll_plain(i):
        return {"done": True} if evs[i].query() else None

    saved = reqs
    reqs = reqs[:nb]
    done_b, wall_b = drive(submit_plain, poll_plain)
    reqs = saved
    lat_b = np.array([done_b[k][1] for k in range(nb)])
    flips_b = sum(labs.decode_results(outs[k], insts[k].N)[0]["flip_evals"] for k in range(nb))
    return {
        "requests": requests, "flip_evals_per_s": served_rate,
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "p50_target_mode": float(np.percentile(lat[tmode], 50)) if tmode.any() else None,
                      "p99_target_mode": float(np.percentile(lat[tmode], 99)) if tmode.any() else None,
                      "p50_cap_mode": float(np.percentile(lat[~tmode], 50)) if (~tmode).any() else None,
                      "p99_cap_mode": float(np.percentile(lat[~tmode], 99)) if (~tmode).any() else None},
        "target_misses": missed, "wall_s": wall, "gpu_busy_s": st["gpu_seconds"], "quanta": st["quanta"],
        "in_flight": {"mean": mean_in_flight, "max": int(max(in_flight)) if in_flight else 0},
        "warps_per_request": args.warps_per_request, "pair_quanta": st["pair_quanta"],
        "admission_held_back": {"slots": st["deferred_slots"], "shared_memory": st["deferred_smem"],
                                "arena": st["deferred_hbm"]},
        "arena_bytes": st["arena_bytes"],
        "plain_one_launch_per_request": {
            "requests": nb, "streams": n_streams, "flip_evals_per_s": flips_b / wall_b,
            "latency_p50_s": float(np.percentile(lat_b, 50)),
            "latency_p99_s": float(np.percentile(lat_b, 99))},
    }


def serve_config(args, requests) -> dict:
    return {"workload": f"serve_poisson: {requests} requests at 200/s, N~U{{32..160}}, K=100, "
                        "half target mode (oracle 10 s best, cap 1e7 steps), half 1e5 steps, seed 11",
            "slots": args.slots or 4096,
            "quantum": (f"{args.quantum_us} us of device time per slot" if args.quantum_us
                        else f"{args.quantum_steps} tabu steps per slot")}


def run_serve(args) -> None:
    """The solve service as its own JSON line (`--workload serve`)."""
    torch, dev, pg, world, rank = gpu_context(args)
    import paper_2504_00987_gb300 as labs

    r = serve_measure(args, torch, labs, world, rank, args.requests, args.baseline_requests)
    if rank == 0:
        line = {"metric": "flip-evals/s", "value": r.pop("flip_evals_per_s"), "unit": "flip-evals/s",
                "n_gpus": world, "higher_is_better": True, "dtype": "int32", "data": "synthetic",
                "config": serve_config(args, r.pop("requests"))}
        line.update(r)
        print(json.dumps(line), flush=True)


def run_skew(args) -> None:
    """d(S) of Appendix A for 100,000 random N=120 sequences (even N: rotations x deletions)."""
    torch, dev, pg, world, rank = gpu_context(args)
    import numpy as np

    import paper_2504_00987_gb300 as labs
    from paper_2504_00987_gb300 import workloads

    n, B = 120, args.replicas or 100_000
    seqs = torch.from_numpy(workloads.random_sequences(n, B, seed=5).view(np.int64)).to(dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        labs.skew_deviation_batch(seqs, n)
    ms = statistics.mean(timed_launch(torch, lambda: labs.skew_deviation_batch(seqs, n), stream)[0]
                         for _ in range(args.steps))
    ms = parallel.max_over_ranks(pg, [ms], dev)[0]
    line = {"metric": "sequences/s", "value": B * world / (ms / 1e3), "unit": "sequences/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"skew_deviation_n120: {B} random sequences, d(S) over 120 rotations x 120 deletions"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        host = seqs[:200].cpu().numpy().view(np.uint64)
        t0 = time.perf_counter()
        for b in range(len(host)):
            oracle.skew_deviation(host[b], n)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(host) / dt, "unit": "sequences/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {len(host)} sequences, one core"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without its N=92..120 sweep, time-to-target, batch and service keys")
    ap.add_argument("--tts-runs", type=int, default=50, help="default line: time-to-target runs per N")
    ap.add_argument("--replicas", type=int, default=0, help="profiling only: override replicas")
    ap.add_argument("--steps-per-replica", type=int, default=0, help="profiling only: override budget")
    ap.add_argument("--n", type=int, default=0, help="profiling only: override N of the default workload")
    ap.add_argument("--workload", choices=["replicas_n64", "sweep_n92_120", "tts", "tts_ab", "skew_ab", "batch",
                                           "serve", "skew"],
                    default="replicas_n64")
    ap.add_argument("--runs", type=int, default=50, help="tts: runs per N")
    ap.add_argument("--tts-n", default="", help="tts: comma-separated N (default: all; tts_ab: first five)")
    ap.add_argument("--tts-targets", choices=["oracle", "optimum"], default="oracle",
                    help="tts: oracle one-minute best (N=92..120) or exact optimum (N=16..36)")
    ap.add_argument("--fit-min-n", type=int, default=30,
                    help="tts: smallest N of the second steps fit (above the one-generation floor)")
    ap.add_argument("--requests", type=int, default=20_000, help="serve: requests")
    ap.add_argument("--extras-requests", type=int, default=2_000,
                    help="default line: requests of the shortened service run")
    ap.add_argument("--baseline-requests", type=int, default=400, help="serve: plain-form prefix")
    ap.add_argument("--slots", type=int, default=0, help="serve: resident slots")
    ap.add_argument("--quantum-steps", type=int, default=2000, help="serve: tabu steps per slot per quantum")
    ap.add_argument("--batch-mapping", default="",
                    help="batch, profiling only: 'warps_per_block,blocks_per_sm,warps_per_seq', one mapping")
    ap.add_argument("--warps-per-request", type=int, default=1,
                    help="serve: 1 = one warp per request, 2 = warp pairs while they fit")
    ap.add_argument("--quantum-us", type=int, default=4000,
                    help="serve: device-time budget per slot per quantum (0: the step count instead)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep_n92_120":
        run_sweep(args)
    elif args.workload == "tts":
        run_tts(args)
    elif args.workload == "tts_ab":
        run_tts_ab(args)
    elif args.workload == "skew_ab":
        run_skew_ab(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "skew":
        run_skew(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
