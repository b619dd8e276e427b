#!/usr/bin/env python3
"""Throughput benchmark of the GB300 memetic tabu search (flip-evals/s).

One step = one launch of the whole hot path over the workload: N=64, K=100,
1,024 independent MTS replicas (Philox streams 0..1023), each running
exactly 10^5 tabu steps (every step scores all N one-bit-flip neighbours).
flip-evals = tabu steps x N; pair-terms = flip-evals x (N-1).

    python bench.py [--gpus G] [--steps S] [--warmup W] [--impl gpu|reference]

Under torchrun each rank runs its own 1,024 replicas (instances offset by
rank x 1,024; weak scaling, no collective on the data path).  Rank 0 prints
one JSON line.  `--impl reference` times the CPU oracle (test
infrastructure) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, K, REPLICAS, STEPS_PER_REPLICA = 64, 100, 1024, 100_000
WORKLOAD = "replicas_n64"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
SM_COUNT_GB300 = 152
INT32_LANES_PER_SM = 128  # 4 SM sub-partitions x 32 lanes
SM_MAX_MHZ_GB300 = 2070.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "mts_kernel_n64_traffic.json")
KERNEL_SOURCES = ["tabu_core.cuh", "mts.cu", "labs_device.cuh", "kernels.h"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2504_00987_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
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


def cpu_baseline_run(replicas: int, threads: int, steps: int) -> dict:
    import oracle

    oracle.build()
    P = oracle.make_params(N, K, max_steps=steps)
    t0 = time.perf_counter()
    res = oracle.mts_run_many(P, 0, 0, replicas, threads)
    dt = time.perf_counter() - t0
    total = sum(r["steps"] for r in res) * N
    return {"value": total / dt, "unit": "flip-evals/s", "cores": threads, "kind": "oracle",
            "sample": f"{replicas} of the {REPLICAS} replicas (instances 0..{replicas - 1}), "
                      f"{steps} tabu steps each, one replica per thread, {dt:.1f} s wall"}


def run_reference(args) -> None:
    world, rank, _ = dist_env()
    if rank != 0:
        return
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

    global REPLICAS, STEPS_PER_REPLICA
    if args.replicas:
        REPLICAS = args.replicas
    if args.steps_per_replica:
        STEPS_PER_REPLICA = args.steps_per_replica
    first = rank * REPLICAS
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

    # max over ranks of the timed region
    if pg is not None:
        t = torch.tensor([local_ms, sum(e2e_ms) / len(e2e_ms)], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total_ms, e2e_step_ms = float(t[0]), float(t[1])
    else:
        total_ms, e2e_step_ms = local_ms, sum(e2e_ms) / len(e2e_ms)
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
        if rec.get("kernel_hash") == kernel_hash():
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
        "e2e": {"value": flips_per_step_all / (e2e_step_ms / 1e3), "unit": "flip-evals/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": REPLICAS * 64,
                "call": "labs_mts_run (blocking; results copied to host)"},
        "gpu_launches": args.steps,
        "wall_s_timed": wall,
        "clocks": clock,
    }
    if world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        line["cpu_baseline"] = cpu_baseline_run(2 * cores, cores, STEPS_PER_REPLICA)
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--replicas", type=int, default=0, help="profiling only: override replicas")
    ap.add_argument("--steps-per-replica", type=int, default=0, help="profiling only: override budget")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
