"""Writes tests/golden/targets.json: target energies for the time-to-target
measurements, computed by the CPU oracle only.

Two sets, each a fixed amount of oracle work so the file is reproducible
(step budgets instead of wall-clock limits):

  sweep_n92_120 -- for N = 92, 96, ..., 120: the best E of 8 oracle replicas
                   (seed 0, instances 0..7), each with 7.2e5 * (120/N)^2 tabu
                   steps, about one minute of the incremental oracle on 8
                   cores of a current x86 host ("the oracle's 60 s best").
  serve_n32_160 -- for N = 32..160: the best E of one oracle replica (seed 0,
                   instance 0) with 4.3e5 * (64/N)^2 steps, about ten seconds
                   of one core ("the oracle's 10 s best").
  optimum_n16_36 -- for N = 16..36: the exact minimum of E over all 2^N
                   sequences and the number of minimisers (the oracle's
                   exhaustive search, split over threads).
  skew_optimum_odd_n17_45 -- for odd N = 17..45: the exact minimum of E over
                   the 2^((N+1)/2) skew-symmetric sequences (Sec. II.C; the
                   oracle's exhaustive search over the free half).

Usage:  python tests/golden/make_targets.py [--only sweep|serve|optimum|skew] [--threads T]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

OUT = os.path.join(HERE, "targets.json")


def sweep_steps(N: int) -> int:
    return int(7.2e5 * (120 / N) ** 2)


def serve_steps(N: int) -> int:
    return int(4.3e5 * (64 / N) ** 2)


def run_one(N: int, instance: int, steps: int) -> int:
    P = oracle.make_params(N, 100, max_steps=steps)
    return oracle.mts_run(P, 0, instance)[0]["E"]


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", choices=["sweep", "serve", "optimum", "skew"], default=None)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    oracle.build()
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    t0 = time.time()
    with ThreadPoolExecutor(max_workers=args.threads) as ex:
        if args.only in (None, "sweep"):
            sweep = {}
            for N in range(92, 121, 4):
                Es = list(ex.map(lambda i, N=N: run_one(N, i, sweep_steps(N)), range(8)))
                sweep[str(N)] = {"E": min(Es), "replicas": 8, "steps_per_replica": sweep_steps(N)}
                print(f"sweep N={N}: E={min(Es)}  ({time.time() - t0:.0f}s)", flush=True)
            data["sweep_n92_120"] = {"seed": 0, "K": 100, "targets": sweep}
        if args.only in (None, "serve"):
            Ns = list(range(32, 161))
            Es = list(ex.map(lambda N: run_one(N, 0, serve_steps(N)), Ns))
            data["serve_n32_160"] = {
                "seed": 0, "K": 100, "instance": 0,
                "targets": {str(N): {"E": E, "steps": serve_steps(N)} for N, E in zip(Ns, Es)},
            }
            print(f"serve: {len(Ns)} targets ({time.time() - t0:.0f}s)", flush=True)
        if args.only in (None, "optimum"):
            targets = {}
            for N in range(16, 37):  # one N at a time, every thread on it
                E, n = oracle.bruteforce_mt(N, args.threads)
                targets[str(N)] = {"E": E, "minimisers": n}
                print(f"optimum N={N}: E={E} ({time.time() - t0:.0f}s)", flush=True)
            data["optimum_n16_36"] = {"targets": targets}
        if args.only in (None, "skew"):
            Ns = list(range(17, 46, 2))
            opts = list(ex.map(oracle.bruteforce_skew, Ns))
            data["skew_optimum_odd_n17_45"] = {
                "targets": {str(N): {"E": E, "minimisers": n} for N, (E, n) in zip(Ns, opts)}}
            print(f"skew: {len(Ns)} exhaustive skew-symmetric minima ({time.time() - t0:.0f}s)", flush=True)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
