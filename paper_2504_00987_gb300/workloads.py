"""Seeded synthetic inputs for the LABS solver, shared by the tests, the
benchmark and the oracle-side checks.

This module holds no arithmetic of the method (no energies, no search): only
seeded numpy draws of packed +-1 sequences and the workload descriptions.
LABS has no dataset -- an instance is defined by its length N alone -- so
every workload here is a list of (N, population, seed, budget) tuples.

Packed format: N spins in ceil(N/64) uint64 words, spin i at bit i % 64 of
word i // 64, bit 1 <-> +1, bits >= N zero.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MAX_N = 256


def words_for(N: int) -> int:
    return (N + 63) // 64


def random_sequences(N: int, B: int, seed: int) -> np.ndarray:
    """B uniformly random packed sequences of length N, shape (B, ceil(N/64)) uint64."""
    rng = np.random.default_rng(seed)
    W = words_for(N)
    a = rng.integers(0, 1 << 63, size=(B, W), dtype=np.int64).astype(np.uint64)
    a ^= rng.integers(0, 2, size=(B, W), dtype=np.int64).astype(np.uint64) << np.uint64(63)
    tail = N - 64 * (W - 1)
    if tail < 64:
        a[:, W - 1] &= np.uint64((1 << tail) - 1)
    return a


def sequence_edge_cases(N: int) -> np.ndarray:
    """All +1, all -1, alternating, and one-hot patterns, packed."""
    W = words_for(N)
    rows = []
    for pattern in ("ones", "zeros", "alt0", "alt1", "first", "last"):
        bits = np.zeros(N, dtype=bool)
        if pattern == "ones":
            bits[:] = True
        elif pattern == "alt0":
            bits[0::2] = True
        elif pattern == "alt1":
            bits[1::2] = True
        elif pattern == "first":
            bits[0] = True
        elif pattern == "last":
            bits[N - 1] = True
        w = np.zeros(W, dtype=np.uint64)
        for i in np.nonzero(bits)[0]:
            w[i // 64] |= np.uint64(1) << np.uint64(i % 64)
        rows.append(w)
    return np.stack(rows)


@dataclass(frozen=True)
class Instance:
    """One MTS problem: length N, population K, Philox seed/instance, step budget."""

    N: int
    K: int
    seed: int
    instance: int
    max_steps: int
    target_E: int = -1


def plain_n24() -> dict:
    """Plain MTS, one instance, N=24, K=100, seed 0, 2,000 generations."""
    return {"N": 24, "K": 100, "seed": 0, "replicas": 1, "max_generations": 2000}


def replicas_n64(replicas: int = 1024, max_steps: int = 100_000) -> dict:
    """N=64 (one uint64 word), 1,024 independent replicas (Philox streams 0..1023), K=100,
    10^5 tabu steps per replica."""
    return {"N": 64, "K": 100, "seed": 0, "replicas": replicas, "max_steps": max_steps}


def sweep_n92_120(max_steps: int = 1_000_000) -> list[dict]:
    """N = 92, 96, ..., 120 (two uint64 words), one K=100 population per replica."""
    return [{"N": N, "K": 100, "seed": 0, "max_steps": max_steps} for N in range(92, 121, 4)]


def uneven_batch(count: int = 512, seed: int = 7, steps_per_n2: int = 10) -> list[Instance]:
    """Uneven instances: N ~ U{40..127}, K ~ U{50..200}, budget = steps_per_n2 * N^2 steps."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(40, 128, size=count)
    Ks = rng.integers(50, 201, size=count)
    return [Instance(int(n), int(k), seed, i, int(steps_per_n2 * n * n)) for i, (n, k) in enumerate(zip(Ns, Ks))]


@dataclass(frozen=True)
class Request:
    arrival_s: float
    N: int
    K: int
    seed: int
    target_mode: bool
    max_steps: int


def poisson_requests(count: int = 20_000, rate_per_s: float = 200.0, seed: int = 11,
                     cap_steps: int = 100_000, target_cap_steps: int = 10_000_000) -> list[Request]:
    """Poisson arrivals (exponential gaps, mean 1/rate), N ~ U{32..160}, K=100, and a fair
    coin between target mode (safety cap) and a plain step cap."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps)
    Ns = rng.integers(32, 161, size=count)
    modes = rng.integers(0, 2, size=count).astype(bool)
    out = []
    for i in range(count):
        tm = bool(modes[i])
        out.append(Request(float(arrivals[i]), int(Ns[i]), 100, i, tm, target_cap_steps if tm else cap_steps))
    return out
