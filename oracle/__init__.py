"""CPU oracle for the LABS memetic tabu search (arXiv 2504.00987).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and ``paper_2504_00987_gb300``) never imports it, and this
package imports nothing from the product.

The arithmetic lives in ``labs_oracle.c`` (plain C, see its header for the
passage each function follows); this module only loads it with ``ctypes`` and
marshals numpy arrays.  The pure-Python helpers below (hex decoding of the
paper's Table II format, the Philox constants of the RNG contract) hold no
method arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "labs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblabs_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_N = 256
MAX_W = 4
REPLACE_RANDOM = 0
REPLACE_WORST = 1
VARIANT_UNIFORM_CROSSOVER = 1
VARIANT_FIX_FIRST_SPIN = 2
VARIANT_SKEW = 4  # odd N: skew-symmetric sequences only (Sec. II.C)
STATUS_BUDGET = 0
STATUS_REACHED = 1
P_COMB_U32 = 3865470566  # floor(0.9 * 2^32), Sec. III.A: p_comb = 0.9


def p_mut_u32(N: int) -> int:
    """floor(2^32 / N): the per-bit mutation threshold for p_mutate = 1/N (Sec. III.A)."""
    return (1 << 32) // N


def build(force: bool = False) -> str:
    """Compile ``labs_oracle.c`` with gcc into ``liblabs_oracle.so``."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "labs_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-Wall", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("p_comb_u32", ctypes.c_uint32),
        ("p_mut_u32", ctypes.c_uint32),
        ("replace_policy", ctypes.c_int32),
        ("target_E", ctypes.c_int32),
        ("max_generations", ctypes.c_int64),
        ("max_steps", ctypes.c_int64),
        ("max_iter", ctypes.c_int32),
        ("variant", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("seq", ctypes.c_uint64 * MAX_W),
        ("E", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("generations", ctypes.c_int64),
        ("steps", ctypes.c_int64),
    ]


class GenLog(ctypes.Structure):
    _fields_ = [
        ("g", ctypes.c_int32),
        ("crossover", ctypes.c_int32),
        ("p1", ctypes.c_int32),
        ("p2", ctypes.c_int32),
        ("cut", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("min_tabu", ctypes.c_int32),
        ("max_tabu", ctypes.c_int32),
        ("replace", ctypes.c_int32),
        ("E_child", ctypes.c_int32),
        ("steps", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("pre_mut", ctypes.c_uint64 * MAX_W),
        ("pre_tabu", ctypes.c_uint64 * MAX_W),
        ("post_tabu", ctypes.c_uint64 * MAX_W),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # LABS_ORACLE_LIB: a library built from a modified copy of labs_oracle.c
            # (tests/test_oracle_mutants.py plants mistakes that way)
            L = ctypes.CDLL(os.environ.get("LABS_ORACLE_LIB") or build())
            P = ctypes.POINTER
            u64p, i32p, i64p, u32p = (
                P(ctypes.c_uint64),
                P(ctypes.c_int32),
                P(ctypes.c_int64),
                P(ctypes.c_uint32),
            )
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox4x32_batch.argtypes = [u32p, ctypes.c_int64, ctypes.c_uint64, u32p]
            L.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
            L.orc_energy.argtypes = [u64p, ctypes.c_int32, i32p]
            L.orc_energy.restype = ctypes.c_int64
            L.orc_neighbour_energies.argtypes = [u64p, ctypes.c_int32, i32p]
            L.orc_tabu_run.argtypes = [
                u64p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, u64p, i32p, i32p,
                ctypes.c_int64, i64p,
            ]
            L.orc_tabu_run.restype = ctypes.c_int64
            L.orc_tabu_run_v.argtypes = [
                u64p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, u64p, i32p, i32p,
                ctypes.c_int64, i64p,
            ]
            L.orc_tabu_run_v.restype = ctypes.c_int64
            L.orc_mts_run.argtypes = [
                P(Params), ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, P(Result), i32p,
                ctypes.c_int64, i64p, P(GenLog), ctypes.c_int64, i64p,
            ]
            L.orc_mts_run_many.argtypes = [
                P(Params), ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                P(Result),
            ]
            L.orc_bruteforce.argtypes = [ctypes.c_int32, i32p, i64p, u64p]
            L.orc_bruteforce_skew.argtypes = [ctypes.c_int32, i32p, i64p]
            L.orc_bruteforce_mt.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i64p]
            L.orc_non_skew_pairs.argtypes = [u64p, ctypes.c_int32]
            L.orc_skew_deviation.argtypes = [u64p, ctypes.c_int32]
            L.orc_skew_deviation_mode.argtypes = [u64p, ctypes.c_int32, ctypes.c_int32]
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def words_for(N: int) -> int:
    return (N + 63) // 64


def _words(seq, N: int) -> np.ndarray:
    w = np.zeros(MAX_W, dtype=np.uint64)
    a = np.asarray(seq, dtype=np.uint64).ravel()
    w[: len(a)] = a
    return w


# ---------------------------------------------------------------------------
# Table II format: hexadecimal, most significant bit first, zeros appended to
# reach a multiple of 4 bits.  Used only to read the paper's printed rows.
# ---------------------------------------------------------------------------


def hex_to_words(hexstr: str, N: int) -> np.ndarray:
    bits = "".join(f"{int(c, 16):04b}" for c in hexstr.strip())
    if len(bits) < N or any(b != "0" for b in bits[N:]):
        raise ValueError("hex string does not encode N spins with a zero tail")
    w = np.zeros(words_for(N), dtype=np.uint64)
    for i, b in enumerate(bits[:N]):
        if b == "1":
            w[i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return w


def words_to_spins(words, N: int) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint64)
    return np.array([1 if (int(w[i // 64]) >> (i % 64)) & 1 else -1 for i in range(N)], dtype=np.int64)


def spins_to_words(s) -> np.ndarray:
    s = np.asarray(s)
    N = len(s)
    w = np.zeros(words_for(N), dtype=np.uint64)
    for i in range(N):
        if s[i] > 0:
            w[i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return w


# ---------------------------------------------------------------------------
# Thin wrappers
# ---------------------------------------------------------------------------


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint64).copy()
    k = np.asarray(key, dtype=np.uint64).copy()
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c, ctypes.c_uint64), _ptr(k, ctypes.c_uint64), _ptr(out, ctypes.c_uint64))
    return out


def energy(words, N: int, with_C: bool = False):
    w = _words(words, N)
    C = np.zeros(max(N - 1, 1), dtype=np.int32)
    E = lib().orc_energy(_ptr(w, ctypes.c_uint64), N, _ptr(C, ctypes.c_int32))
    if E < 0:
        raise ValueError("bad arguments")
    return (int(E), C[: N - 1].copy()) if with_C else int(E)


def neighbour_energies(words, N: int) -> np.ndarray:
    w = _words(words, N)
    out = np.zeros(N, dtype=np.int32)
    if lib().orc_neighbour_energies(_ptr(w, ctypes.c_uint64), N, _ptr(out, ctypes.c_int32)) != 0:
        raise ValueError("bad arguments")
    return out


def tabu_run(start, N: int, seed: int, instance: int, g: int = 0, max_iter: int = -1,
             step_budget: int = -1, incremental: bool = True, trace_cap: int = 0, variant: int = 0):
    """One tabu search (Algorithm 2).  Returns (best_words, best_E, steps, trace[n,4])."""
    w = _words(start, N)
    best = np.zeros(MAX_W, dtype=np.uint64)
    bestE = np.zeros(1, dtype=np.int32)
    tr = np.zeros((max(trace_cap, 1), 4), dtype=np.int32)
    tl = np.zeros(1, dtype=np.int64)
    steps = lib().orc_tabu_run_v(
        _ptr(w, ctypes.c_uint64), N, seed, instance, g, max_iter, step_budget, int(incremental),
        variant, _ptr(best, ctypes.c_uint64), _ptr(bestE, ctypes.c_int32),
        _ptr(tr, ctypes.c_int32) if trace_cap > 0 else None, trace_cap, _ptr(tl, ctypes.c_int64),
    )
    if steps < 0:
        raise ValueError("bad arguments")
    return best[: words_for(N)].copy(), int(bestE[0]), int(steps), tr[: int(tl[0])].copy()


def make_params(N: int, K: int = 100, *, p_comb_u32: int = P_COMB_U32, p_mut: int | None = None,
                replace_policy: int = REPLACE_RANDOM, target_E: int = -1,
                max_generations: int = -1, max_steps: int = -1, max_iter: int = -1,
                variant: int = 0) -> Params:
    if p_mut is None:  # 1/(number of spins mutation acts on)
        p_mut = p_mut_u32((N + 1) // 2 if variant & VARIANT_SKEW else N)
    return Params(N, K, p_comb_u32, p_mut, replace_policy, target_E, max_generations, max_steps,
                  max_iter, variant)


def mts_run(params: Params, seed: int, instance: int = 0, incremental: bool = True,
            trace_cap: int = 0, genlog_cap: int = 0):
    """Algorithm 1 for one replica.  Returns (result dict, trace[n,4], genlog list)."""
    res = Result()
    tr = np.zeros((max(trace_cap, 1), 4), dtype=np.int32)
    tl = np.zeros(1, dtype=np.int64)
    gl = (GenLog * max(genlog_cap, 1))()
    gll = np.zeros(1, dtype=np.int64)
    rc = lib().orc_mts_run(
        ctypes.byref(params), seed, instance, int(incremental), ctypes.byref(res),
        _ptr(tr, ctypes.c_int32) if trace_cap > 0 else None, trace_cap, _ptr(tl, ctypes.c_int64),
        gl if genlog_cap > 0 else None, genlog_cap, _ptr(gll, ctypes.c_int64),
    )
    if rc != 0:
        raise ValueError("bad arguments")
    return _result_dict(res, params.N), tr[: int(tl[0])].copy(), [gl[i] for i in range(int(gll[0]))]


def mts_run_many(params: Params, seed: int, first_instance: int, replicas: int, threads: int):
    res = (Result * max(replicas, 1))()
    if lib().orc_mts_run_many(ctypes.byref(params), seed, first_instance, replicas, threads, res) != 0:
        raise ValueError("bad arguments")
    return [_result_dict(res[i], params.N) for i in range(replicas)]


def _result_dict(r: Result, N: int) -> dict:
    return {
        "seq": np.array(list(r.seq)[: words_for(N)], dtype=np.uint64),
        "E": int(r.E),
        "status": int(r.status),
        "generations": int(r.generations),
        "steps": int(r.steps),
    }


def bruteforce(N: int):
    """Exhaustive optimum over all 2^N sequences: (E_min, number of minimisers, one minimiser)."""
    E = np.zeros(1, dtype=np.int32)
    n = np.zeros(1, dtype=np.int64)
    a = np.zeros(1, dtype=np.uint64)
    if lib().orc_bruteforce(N, _ptr(E, ctypes.c_int32), _ptr(n, ctypes.c_int64), _ptr(a, ctypes.c_uint64)) != 0:
        raise ValueError("bad arguments")
    return int(E[0]), int(n[0]), a.copy()



def philox4x32_batch(counters, seed: int):
    """Philox4x32-10 words at each row of counters (B x 4 uint32) under key (seed lo, seed hi)."""
    c = np.ascontiguousarray(counters, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().orc_philox4x32_batch(_ptr(c, ctypes.c_uint32), c.shape[0], seed, _ptr(out, ctypes.c_uint32))
    return out


def bruteforce_mt(N: int, threads: int):
    """Exhaustive minimum over all 2^N sequences on `threads` threads (8 <= N <= 40):
    (E_min, number of minimisers)."""
    E = np.zeros(1, dtype=np.int32)
    n = np.zeros(1, dtype=np.int64)
    if lib().orc_bruteforce_mt(N, threads, _ptr(E, ctypes.c_int32), _ptr(n, ctypes.c_int64)) != 0:
        raise ValueError("8 <= N <= 40 and threads >= 1")
    return int(E[0]), int(n[0])


def bruteforce_skew(N: int):
    """Exhaustive minimum over the skew-symmetric sequences of odd N <= 45:
    (E_min, number of minimisers)."""
    E = np.zeros(1, dtype=np.int32)
    n = np.zeros(1, dtype=np.int64)
    if lib().orc_bruteforce_skew(N, _ptr(E, ctypes.c_int32), _ptr(n, ctypes.c_int64)) != 0:
        raise ValueError("odd N in 3..45 only")
    return int(E[0]), int(n[0])

def non_skew_pairs(words, N: int) -> int:
    w = _words(words, N)
    return int(lib().orc_non_skew_pairs(_ptr(w, ctypes.c_uint64), N))


def skew_deviation(words, N: int, mode: int | None = None) -> int:
    """d(S) of Appendix A.  mode: 1 rotations (odd N), 2 insertion, 4 deletion (even N)."""
    w = _words(words, N)
    if mode is None:
        return int(lib().orc_skew_deviation(_ptr(w, ctypes.c_uint64), N))
    return int(lib().orc_skew_deviation_mode(_ptr(w, ctypes.c_uint64), N, mode))
