"""ctypes declarations of liblabs.so (include/labs.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblabs.so")

LABS_OK = 0
LABS_EINVAL = 1
LABS_ENOMEM = 2
LABS_ECUDA = 3
LABS_ETIMEOUT = 4
LABS_EBUSY = 5
LABS_ENOTREADY = 6
LABS_ECANCELED = 7
LABS_ENOTFOUND = 8
STATUS_NAMES = {
    LABS_OK: "LABS_OK", LABS_EINVAL: "LABS_EINVAL", LABS_ENOMEM: "LABS_ENOMEM",
    LABS_ECUDA: "LABS_ECUDA", LABS_ETIMEOUT: "LABS_ETIMEOUT", LABS_EBUSY: "LABS_EBUSY",
    LABS_ENOTREADY: "LABS_ENOTREADY", LABS_ECANCELED: "LABS_ECANCELED",
    LABS_ENOTFOUND: "LABS_ENOTFOUND",
}
MAX_N = 256
MAX_W = 4
MAX_K = 1024
REPLACE_RANDOM = 0
REPLACE_WORST = 1
RUN_BUDGET = 0
RUN_REACHED = 1
RUN_STOPPED = 2
RUN_BADSTATE = 3
RUN_SYNC_LOST = 4

# Every symbol include/labs.h declares.
EXPORTED = [
    "labs_last_error", "labs_version", "labs_energy_batch", "labs_tabu_run",
    "labs_mts_launch", "labs_mts_run", "labs_autotune", "labs_batch_create", "labs_batch_launch",
    "labs_batch_device_results", "labs_batch_results", "labs_batch_get_mapping",
    "labs_batch_destroy", "labs_mts_batch_run", "labs_mts_run_static", "labs_serve_create",
    "labs_serve_submit", "labs_serve_poll", "labs_serve_cancel", "labs_serve_stats_get",
    "labs_serve_destroy", "labs_skew_deviation_batch", "labs_philox_batch",
    "labs_mts_state_bytes", "labs_mts_resume", "labs_results_decode",
]
STATIC_MAX_REPLICAS = 4096
VARIANT_UNIFORM_CROSSOVER = 1
VARIANT_FIX_FIRST_SPIN = 2
VARIANT_SKEW = 4
ORDER_LPT = 0
ORDER_GIVEN = 1


class LabsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


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
        ("glf", ctypes.c_int32),
        ("d_trace", ctypes.c_void_p),
        ("trace_cap", ctypes.c_int64),
        ("variant", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class DeviceResult(ctypes.Structure):
    _fields_ = [
        ("seq", ctypes.c_uint64 * MAX_W),
        ("E", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("generations", ctypes.c_int64),
        ("steps", ctypes.c_int64),
        ("trace_len", ctypes.c_int64),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("seq", ctypes.c_uint64 * MAX_W),
        ("E", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("F", ctypes.c_double),
        ("generations", ctypes.c_int64),
        ("steps", ctypes.c_int64),
        ("flip_evals", ctypes.c_int64),
        ("trace_len", ctypes.c_int64),
        ("instance", ctypes.c_uint64),
        ("seconds", ctypes.c_double),
        ("status", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class TabuOpts(ctypes.Structure):
    _fields_ = [
        ("max_iter", ctypes.c_int32),
        ("generation", ctypes.c_uint32),
        ("first_instance", ctypes.c_uint64),
        ("trace_cap", ctypes.c_int64),
        ("variant", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class Instance(ctypes.Structure):
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
        ("seed", ctypes.c_uint64),
        ("instance", ctypes.c_uint64),
    ]


class Mapping(ctypes.Structure):
    _fields_ = [
        ("warps_per_block", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("warps_per_seq", ctypes.c_int32),
    ]


class ServeOpts(ctypes.Structure):
    _fields_ = [
        ("max_slots", ctypes.c_int32),
        ("max_N", ctypes.c_int32),
        ("max_K", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("quantum_steps", ctypes.c_int64),
        ("queue_capacity", ctypes.c_int64),
        ("hbm_budget_bytes", ctypes.c_int64),
        ("quantum_timeout_ms", ctypes.c_int64),
        ("quantum_us", ctypes.c_int64),
        ("warps_per_request", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class ServeStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("canceled", ctypes.c_int64),
        ("quanta", ctypes.c_int64),
        ("running", ctypes.c_int64),
        ("pending", ctypes.c_int64),
        ("flip_evals", ctypes.c_int64),
        ("gpu_seconds", ctypes.c_double),
        ("failed", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("deferred_slots", ctypes.c_int64),
        ("deferred_smem", ctypes.c_int64),
        ("deferred_hbm", ctypes.c_int64),
        ("arena_bytes", ctypes.c_int64),
        ("arena_used_bytes", ctypes.c_int64),
        ("pair_quanta", ctypes.c_int64),
    ]


assert ctypes.sizeof(DeviceResult) == 64
assert ctypes.sizeof(Instance) == 64

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads liblabs.so; raises if it has not been built (there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
            )
        L = ctypes.CDLL(path)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        L.labs_last_error.restype = ctypes.c_char_p
        L.labs_last_error.argtypes = []
        L.labs_version.restype = i32
        L.labs_version.argtypes = []
        L.labs_energy_batch.restype = i32
        L.labs_energy_batch.argtypes = [vp, i32, i64, vp, vp, vp]
        L.labs_tabu_run.restype = i32
        L.labs_tabu_run.argtypes = [vp, i32, i64, u64, ctypes.POINTER(TabuOpts), vp, vp, vp, vp, vp]
        L.labs_mts_launch.restype = i32
        L.labs_mts_launch.argtypes = [ctypes.POINTER(Params), u64, u64, i64, vp, vp, vp]
        L.labs_mts_run.restype = i32
        L.labs_mts_run.argtypes = [ctypes.POINTER(Params), u64, u64, i64, ctypes.POINTER(Result), vp]
        IP, MP, RP = ctypes.POINTER(Instance), ctypes.POINTER(Mapping), ctypes.POINTER(Result)
        L.labs_autotune.restype = i32
        L.labs_autotune.argtypes = [IP, i64, vp, MP]
        L.labs_batch_create.restype = i32
        L.labs_batch_create.argtypes = [IP, i64, MP, vp, ctypes.POINTER(vp)]
        L.labs_batch_launch.restype = i32
        L.labs_batch_launch.argtypes = [vp, vp]
        L.labs_batch_device_results.restype = i32
        L.labs_batch_device_results.argtypes = [vp, ctypes.POINTER(vp)]
        L.labs_batch_results.restype = i32
        L.labs_batch_results.argtypes = [vp, RP, vp]
        L.labs_batch_get_mapping.restype = i32
        L.labs_batch_get_mapping.argtypes = [vp, MP]
        L.labs_batch_destroy.restype = i32
        L.labs_batch_destroy.argtypes = [vp]
        L.labs_mts_batch_run.restype = i32
        L.labs_mts_batch_run.argtypes = [IP, i64, MP, RP, vp]
        L.labs_serve_create.restype = vp
        L.labs_serve_create.argtypes = [ctypes.POINTER(ServeOpts)]
        L.labs_serve_submit.restype = i32
        L.labs_serve_submit.argtypes = [vp, IP, ctypes.POINTER(u64)]
        L.labs_serve_poll.restype = i32
        L.labs_serve_poll.argtypes = [vp, u64, RP]
        L.labs_serve_cancel.restype = i32
        L.labs_serve_cancel.argtypes = [vp, u64]
        L.labs_serve_stats_get.restype = i32
        L.labs_serve_stats_get.argtypes = [vp, ctypes.POINTER(ServeStats)]
        L.labs_serve_destroy.restype = i32
        L.labs_serve_destroy.argtypes = [vp]
        L.labs_skew_deviation_batch.restype = i32
        L.labs_skew_deviation_batch.argtypes = [vp, i32, i64, vp, vp]
        L.labs_mts_state_bytes.restype = i64
        L.labs_mts_state_bytes.argtypes = [i32, i32]
        L.labs_mts_resume.restype = i32
        L.labs_mts_resume.argtypes = [ctypes.POINTER(Params), u64, u64, i64, vp, i32, vp, vp, vp]
        L.labs_philox_batch.restype = i32
        L.labs_philox_batch.argtypes = [u64, vp, i64, vp, vp]
        L.labs_results_decode.restype = i32
        L.labs_results_decode.argtypes = [vp, i64, i32, u64, RP]
        L.labs_mts_run_static.restype = i32
        L.labs_mts_run_static.argtypes = [ctypes.POINTER(Params), u64, u64, i64, RP, vp]
        _lib = L
        return L


def check(rc: int) -> None:
    if rc != LABS_OK:
        msg = load().labs_last_error()
        raise LabsError(rc, msg.decode() if msg else "")
