"""torch-facing wrappers of the C ABI (argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

import torch

from . import _native as nat

P_COMB_U32 = 3865470566  # floor(0.9 * 2^32): p_comb = 0.9 (Sec. III.A)


def p_mut_u32(N: int) -> int:
    """floor(2^32 / N): per-bit mutation threshold for p_mutate = 1/N (Sec. III.A)."""
    return (1 << 32) // N


def words_for(N: int) -> int:
    return (N + 63) // 64


def version() -> int:
    return int(nat.load().labs_version())


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p | None:
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_seqs(seqs: torch.Tensor, N: int) -> torch.Tensor:
    if not seqs.is_cuda:
        raise ValueError("sequences must be a CUDA tensor")
    if seqs.dtype not in (torch.int64, torch.uint64):
        raise ValueError("sequences must be int64/uint64 words")
    if seqs.dim() != 2 or seqs.shape[1] != words_for(N):
        raise ValueError(f"sequences must have shape (B, {words_for(N)})")
    return seqs.contiguous()


def energy_batch(seqs: torch.Tensor, N: int, with_C: bool = False, stream=None):
    """E (Eq. 2) of each packed sequence, and optionally C_1..C_{N-1} (Eq. 1)."""
    seqs = _check_seqs(seqs, N)
    B = seqs.shape[0]
    E = torch.empty(B, dtype=torch.int32, device=seqs.device)
    C = torch.empty((B, max(N - 1, 1)), dtype=torch.int32, device=seqs.device) if with_C else None
    nat.check(nat.load().labs_energy_batch(_ptr(seqs), N, B, _ptr(E), _ptr(C), _stream(stream)))
    return (E, C) if with_C else E


def skew_deviation_batch(seqs: torch.Tensor, N: int, stream=None) -> torch.Tensor:
    """d(S) of Appendix A (Eqs. 5-9) of each packed sequence."""
    seqs = _check_seqs(seqs, N)
    out = torch.empty(seqs.shape[0], dtype=torch.int32, device=seqs.device)
    nat.check(nat.load().labs_skew_deviation_batch(_ptr(seqs), N, seqs.shape[0], _ptr(out), _stream(stream)))
    return out


def philox_batch(counters: torch.Tensor, seed: int, stream=None) -> torch.Tensor:
    """Philox4x32-10 words of the randomness contract at B counters
    (instance, a, b, purpose): an int32/uint32 CUDA tensor of shape (B, 4)."""
    if not counters.is_cuda or counters.dtype not in (torch.int32, torch.uint32):
        raise ValueError("counters must be an int32/uint32 CUDA tensor")
    if counters.dim() != 2 or counters.shape[1] != 4:
        raise ValueError("counters must have shape (B, 4)")
    counters = counters.contiguous()
    out = torch.empty_like(counters)
    nat.check(nat.load().labs_philox_batch(seed, _ptr(counters), counters.shape[0], _ptr(out), _stream(stream)))
    return out


def tabu_run(start: torch.Tensor, N: int, seed: int, *, max_iter: int = -1, generation: int = 0,
             first_instance: int = 0, trace_cap: int = 0, variant: int = 0, stream=None) -> dict:
    """B independent tabu searches (Algorithm 2), one from each start sequence."""
    start = _check_seqs(start, N)
    B, dev = start.shape[0], start.device
    best = torch.empty_like(start)
    bestE = torch.empty(B, dtype=torch.int32, device=dev)
    steps = torch.empty(B, dtype=torch.int64, device=dev)
    trace = torch.zeros((B, trace_cap, 4), dtype=torch.int32, device=dev) if trace_cap > 0 else None
    opts = nat.TabuOpts(max_iter, generation, first_instance, trace_cap, variant, 0)
    nat.check(nat.load().labs_tabu_run(_ptr(start), N, B, seed, ctypes.byref(opts), _ptr(best),
                                       _ptr(bestE), _ptr(steps), _ptr(trace), _stream(stream)))
    return {"best": best, "bestE": bestE, "steps": steps, "trace": trace}


def make_params(N: int, K: int = 100, *, p_comb_u32: int = P_COMB_U32, p_mut: int = 0,
                replace_policy: int = nat.REPLACE_RANDOM, target_E: int = -1,
                max_generations: int = -1, max_steps: int = -1, max_iter: int = -1,
                glf: bool = False, trace: torch.Tensor | None = None, variant: int = 0) -> nat.Params:
    """labs_params; `trace` is an int32 CUDA tensor of shape (replicas, cap, 4) or None."""
    cap = 0 if trace is None else int(trace.shape[1])
    ptr = None if trace is None else trace.data_ptr()
    return nat.Params(N, K, p_comb_u32, p_mut, replace_policy, target_E, max_generations,
                      max_steps, max_iter, 1 if glf else 0, ptr, cap, variant, 0)


def mts_launch(params: nat.Params, seed: int, first_instance: int, replicas: int,
               out: torch.Tensor | None = None, glf_flag: torch.Tensor | None = None,
               device=None, stream=None) -> torch.Tensor:
    """Asynchronous launch of `replicas` MTS replicas.  Returns the (replicas, 8) int64
    device tensor holding one labs_device_result per replica (decode with
    decode_results)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = torch.empty((replicas, 8), dtype=torch.int64, device=dev)
    if params.glf and glf_flag is None:
        glf_flag = torch.zeros(1, dtype=torch.int32, device=out.device)
    nat.check(nat.load().labs_mts_launch(ctypes.byref(params), seed, first_instance, replicas,
                                         _ptr(out), _ptr(glf_flag), _stream(stream)))
    return out


def mts_state_bytes(N: int, K: int) -> int:
    """Bytes of one replica's resumable state record (labs_mts_state_bytes)."""
    n = nat.load().labs_mts_state_bytes(N, K)
    if n < 0:
        raise nat.LabsError(nat.LABS_EINVAL, nat.load().labs_last_error().decode())
    return int(n)


def mts_resume(params: nat.Params, seed: int, first_instance: int, replicas: int, state: torch.Tensor,
               resume: bool, out: torch.Tensor | None = None, glf_flag: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """mts_launch with a resumable state record per replica in `state` (a CUDA
    uint8 tensor of replicas * mts_state_bytes(N, K) bytes): start fresh
    (resume=False) or continue every replica from its record (resume=True);
    the records are rewritten at the end.  Returns the (replicas, 8) results."""
    need = replicas * mts_state_bytes(params.N, params.K)
    if not state.is_cuda or state.dtype != torch.uint8 or state.numel() < need or not state.is_contiguous():
        raise ValueError(f"state must be a contiguous CUDA uint8 tensor of at least {need} bytes")
    if out is None:
        out = torch.empty((replicas, 8), dtype=torch.int64, device=state.device)
    if params.glf and glf_flag is None:
        glf_flag = torch.zeros(1, dtype=torch.int32, device=out.device)
    nat.check(nat.load().labs_mts_resume(ctypes.byref(params), seed, first_instance, replicas, _ptr(state),
                                         1 if resume else 0, _ptr(out), _ptr(glf_flag), _stream(stream)))
    return out


def decode_results(out: torch.Tensor, N: int, first_instance: int = 0) -> list[dict]:
    """labs_device_result rows (from mts_launch / mts_resume) -> dicts, decoded on
    the host by labs_results_decode (merit factor, flip evaluations)."""
    h = out.detach().to("cpu").contiguous()
    if h.dtype != torch.int64 or h.dim() != 2 or h.shape[1] != 8:
        raise ValueError("device results must be an (n, 8) int64 tensor")
    n = h.shape[0]
    res = (nat.Result * max(n, 1))()
    nat.check(nat.load().labs_results_decode(ctypes.c_void_p(h.data_ptr()), n, N, first_instance, res))
    return _result_dicts(res, n, with_N=False)


def mts_run(params: nat.Params, seed: int, first_instance: int, replicas: int, stream=None) -> list[dict]:
    """Blocking run of `replicas` MTS replicas; results in host memory."""
    res = (nat.Result * max(replicas, 1))()
    nat.check(nat.load().labs_mts_run(ctypes.byref(params), seed, first_instance, replicas, res,
                                      _stream(stream)))
    return _result_dicts(res, replicas, with_N=False)


# ---------------------------------------------------------------- batches


def make_instance(N: int, K: int = 100, *, seed: int = 0, instance: int = 0, max_steps: int = -1,
                  max_generations: int = -1, target_E: int = -1, p_comb_u32: int = P_COMB_U32,
                  p_mut: int = 0, replace_policy: int = nat.REPLACE_RANDOM,
                  max_iter: int = -1, variant: int = 0) -> nat.Instance:
    return nat.Instance(N, K, p_comb_u32, p_mut, replace_policy, target_E, max_generations,
                        max_steps, max_iter, variant, seed, instance)


def _inst_array(instances):
    n = len(instances)
    arr = (nat.Instance * max(n, 1))()
    for i, x in enumerate(instances):
        arr[i] = x
    return arr, n


def _mapping(mapping):
    if mapping is None:
        return None
    if isinstance(mapping, nat.Mapping):
        return mapping
    return nat.Mapping(int(mapping["warps_per_block"]), int(mapping["blocks_per_sm"]),
                       int(mapping.get("order", nat.ORDER_LPT)), int(mapping.get("warps_per_seq", 1)))


def _mapping_dict(m: nat.Mapping) -> dict:
    return {"warps_per_block": m.warps_per_block, "blocks_per_sm": m.blocks_per_sm, "order": m.order,
            "warps_per_seq": max(1, m.warps_per_seq)}


def _result_dicts(res, n, with_N=True):
    """labs_result array -> list of dicts, converted column by column through a
    numpy view of the ctypes array (several times faster than per-field access)."""
    if n <= 0:
        return []
    a = np.ctypeslib.as_array(res)[:n]
    Ns = a["N"].tolist()
    seqs = a["seq"].tolist()
    out = [{"instance": i, "seq": q[: (N + 63) // 64], "E": E, "F": F, "status": st, "generations": g,
            "steps": sp, "flip_evals": fe, "trace_len": tl, "seconds": sec}
           for i, q, N, E, F, st, g, sp, fe, tl, sec in zip(
               *(a[k].tolist() if k not in ("seq", "N") else (seqs if k == "seq" else Ns)
                 for k in ("instance", "seq", "N", "E", "F", "status", "generations", "steps",
                           "flip_evals", "trace_len", "seconds")))]
    if with_N:
        for d, N in zip(out, Ns):
            d["N"] = N
    return out


def autotune(instances, stream=None) -> dict:
    """The mapping labs_autotune picks for these instances (cached per batch signature)."""
    arr, n = _inst_array(instances)
    m = nat.Mapping()
    nat.check(nat.load().labs_autotune(arr, n, _stream(stream), ctypes.byref(m)))
    return _mapping_dict(m)


class Batch:
    """A captured persistent launch over uneven instances (labs_batch_*)."""

    def __init__(self, instances, mapping=None, stream=None):
        arr, self.n = _inst_array(instances)
        self._h = ctypes.c_void_p()
        m = _mapping(mapping)
        nat.check(nat.load().labs_batch_create(arr, self.n, ctypes.byref(m) if m is not None else None,
                                               _stream(stream), ctypes.byref(self._h)))

    @property
    def mapping(self) -> dict:
        m = nat.Mapping()
        nat.check(nat.load().labs_batch_get_mapping(self._h, ctypes.byref(m)))
        return _mapping_dict(m)

    def launch(self, stream=None) -> None:
        nat.check(nat.load().labs_batch_launch(self._h, _stream(stream)))

    def results(self, stream=None) -> list[dict]:
        res = (nat.Result * max(self.n, 1))()
        nat.check(nat.load().labs_batch_results(self._h, res, _stream(stream)))
        return _result_dicts(res, self.n)

    def close(self) -> None:
        if self._h:
            nat.load().labs_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mts_batch_run(instances, mapping=None, stream=None) -> list[dict]:
    """Blocking: create, launch, collect and destroy a batch."""
    arr, n = _inst_array(instances)
    res = (nat.Result * max(n, 1))()
    m = _mapping(mapping)
    nat.check(nat.load().labs_mts_batch_run(arr, n, ctypes.byref(m) if m is not None else None, res,
                                            _stream(stream)))
    return _result_dicts(res, n)


# ---------------------------------------------------------------- serving


class Server:
    """Continuous-batching solve service (labs_serve_*): submit requests at any
    time, poll for results; the library's scheduler thread runs the GPU."""

    def __init__(self, max_slots: int = 1024, max_N: int = 256, max_K: int = 128,
                 warps_per_block: int = 4, quantum_steps: int = 2000,
                 queue_capacity: int = 1 << 20, hbm_budget_bytes: int = 0,
                 quantum_timeout_ms: int = 0, quantum_us: int = 0, warps_per_request: int = 0):
        opts = nat.ServeOpts(max_slots, max_N, max_K, warps_per_block, quantum_steps,
                             queue_capacity, hbm_budget_bytes, quantum_timeout_ms, quantum_us,
                             warps_per_request, 0)
        L = nat.load()
        self._h = L.labs_serve_create(ctypes.byref(opts))
        if not self._h:
            msg = L.labs_last_error()
            raise nat.LabsError(nat.LABS_EINVAL, msg.decode() if msg else "labs_serve_create failed")

    def submit(self, instance: nat.Instance) -> int:
        t = ctypes.c_uint64()
        nat.check(nat.load().labs_serve_submit(self._h, ctypes.byref(instance), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int) -> dict | None:
        """The result dict, or None while it is not ready."""
        r = (nat.Result * 1)()
        rc = nat.load().labs_serve_poll(self._h, ticket, r)
        if rc == nat.LABS_ENOTREADY:
            return None
        nat.check(rc)
        return _result_dicts(r, 1)[0]

    def cancel(self, ticket: int) -> None:
        nat.check(nat.load().labs_serve_cancel(self._h, ticket))

    def stats(self) -> dict:
        st = nat.ServeStats()
        nat.check(nat.load().labs_serve_stats_get(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in nat.ServeStats._fields_ if k != "pad"}

    def close(self) -> None:
        if self._h:
            nat.load().labs_serve_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
