"""labs_mts_run_static: the Memetic-Tabu run for callers that cannot allocate
memory (an application that owns the GPU memory budget, a latency-critical
loop that cannot wait on cudaMalloc/cudaFree, a hard device-memory quota).
Its scratch is a fixed array inside the library shared by every call, so
this file checks, through the C ABI, that consecutive calls give exactly
what labs_mts_run gives -- including after a call that left the global
termination flag set -- and that over-large requests are refused.  It runs
last so that a failure here never hides the other tests."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_00987_gb300 import _native

    torch.cuda.init()
    return _native.load()


def run(lib, fn, P, seed, first, replicas):
    from paper_2504_00987_gb300 import _native as nat

    res = (nat.Result * replicas)()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(ctypes.byref(P), seed, first, replicas, res, stream)
    assert rc == nat.LABS_OK, lib.labs_last_error()
    return [(r.E, list(r.seq), r.steps, r.generations, r.status, r.instance, r.N, r.flip_evals, r.F)
            for r in res]


def test_static_matches_allocating_run(lib):
    from paper_2504_00987_gb300 import _native as nat
    from paper_2504_00987_gb300.api import make_params

    # A call with a reachable target and the global termination flag on leaves the flag set.
    P0 = make_params(20, 30, target_E=30, max_generations=400, glf=True)
    first = run(lib, "labs_mts_run_static", P0, 5, 0, 64)
    assert any(s == nat.RUN_REACHED for (_, _, _, _, s, *_rest) in first)
    # Two calls in a row, each compared with labs_mts_run on the same arguments.
    P1 = make_params(64, 50, target_E=0, max_steps=20_000, glf=True)  # unreachable target
    assert run(lib, "labs_mts_run_static", P1, 7, 10, 300) == run(lib, "labs_mts_run", P1, 7, 10, 300)
    P2 = make_params(100, 40, max_steps=8_000, replace_policy=nat.REPLACE_WORST)
    assert run(lib, "labs_mts_run_static", P2, 3, 0, nat.STATIC_MAX_REPLICAS) == \
        run(lib, "labs_mts_run", P2, 3, 0, nat.STATIC_MAX_REPLICAS)


def test_static_rejects_more_replicas_than_its_scratch(lib):
    from paper_2504_00987_gb300 import _native as nat
    from paper_2504_00987_gb300.api import make_params

    P = make_params(64, 10, max_steps=100)
    res = (nat.Result * 1)()
    rc = lib.labs_mts_run_static(ctypes.byref(P), 0, 0, nat.STATIC_MAX_REPLICAS + 1, res, None)
    assert rc == nat.LABS_EINVAL
    assert b"static scratch maximum" in lib.labs_last_error()


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so.13"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("no libcudart to read the default memory pool from")


def test_static_allocates_nothing(lib):
    """The property the entry point exists for: a warmed-up call takes no
    memory from the device's default pool (where labs_mts_run's
    cudaMallocAsync scratch comes from) and no device memory at all
    (cudaMemGetInfo's free bytes do not move).  labs_mts_run on the same
    arguments is the control: it raises the pool's high-water mark."""
    from paper_2504_00987_gb300.api import make_params

    rt = _cudart()
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used_high = 8  # cudaMemPoolAttrUsedMemHigh

    def reset_high():
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, used_high, ctypes.byref(zero)) == 0

    def high():
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, used_high, ctypes.byref(v)) == 0
        return v.value

    P = make_params(64, 40, max_steps=4_000, glf=True)
    run(lib, "labs_mts_run_static", P, 1, 0, 256)  # loads the module and places the array
    torch.cuda.synchronize()
    reset_high()
    base = high()
    free0 = torch.cuda.mem_get_info()[0]
    run(lib, "labs_mts_run_static", P, 2, 0, 256)
    torch.cuda.synchronize()
    assert high() == base
    assert torch.cuda.mem_get_info()[0] == free0
    run(lib, "labs_mts_run", P, 2, 0, 256)  # control: this one allocates its scratch
    assert high() > base
