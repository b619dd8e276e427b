"""The C ABI library builds, loads without a GPU and exports every function
include/labs.h declares; struct layouts of the binding match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(labs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_00987_gb300 import _build, _native

    _build.build()
    return _native.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["labs_energy_batch", "labs_tabu_run", "labs_mts_launch", "labs_mts_run",
                     "labs_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2504_00987_gb300 import _native

    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"
    assert sorted(_native.EXPORTED) == sorted(declared_functions())


def test_version_and_error_string_without_gpu(lib):
    assert lib.labs_version() == 100
    assert lib.labs_last_error() == b""


def test_argument_errors_without_gpu(lib):
    """Argument checks run before any device work, so they answer on a CPU machine."""
    from paper_2504_00987_gb300 import _native as nat

    assert lib.labs_energy_batch(None, 2, 1, None, None, None) == nat.LABS_EINVAL
    assert b"N=2" in lib.labs_last_error()
    assert lib.labs_energy_batch(None, 257, 1, None, None, None) == nat.LABS_EINVAL
    assert lib.labs_energy_batch(None, 64, -1, None, None, None) == nat.LABS_EINVAL
    assert lib.labs_energy_batch(None, 64, 0, None, None, None) == nat.LABS_OK  # empty batch
    P = nat.Params(64, 100, 0, 0, 0, -1, -1, -1, -1, 0, None, 0, 0, 0)  # no budget at all
    res = (nat.Result * 1)()
    assert lib.labs_mts_run(ctypes.byref(P), 0, 0, 1, res, None) == nat.LABS_EINVAL
    assert b"unbounded" in lib.labs_last_error()
    P.max_steps, P.max_iter = 100, 0  # steps never advance
    assert lib.labs_mts_run(ctypes.byref(P), 0, 0, 1, res, None) == nat.LABS_EINVAL
    P.max_iter, P.K = -1, 0
    assert lib.labs_mts_run(ctypes.byref(P), 0, 0, 1, res, None) == nat.LABS_EINVAL
    P.K, P.replace_policy = 100, 7
    assert lib.labs_mts_run(ctypes.byref(P), 0, 0, 1, res, None) == nat.LABS_EINVAL
    P.replace_policy = 0
    assert lib.labs_mts_run(ctypes.byref(P), 0, 2**32 - 1, 2, res, None) == nat.LABS_EINVAL
    assert lib.labs_mts_run(ctypes.byref(P), 0, 0, 0, res, None) == nat.LABS_OK  # no replicas
    P.variant = 8  # no such flag
    assert lib.labs_mts_run(ctypes.byref(P), 0, 0, 1, res, None) == nat.LABS_EINVAL
    assert b"variant" in lib.labs_last_error()
    assert lib.labs_mts_run_static(ctypes.byref(P), 0, 0, 1, res, None) == nat.LABS_EINVAL
    P.variant = nat.VARIANT_SKEW  # N = 64 is even
    assert lib.labs_mts_run(ctypes.byref(P), 0, 0, 1, res, None) == nat.LABS_EINVAL
    assert b"odd N" in lib.labs_last_error()
    P.variant = 0
    opts = nat.TabuOpts(-2, 0, 0, 0, 0, 0)
    assert lib.labs_tabu_run(None, 64, 1, 0, ctypes.byref(opts), None, None, None, None, None) == nat.LABS_EINVAL


def test_struct_sizes():
    from paper_2504_00987_gb300 import _native as nat

    assert ctypes.sizeof(nat.DeviceResult) == 64
    assert ctypes.sizeof(nat.Params) == 4 * 6 + 8 * 2 + 4 * 2 + 8 + 8 + 8
    assert ctypes.sizeof(nat.TabuOpts) == 32


def test_no_oracle_in_product():
    """The product package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2504_00987_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "labs_oracle" not in text, f


def test_resume_state_size_and_argument_errors_without_gpu(lib):
    from paper_2504_00987_gb300 import _native as nat

    # 80-byte header + K (NW + 1) 32-bit words, padded to 16 bytes
    assert lib.labs_mts_state_bytes(64, 100) == 80 + 1200
    assert lib.labs_mts_state_bytes(65, 7) == 80 + 144
    assert lib.labs_mts_state_bytes(256, 3) == 80 + 112
    assert lib.labs_mts_state_bytes(2, 10) == -1 and b"N=2" in lib.labs_last_error()
    assert lib.labs_mts_state_bytes(64, 0) == -1
    P = nat.Params(64, 100, 0, 0, 0, -1, 10, -1, -1, 0, None, 0, 0, 0)
    assert lib.labs_mts_resume(ctypes.byref(P), 0, 0, 4, None, 0, None, None, None) == nat.LABS_EINVAL
    assert b"d_state" in lib.labs_last_error()
    P.trace_cap, P.d_trace = 4, 16  # any non-NULL trace is refused first
    assert lib.labs_mts_resume(ctypes.byref(P), 0, 0, 4, None, 0, None, None, None) == nat.LABS_EINVAL
    assert b"trace" in lib.labs_last_error()


def test_batch_argument_errors_without_gpu(lib):
    from paper_2504_00987_gb300 import _native as nat

    arr = (nat.Instance * 2)()
    arr[0] = nat.Instance(64, 100, 0, 0, 0, -1, -1, 100, -1, 0, 0, 0)
    arr[1] = nat.Instance(64, 100, 0, 0, 0, -1, -1, -1, -1, 0, 0, 1)  # unbounded
    m = nat.Mapping()
    assert lib.labs_autotune(arr, 2, None, ctypes.byref(m)) == nat.LABS_EINVAL
    assert b"instance 1" in lib.labs_last_error()
    arr[1].max_steps, arr[1].variant = 10, 16
    assert lib.labs_autotune(arr, 2, None, ctypes.byref(m)) == nat.LABS_EINVAL
    assert b"variant" in lib.labs_last_error()
    arr[1].N, arr[1].variant = 63, nat.VARIANT_SKEW  # skew-symmetric runs are not batched
    assert lib.labs_autotune(arr, 2, None, ctypes.byref(m)) == nat.LABS_EINVAL
    assert b"SKEW" in lib.labs_last_error()
    arr[1].N, arr[1].max_steps, arr[1].variant = 64, -1, 0
    h = ctypes.c_void_p()
    bad_map = nat.Mapping(3, 1, 0, 0)
    arr[1].max_steps = 10
    assert lib.labs_batch_create(arr, 2, ctypes.byref(bad_map), None, ctypes.byref(h)) == nat.LABS_EINVAL
    for bad_map in (nat.Mapping(1, 1, 0, 2), nat.Mapping(4, 1, 0, 3)):  # a pair needs 2+ warps; 1 or 2
        assert lib.labs_batch_create(arr, 2, ctypes.byref(bad_map), None, ctypes.byref(h)) == nat.LABS_EINVAL
        assert b"warps_per_seq" in lib.labs_last_error()
    assert lib.labs_batch_destroy(None) == nat.LABS_OK


def test_serve_argument_errors_without_gpu(lib):
    from paper_2504_00987_gb300 import _native as nat

    bad = nat.ServeOpts(0, 64, 100, 4, 1000, 10, 0, 0, 0)
    assert not lib.labs_serve_create(ctypes.byref(bad))
    assert b"max_slots" in lib.labs_last_error()
    bad = nat.ServeOpts(16, 64, 100, 3, 1000, 10, 0, 0, 0)
    assert not lib.labs_serve_create(ctypes.byref(bad))
    bad = nat.ServeOpts(16, 64, 100, 4, 1000, 10, 0, 0, -5)  # negative time budget
    assert not lib.labs_serve_create(ctypes.byref(bad))
    assert b"quantum_us" in lib.labs_last_error()
    bad = nat.ServeOpts(16, 64, 100, 4, 1000, 10, 0, 0, 0, 3, 0)  # warps_per_request 3
    assert not lib.labs_serve_create(ctypes.byref(bad))
    assert b"warps_per_request" in lib.labs_last_error()
    assert ctypes.sizeof(nat.ServeOpts) == 4 * 4 + 8 * 5 + 4 * 2
    assert lib.labs_serve_destroy(None) == nat.LABS_OK
    assert lib.labs_serve_poll(None, 1, None) == nat.LABS_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror has the size and field offsets the C compiler gives
    the struct of include/labs.h (a C program compiled here prints them)."""
    import shutil
    import subprocess

    from paper_2504_00987_gb300 import _native as nat

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    pairs = [("labs_params", nat.Params), ("labs_device_result", nat.DeviceResult),
             ("labs_result", nat.Result), ("labs_tabu_opts", nat.TabuOpts), ("labs_instance", nat.Instance),
             ("labs_mapping", nat.Mapping), ("labs_serve_opts", nat.ServeOpts),
             ("labs_serve_stats", nat.ServeStats)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "labs.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    include = os.path.join(ROOT, "include")
    subprocess.check_call(["gcc", "-std=c11", "-I", include, "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, what, value = line.split()
        got[(cname, what)] = int(value)
    for cname, py in pairs:
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_every_entry_point_has_declared_ctypes_types(lib):
    """No call goes through ctypes' default int conversion (64-bit arguments
    would be truncated): every exported function has argtypes and restype."""
    from paper_2504_00987_gb300 import _native as nat

    for name in nat.EXPORTED:
        fn = getattr(lib, name)
        assert fn.argtypes is not None and fn.restype is not None, name


def test_results_decode_without_gpu(lib):
    """labs_results_decode is host code: the merit factor of Eq. 3, flip
    evaluations = steps * N and a signed E, checked on hand-made records."""
    import numpy as np

    from paper_2504_00987_gb300 import _native as nat

    rec = np.zeros((3, 8), dtype=np.int64)
    rec[0, 0] = 0x1234
    rec[0, 4] = (nat.RUN_REACHED << 32) | 100      # E = 100
    rec[0, 5:8] = (3, 7, 2)                         # generations, steps, trace_len
    rec[1, 4] = (nat.RUN_BADSTATE << 32) | 0xFFFFFFFF  # E = -1
    rec[2, 4] = (nat.RUN_BUDGET << 32) | 26         # E = 26
    rec[2, 6] = 5
    res = (nat.Result * 3)()
    assert lib.labs_results_decode(rec.ctypes.data_as(ctypes.c_void_p), 3, 64, 40, res) == nat.LABS_OK
    assert (res[0].E, res[0].F, res[0].flip_evals, res[0].steps, res[0].generations) == (100, 64 * 64 / 200.0,
                                                                                         7 * 64, 7, 3)
    assert res[0].seq[0] == 0x1234 and res[0].instance == 40 and res[0].status == nat.RUN_REACHED
    assert (res[1].E, res[1].F, res[1].status, res[1].instance) == (-1, 0.0, nat.RUN_BADSTATE, 41)
    assert res[2].F == 64 * 64 / 52.0 and res[2].flip_evals == 5 * 64
    assert lib.labs_results_decode(rec.ctypes.data_as(ctypes.c_void_p), 3, 2, 0, res) == nat.LABS_EINVAL
    assert lib.labs_results_decode(None, 1, 64, 0, res) == nat.LABS_EINVAL
    assert lib.labs_results_decode(None, 0, 64, 0, None) == nat.LABS_OK
