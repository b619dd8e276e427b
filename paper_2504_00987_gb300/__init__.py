"""GB300 (sm_103a) memetic tabu search for LABS (arXiv 2504.00987).

Thin Python binding of liblabs.so (include/labs.h): every function here only
marshals torch tensors (device memory, the current CUDA stream) into the C
ABI; all computation runs in the library's CUDA kernels.  Importing this
package does not load the library; the first call does, and fails loudly if
it has not been built.

Sequences are packed as in labs.h: shape (B, ceil(N/64)) int64 (or uint64)
tensors, spin i at bit i % 64 of word i // 64, bit 1 <-> +1.
"""
from __future__ import annotations

from .api import (  # noqa: F401
    P_COMB_U32,
    Batch,
    Server,
    autotune,
    make_instance,
    mts_batch_run,
    decode_results,
    energy_batch,
    mts_launch,
    mts_resume,
    mts_run,
    mts_state_bytes,
    make_params,
    p_mut_u32,
    philox_batch,
    skew_deviation_batch,
    tabu_run,
    version,
)
from ._native import (  # noqa: F401
    LabsError,
    REPLACE_RANDOM,
    REPLACE_WORST,
    RUN_BUDGET,
    RUN_REACHED,
    RUN_BADSTATE,
    RUN_STOPPED,
    VARIANT_FIX_FIRST_SPIN,
    VARIANT_SKEW,
    VARIANT_UNIFORM_CROSSOVER,
)
