"""GPU parity of the Algorithm 1 variants (uniform crossover; s_1 fixed to +1
as the symmetry break of Sec. II.B; the search restricted to skew-symmetric
sequences of Sec. II.C) against the oracle: every tabu step, the final
sequences and counters, through labs_tabu_run, labs_mts_launch, the
batched launch and the solve service.  All exact integer work, so every
comparison is bit-exact."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

UNIFORM, FIX, SKEW = 1, 2, 4


@pytest.fixture(scope="module")
def labs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2504_00987_gb300 as labs

    return labs


@pytest.fixture(scope="module")
def wl():
    from paper_2504_00987_gb300 import workloads

    return workloads


def dev_seqs(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("N", [3, 5, 31, 32, 33, 64, 65, 100, 128, 129, 200, 256])
def test_tabu_fixed_first_spin(labs, wl, orc, N):
    B = 37
    starts = wl.random_sequences(N, B, seed=300 + N)
    cap = 2 * N + 2
    out = labs.tabu_run(dev_seqs(starts), N, seed=13, generation=2, first_instance=5, trace_cap=cap,
                        variant=FIX)
    best = out["best"].cpu().numpy().view(np.uint64)
    bestE, steps, trace = out["bestE"].cpu().numpy(), out["steps"].cpu().numpy(), out["trace"].cpu().numpy()
    for b in range(B):
        ob, oE, osteps, otr = orc.tabu_run(starts[b], N, 13, 5 + b, 2, trace_cap=cap, variant=FIX)
        assert steps[b] == osteps and bestE[b] == oE
        assert np.array_equal(best[b], ob)
        assert np.array_equal(trace[b, :osteps], otr)
        assert not np.any(otr[:, 2] == 0)  # bit 0 is never a move
        assert (int(best[b, 0]) & 1) == (int(starts[b, 0]) & 1)


def run_gpu_mts(labs, N, K, seed, R, cap, **kw):
    trace = torch.zeros((R, cap, 4), dtype=torch.int32, device="cuda")
    P = labs.make_params(N, K, trace=trace, **kw)
    res = labs.decode_results(labs.mts_launch(P, seed, 0, R), N, 0)
    return res, trace.cpu().numpy()


@pytest.mark.parametrize("variant", [UNIFORM, FIX, UNIFORM | FIX])
@pytest.mark.parametrize("N,K", [(3, 2), (8, 5), (24, 100), (63, 20), (64, 100), (65, 7), (100, 50),
                                 (129, 20), (200, 10), (256, 3)])
def test_mts_variants(labs, orc, variant, N, K):
    R, G = 6, 6
    cap = G * (3 * N // 2 + 2) + G
    kw = dict(max_generations=G, variant=variant, replace_policy=G % 2)
    res, tr = run_gpu_mts(labs, N, K, 41, R, cap, **kw)
    for r, g in enumerate(res):
        o, otr, _ = orc.mts_run(orc.make_params(N, K, **kw), 41, r, trace_cap=cap)
        assert (g["E"], g["status"], g["generations"], g["steps"]) == \
            (o["E"], o["status"], o["generations"], o["steps"])
        assert g["seq"] == [int(x) for x in o["seq"]]
        assert g["trace_len"] == len(otr)
        assert np.array_equal(tr[r, : len(otr)], otr)
        if variant & FIX:
            assert g["seq"][0] & 1 == 1  # s_1 = +1
            moves = otr[otr[:, 1] > 0]  # t = 0 records name the replaced member
            assert not np.any(moves[:, 2] == 0)


def test_mts_uniform_crossover_high_rates(labs, orc):
    """Every generation combines (p_comb = 1 - 2^-32) and mutates heavily:
    the crossover and mutation masks of each generation decide the run."""
    N, K, R = 90, 16, 5
    kw = dict(max_generations=12, max_iter=5, p_comb_u32=0xFFFFFFFF, p_mut=(1 << 32) // 3,
              variant=UNIFORM | FIX)
    res, tr = run_gpu_mts(labs, N, K, 3, R, 100, **kw)
    for r, g in enumerate(res):
        o, otr, _ = orc.mts_run(orc.make_params(N, K, **kw), 3, r, trace_cap=100)
        assert g["E"] == o["E"] and g["seq"] == [int(x) for x in o["seq"]]
        assert np.array_equal(tr[r, : len(otr)], otr)


def test_variants_in_batch_and_static_and_serve(labs, orc):
    rng = np.random.default_rng(5)
    inst, kws = [], []
    for i in range(48):
        N, K = int(rng.integers(20, 140)), int(rng.integers(5, 60))
        kw = dict(max_steps=int(rng.integers(200, 3000)), variant=int(i % 4))
        inst.append(labs.make_instance(N, K, seed=17, instance=i, **kw))
        kws.append((N, K, kw))
    with labs.Batch(inst) as b:
        b.launch()
        got = b.results()
    with labs.Server(max_slots=8, max_N=160, max_K=64, quantum_steps=250) as srv:
        tickets = [srv.submit(x) for x in inst[:16]]
        served = {}
        import time

        deadline = time.time() + 120
        while len(served) < len(tickets):
            assert time.time() < deadline
            for t in tickets:
                if t not in served:
                    r = srv.poll(t)
                    if r is not None:
                        served[t] = r
            time.sleep(0.001)
    for i, ((N, K, kw), g) in enumerate(zip(kws, got)):
        o, _, _ = orc.mts_run(orc.make_params(N, K, **kw), 17, i)
        want = (o["E"], [int(x) for x in o["seq"]], o["steps"], o["generations"], o["status"])
        assert (g["E"], g["seq"], g["steps"], g["generations"], g["status"]) == want
        if i < 16:
            s = served[tickets[i]]
            assert (s["E"], s["seq"], s["steps"], s["generations"], s["status"]) == want
    # the blocking and the allocation-free entry points carry the flag too
    N, K = 77, 25
    P = labs.make_params(N, K, max_generations=8, variant=UNIFORM | FIX)
    a = labs.mts_run(P, 9, 0, 4)
    for r, g in enumerate(a):
        o, _, _ = orc.mts_run(orc.make_params(N, K, max_generations=8, variant=UNIFORM | FIX), 9, r)
        assert g["E"] == o["E"] and g["seq"] == [int(x) for x in o["seq"]]


def test_unknown_variant_flags_rejected(labs):
    from paper_2504_00987_gb300 import _native as nat

    with pytest.raises(nat.LabsError):
        labs.mts_launch(labs.make_params(40, 10, max_generations=1, variant=8), 0, 0, 1)
    with pytest.raises(nat.LabsError):
        labs.tabu_run(dev_seqs(np.zeros((1, 1), dtype=np.uint64)), 40, 0, variant=8)


def is_skew_words(words, N):
    """Sec. II.C on packed bits: b_{c+i} = b_{c-i} xor (i odd), c = (N-1)/2."""
    v = sum(int(w) << (64 * k) for k, w in enumerate(words))
    b = [(v >> i) & 1 for i in range(N)]
    c = (N - 1) // 2
    return all(b[c + i] == b[c - i] ^ (i & 1) for i in range(1, c + 1))


@pytest.mark.parametrize("N", [3, 5, 31, 33, 63, 65, 101, 127, 129, 191, 193, 255])
@pytest.mark.parametrize("fix", [False, True])
def test_tabu_skew(labs, wl, orc, N, fix):
    """Pair moves of the skew-restricted search: every step's move and energy."""
    B = 37
    variant = SKEW | (FIX if fix else 0)
    starts = wl.random_sequences(N, B, seed=500 + N)
    cap = N + 2
    out = labs.tabu_run(dev_seqs(starts), N, seed=21, generation=3, first_instance=9, trace_cap=cap,
                        variant=variant)
    best = out["best"].cpu().numpy().view(np.uint64)
    bestE, steps, trace = out["bestE"].cpu().numpy(), out["steps"].cpu().numpy(), out["trace"].cpu().numpy()
    for b in range(B):
        ob, oE, osteps, otr = orc.tabu_run(starts[b], N, 21, 9 + b, 3, trace_cap=cap, variant=variant)
        assert steps[b] == osteps and bestE[b] == oE
        assert np.array_equal(best[b], ob)
        assert np.array_equal(trace[b, :osteps], otr)
        assert is_skew_words(best[b], N)


@pytest.mark.parametrize("variant", [SKEW, SKEW | UNIFORM, SKEW | FIX, SKEW | UNIFORM | FIX])
@pytest.mark.parametrize("N,K", [(3, 2), (7, 5), (25, 100), (63, 20), (65, 7), (101, 50), (129, 20),
                                 (201, 10), (255, 3)])
def test_mts_skew(labs, orc, variant, N, K):
    R, G = 6, 6
    cap = G * (3 * N // 4 + 3) + G
    kw = dict(max_generations=G, variant=variant, replace_policy=N % 2 if K > 5 else 0)
    res, tr = run_gpu_mts(labs, N, K, 43, R, cap, **kw)
    for r, g in enumerate(res):
        o, otr, _ = orc.mts_run(orc.make_params(N, K, **kw), 43, r, trace_cap=cap)
        assert (g["E"], g["status"], g["generations"], g["steps"]) == \
            (o["E"], o["status"], o["generations"], o["steps"])
        assert g["seq"] == [int(x) for x in o["seq"]]
        assert g["trace_len"] == len(otr)
        assert np.array_equal(tr[r, : len(otr)], otr)
        assert is_skew_words(g["seq"], N)


def test_mts_skew_budget_target_and_entry_points(labs, orc):
    """A step budget that ends a search mid-way, a target, and the blocking
    and allocation-free entry points, all against the oracle."""
    N, K, R = 77, 30, 8
    res, tr = run_gpu_mts(labs, N, K, 5, R, 3000, max_steps=1111, variant=SKEW)
    for r, g in enumerate(res):
        o, otr, _ = orc.mts_run(orc.make_params(N, K, max_steps=1111, variant=SKEW), 5, r, trace_cap=3000)
        assert g["steps"] == o["steps"] == 1111 and g["E"] == o["E"]
        assert np.array_equal(tr[r, : len(otr)], otr)
    target = min(g["E"] for g in res) + 40
    P = labs.make_params(N, K, target_E=target, max_generations=500, variant=SKEW | FIX)
    a = labs.mts_run(P, 2, 0, 4)
    for r, g in enumerate(a):
        o, _, _ = orc.mts_run(orc.make_params(N, K, target_E=target, max_generations=500, variant=SKEW | FIX),
                              2, r)
        assert (g["E"], g["seq"], g["steps"], g["status"]) == (o["E"], [int(x) for x in o["seq"]], o["steps"],
                                                              o["status"])
    from paper_2504_00987_gb300 import _native as nat
    import ctypes

    res_s = (nat.Result * 4)()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert nat.load().labs_mts_run_static(ctypes.byref(P), 2, 0, 4, res_s, stream) == nat.LABS_OK
    assert [(r.E, list(r.seq)[:2], r.steps) for r in res_s] == [(g["E"], g["seq"], g["steps"]) for g in a]


def test_skew_reaches_exhaustive_skew_optimum(labs):
    """N = 25: 304 replicas reach the skew-symmetric optimum of the
    exhaustive enumeration (52), above the unrestricted optimum (36)."""
    import tests.test_oracle_pins as pins

    N = 25
    E_skew = pins.skew_optimum(N)
    P = labs.make_params(N, 50, target_E=E_skew, max_generations=2000, variant=SKEW)
    res = labs.mts_run(P, 7, 0, 304)
    assert all(r["E"] == E_skew and r["status"] == 1 for r in res)
