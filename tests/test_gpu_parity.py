"""GPU parity: every call of the C ABI against the CPU oracle on the same
seeded inputs.  All arithmetic is exact integer work, so every comparison is
bit-exact: energies, correlations, every chosen move and energy of every
tabu step, the per-generation records, the final sequences and counters."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NS = [3, 4, 5, 17, 31, 32, 33, 63, 64, 65, 95, 96, 100, 120, 127, 128, 129, 160, 191, 192, 193,
      255, 256]


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


# ------------------------------------------------------------------ energy


@pytest.mark.parametrize("N", NS)
def test_energy_batch_random_and_edges(labs, wl, orc, N):
    B = 1000  # several 256-thread blocks plus a ragged tail
    seqs = np.concatenate([wl.random_sequences(N, B, seed=N), wl.sequence_edge_cases(N)])
    E, C = labs.energy_batch(dev_seqs(seqs), N, with_C=True)
    E2 = labs.energy_batch(dev_seqs(seqs), N)
    E, C, E2 = E.cpu().numpy(), C.cpu().numpy(), E2.cpu().numpy()
    for b in range(len(seqs)):
        e, c = orc.energy(seqs[b], N, with_C=True)
        assert E[b] == e and E2[b] == e
        assert np.array_equal(C[b, : N - 1], c)


def test_energy_batch_table2(labs, orc):
    import tests.test_oracle_pins as pins

    for N, E, _, hx, _ in pins.table2_rows():
        w = orc.hex_to_words(hx, N)[None, :]
        assert int(labs.energy_batch(dev_seqs(w), N)[0]) == E


def test_energy_batch_ignores_tail_bits(labs, wl, orc):
    N = 70
    seqs = wl.random_sequences(N, 64, seed=3)
    dirty = seqs.copy()
    dirty[:, 1] |= np.uint64(0xFFFF_FFFF_FFFF_FFC0)  # set every bit >= 70
    assert torch.equal(labs.energy_batch(dev_seqs(seqs), N), labs.energy_batch(dev_seqs(dirty), N))


def test_energy_batch_empty_and_errors(labs):
    E = labs.energy_batch(torch.zeros((0, 1), dtype=torch.int64, device="cuda"), 64)
    assert E.numel() == 0
    from paper_2504_00987_gb300 import _native as nat

    lib = nat.load()
    host = np.zeros(4, dtype=np.uint64)
    dE = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = lib.labs_energy_batch(host.ctypes.data, 64, 4, dE.data_ptr(), None, None)
    assert rc == nat.LABS_EINVAL and b"not device memory" in lib.labs_last_error()


# ------------------------------------------------------------------ tabu


@pytest.mark.parametrize("N", NS)
def test_tabu_trajectories(labs, wl, orc, N):
    B = 37  # ten 4-warp blocks, the last one ragged
    starts = wl.random_sequences(N, B, seed=100 + N)
    cap = 2 * N + 2
    out = labs.tabu_run(dev_seqs(starts), N, seed=11, generation=5, first_instance=7, trace_cap=cap)
    best = out["best"].cpu().numpy().view(np.uint64)
    bestE, steps, trace = out["bestE"].cpu().numpy(), out["steps"].cpu().numpy(), out["trace"].cpu().numpy()
    for b in range(B):
        ob, oE, osteps, otr = orc.tabu_run(starts[b], N, 11, 7 + b, 5, trace_cap=cap)
        assert steps[b] == osteps and bestE[b] == oE
        assert np.array_equal(best[b], ob)
        assert np.array_equal(trace[b, :osteps], otr)


@pytest.mark.parametrize("N,max_iter", [(64, 0), (64, 1), (64, 500), (9, 40), (256, 300)])
def test_tabu_fixed_length(labs, wl, orc, N, max_iter):
    starts = wl.random_sequences(N, 5, seed=N + max_iter)
    out = labs.tabu_run(dev_seqs(starts), N, seed=2, max_iter=max_iter, trace_cap=max(max_iter, 1))
    for b in range(5):
        ob, oE, osteps, otr = orc.tabu_run(starts[b], N, 2, b, 0, max_iter=max_iter, trace_cap=max(max_iter, 1))
        assert int(out["steps"][b]) == osteps == max_iter
        assert int(out["bestE"][b]) == oE
        assert np.array_equal(out["trace"][b, :osteps].cpu().numpy(), otr)


def test_tabu_trace_shorter_than_run(labs, wl, orc):
    N = 80
    starts = wl.random_sequences(N, 3, seed=1)
    out = labs.tabu_run(dev_seqs(starts), N, seed=4, trace_cap=10)
    for b in range(3):
        _, oE, osteps, otr = orc.tabu_run(starts[b], N, 4, b, 0, trace_cap=10)
        assert int(out["steps"][b]) == osteps > 10
        assert np.array_equal(out["trace"][b].cpu().numpy(), otr)


# ------------------------------------------------------------------ MTS


def run_gpu_mts(labs, N, K, seed, first, R, cap, **kw):
    trace = torch.zeros((R, cap, 4), dtype=torch.int32, device="cuda") if cap else None
    P = labs.make_params(N, K, trace=trace, **kw)
    res = labs.decode_results(labs.mts_launch(P, seed, first, R), N, first)
    return res, (trace.cpu().numpy() if cap else None)


def check_against_oracle(orc, res, trace, N, K, seed, first, cap, **kw):
    for r, g in enumerate(res):
        P = orc.make_params(N, K, **kw)
        o, otr, _ = orc.mts_run(P, seed, first + r, trace_cap=cap)
        assert g["E"] == o["E"], (r, g["E"], o["E"])
        assert g["seq"] == [int(x) for x in o["seq"]]
        assert g["status"] == o["status"] and g["generations"] == o["generations"]
        assert g["steps"] == o["steps"]
        # decoded by the C boundary (labs_results_decode): Eq. 3 and steps * N
        assert g["F"] == (N * N / (2.0 * o["E"]) if o["E"] > 0 else 0.0)
        assert g["flip_evals"] == o["steps"] * N and g["instance"] == first + r
        if trace is not None:
            assert g["trace_len"] == len(otr)
            assert np.array_equal(trace[r, : len(otr)], otr)


@pytest.mark.parametrize("N,K", [(3, 2), (8, 5), (24, 100), (40, 33), (64, 100), (65, 7), (80, 40), (96, 64),
                                 (97, 9), (100, 50),
                                 (128, 100), (129, 20), (200, 10), (256, 3)])
@pytest.mark.parametrize("policy", [0, 1])
def test_mts_trajectories(labs, orc, N, K, policy):
    R, G = 6, 6
    cap = G * (3 * N // 2 + 2) + G
    res, tr = run_gpu_mts(labs, N, K, 77, 3, R, cap, max_generations=G, replace_policy=policy)
    check_against_oracle(orc, res, tr, N, K, 77, 3, cap, max_generations=G, replace_policy=policy)


def test_mts_step_budget_truncates_inside_tabu(labs, orc):
    N, K, R = 50, 30, 9
    cap = 2000
    res, tr = run_gpu_mts(labs, N, K, 5, 0, R, cap, max_steps=1234)
    assert all(r["steps"] == 1234 for r in res)
    check_against_oracle(orc, res, tr, N, K, 5, 0, cap, max_steps=1234)


def test_mts_fixed_tabu_length_and_mutation_rates(labs, orc):
    N, K, R = 45, 12, 5
    kw = dict(max_generations=10, max_iter=7, p_mut=(1 << 32) // 5, p_comb_u32=1 << 31)
    res, tr = run_gpu_mts(labs, N, K, 9, 0, R, 200, **kw)
    check_against_oracle(orc, res, tr, N, K, 9, 0, 200, **kw)


def test_mts_max_population(labs, orc):
    N, K = 256, 1024
    res, tr = run_gpu_mts(labs, N, K, 1, 0, 2, 2000, max_generations=3)
    check_against_oracle(orc, res, tr, N, K, 1, 0, 2000, max_generations=3)


def test_mts_target_met_by_initial_population(labs, orc):
    res, _ = run_gpu_mts(labs, 30, 10, 0, 0, 3, 0, target_E=10**6, max_generations=5)
    assert all(r["generations"] == 0 and r["status"] == labs.RUN_REACHED for r in res)


def test_mts_target_stops_replica(labs, orc):
    N, K = 30, 20
    o, _, _ = orc.mts_run(orc.make_params(N, K, max_generations=40), 4, 0)
    kw = dict(target_E=o["E"], max_generations=40)
    res, tr = run_gpu_mts(labs, N, K, 4, 0, 1, 5000, **kw)
    check_against_oracle(orc, res, tr, N, K, 4, 0, 5000, **kw)
    assert res[0]["status"] == labs.RUN_REACHED


def test_mts_glf_stops_every_replica(labs, orc):
    """Algorithm 3: once one replica reaches the target, the others stop at
    their next generation boundary; every replica's trace is a prefix of the
    oracle's trajectory for that instance."""
    N, K, R, cap = 26, 30, 64, 60000
    target = orc.bruteforce(N)[0] + 6
    trace = torch.zeros((R, cap, 4), dtype=torch.int32, device="cuda")
    P = labs.make_params(N, K, target_E=target, max_generations=2000, glf=True, trace=trace)
    res = labs.decode_results(labs.mts_launch(P, 8, 0, R), N)
    trace = trace.cpu().numpy()
    statuses = [r["status"] for r in res]
    assert labs.RUN_REACHED in statuses
    for r, g in enumerate(res):
        o, otr, _ = orc.mts_run(orc.make_params(N, K, target_E=target, max_generations=2000), 8, r,
                                trace_cap=cap)
        n = g["trace_len"]
        assert np.array_equal(trace[r, :n], otr[:n])
        if g["status"] == labs.RUN_REACHED:
            assert g["E"] == o["E"] <= target and g["generations"] == o["generations"]
        elif g["status"] == labs.RUN_STOPPED:
            assert g["generations"] <= o["generations"]


def test_mts_run_blocking_matches_launch(labs):
    P = labs.make_params(64, 40, max_steps=3000)
    a = labs.mts_run(P, 12, 100, 10)
    b = labs.decode_results(labs.mts_launch(P, 12, 100, 10), 64, 100)
    for x, y in zip(a, b):
        assert x["E"] == y["E"] and x["seq"] == y["seq"] and x["steps"] == y["steps"] == 3000
        assert x["instance"] == y["instance"] and abs(x["F"] - 64 * 64 / (2 * x["E"])) < 1e-12


def test_plain_n24_reaches_bruteforce_optimum(labs, orc):
    """N=24, K=100, seed 0, 2,000 generations: equals the oracle and the exhaustive optimum."""
    E_opt, _, _ = orc.bruteforce(24)
    cap = 2000 * 40
    res, tr = run_gpu_mts(labs, 24, 100, 0, 0, 1, cap, max_generations=2000)
    check_against_oracle(orc, res, tr, 24, 100, 0, 0, cap, max_generations=2000)
    assert res[0]["E"] == E_opt


def test_replicas_n64_full_size_sampled(labs, orc):
    """The benchmark's launch: N=64, K=100, 1,024 replicas x 10^5 tabu steps in one
    launch.  Eight replicas spread over the launch are checked against the
    oracle (final sequence, energy and counters); every replica must have
    used exactly its step budget and report an energy consistent with its
    sequence."""
    N, K, R, S = 64, 100, 1024, 100_000
    P = labs.make_params(N, K, max_steps=S)
    out = labs.mts_launch(P, 0, 0, R)
    res = labs.decode_results(out, N)
    assert all(r["steps"] == S for r in res)
    seqs = np.array([r["seq"] for r in res], dtype=np.uint64)
    E = labs.energy_batch(dev_seqs(seqs), N).cpu().numpy()
    assert all(int(E[i]) == res[i]["E"] for i in range(R))
    sample = [0, 1, 137, 300, 511, 777, 1000, 1023]
    ors = {}
    for i in sample:
        o, _, _ = orc.mts_run(orc.make_params(N, K, max_steps=S), 0, i)
        ors[i] = o
    for i in sample:
        assert res[i]["E"] == ors[i]["E"] and res[i]["seq"] == [int(x) for x in ors[i]["seq"]]
        assert res[i]["generations"] == ors[i]["generations"]


def test_sweep_n120_full_size_sampled(labs, orc):
    """The sweep's largest launch: N=120 (two 64-bit words), K=100, one replica
    per warp filling the GPU (16 per SM), 10^6 tabu steps each.  Three replicas
    (first, middle, last) against the oracle, run on three host threads; every
    replica used its budget and its energy matches its sequence."""
    from concurrent.futures import ThreadPoolExecutor

    N, K, S = 120, 100, 1_000_000
    R = torch.cuda.get_device_properties(0).multi_processor_count * 16
    P = labs.make_params(N, K, max_steps=S)
    res = labs.decode_results(labs.mts_launch(P, 0, 0, R), N)
    assert all(r["steps"] == S for r in res)
    seqs = np.array([r["seq"] for r in res], dtype=np.uint64)
    E = labs.energy_batch(dev_seqs(seqs), N).cpu().numpy()
    assert all(int(E[i]) == res[i]["E"] for i in range(R))
    sample = [0, R // 2, R - 1]
    with ThreadPoolExecutor(max_workers=len(sample)) as ex:
        ors = list(ex.map(lambda i: orc.mts_run(orc.make_params(N, K, max_steps=S), 0, i)[0], sample))
    for i, o in zip(sample, ors):
        assert res[i]["E"] == o["E"] and res[i]["seq"] == [int(x) for x in o["seq"]]
        assert res[i]["generations"] == o["generations"] and res[i]["steps"] == o["steps"]
