"""Edge cases of the GPU path against the oracle: degenerate populations and
probabilities, the smallest N, Philox counters and keys at their limits, and
a large energy batch checked on sampled rows."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def labs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2504_00987_gb300 as labs

    return labs


def gpu_vs_oracle(labs, orc, N, K, seed, first, R, cap=4000, **kw):
    trace = torch.zeros((R, cap, 4), dtype=torch.int32, device="cuda")
    P = labs.make_params(N, K, trace=trace, **kw)
    res = labs.decode_results(labs.mts_launch(P, seed, first, R), N, first)
    tr = trace.cpu().numpy()
    okw = dict(kw)
    if "p_mut" in okw and okw["p_mut"] == 0:
        okw.pop("p_mut")
    for r, g in enumerate(res):
        o, otr, _ = orc.mts_run(orc.make_params(N, K, **okw), seed, first + r, trace_cap=cap)
        assert (g["E"], g["seq"], g["steps"], g["generations"], g["status"]) == \
            (o["E"], [int(x) for x in o["seq"]], o["steps"], o["generations"], o["status"])
        assert np.array_equal(tr[r, : len(otr)], otr)


@pytest.mark.parametrize("N,K", [(3, 1), (4, 1), (17, 1), (64, 1), (200, 1)])
def test_population_of_one(labs, orc, N, K):
    gpu_vs_oracle(labs, orc, N, K, 3, 0, 4, max_generations=8)


@pytest.mark.parametrize("p_comb", [0, 1, 0xFFFFFFFF])
def test_crossover_probability_extremes(labs, orc, p_comb):
    gpu_vs_oracle(labs, orc, 50, 20, 1, 0, 4, max_generations=10, p_comb_u32=p_comb)


def test_every_bit_mutates(labs, orc):
    gpu_vs_oracle(labs, orc, 33, 10, 2, 0, 3, max_generations=6, p_mut=0xFFFFFFFF)


def test_instance_numbers_at_the_top_and_wide_seeds(labs, orc):
    top = (1 << 32) - 5
    gpu_vs_oracle(labs, orc, 40, 12, 0xDEADBEEF12345678, top, 5, max_generations=5)
    gpu_vs_oracle(labs, orc, 70, 12, (1 << 64) - 1, 7, 3, max_generations=4)


def test_energy_batch_one_million_sampled(labs, orc):
    from paper_2504_00987_gb300 import workloads

    N, B = 120, 1_000_000
    seqs = workloads.random_sequences(N, B, seed=99)
    E = labs.energy_batch(torch.from_numpy(seqs.view(np.int64)).cuda(), N).cpu().numpy()
    rng = np.random.default_rng(1)
    for b in rng.integers(0, B, 400):
        assert int(E[b]) == orc.energy(seqs[b], N)
    # every energy is consistent with the parity of C_k: E = sum C_k^2 with C_k = N-k mod 2
    floor = sum(1 for k in range(1, N) if (N - k) % 2)
    assert int(E.min()) >= floor


@pytest.mark.parametrize("N", [13, 37, 70, 130])
def test_long_tabu_search_can_run_out_of_moves(labs, orc, N):
    """With a user maxIter of 20 N the tenure bound floor(12 maxIter / 100)
    exceeds N, so every move can be tabu with none aspirating; the search then
    stops early (Alg. 2 has no admissible move).  The GPU stops at the same
    step as the oracle, with the same trajectory, and some search does stop."""
    B, mi = 16, 20 * N
    rng = np.random.default_rng(N)
    starts = rng.integers(0, 1 << 63, size=(B, (N + 63) // 64), dtype=np.int64).astype(np.uint64)
    for w in range((N + 63) // 64):
        hi = N - 64 * w
        if hi < 64:
            starts[:, w] &= np.uint64((1 << max(hi, 0)) - 1)
    out = labs.tabu_run(torch.from_numpy(starts.view(np.int64)).cuda(), N, seed=3, max_iter=mi, trace_cap=mi)
    early = 0
    for b in range(B):
        best, bestE, steps, tr = orc.tabu_run(starts[b], N, 3, b, 0, max_iter=mi, trace_cap=mi)
        assert int(out["steps"][b]) == steps and int(out["bestE"][b]) == bestE
        assert np.array_equal(out["trace"][b, :steps].cpu().numpy(), tr)
        early += steps < mi
    assert early > 0
