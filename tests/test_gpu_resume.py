"""Checkpoint and resume (labs_mts_resume): a run stopped at a generation
budget and continued to a larger one equals the run made straight to the
larger budget, bit for bit -- whether the state stays on the device or goes
through the host -- and equals the oracle's run; records of another run
are refused replica by replica."""
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


def key(r):
    return (r["E"], r["seq"], r["generations"], r["steps"], r["status"])


@pytest.mark.parametrize("N,K,variant", [(24, 100, 0), (64, 100, 0), (65, 30, 1), (129, 20, 2),
                                         (201, 10, 4), (77, 25, 7), (256, 3, 0)])
def test_split_run_equals_straight_run(labs, N, K, variant):
    R, G = 37, 12
    state = torch.zeros(R * labs.mts_state_bytes(N, K), dtype=torch.uint8, device="cuda")
    straight = labs.decode_results(
        labs.mts_launch(labs.make_params(N, K, max_generations=G, variant=variant), 5, 100, R), N, 100)
    half = labs.decode_results(labs.mts_resume(labs.make_params(N, K, max_generations=G // 2, variant=variant),
                                               5, 100, R, state, resume=False), N, 100)
    assert all(r["generations"] == G // 2 for r in half)
    # through the host, as a checkpoint file would be
    saved = state.cpu().numpy().copy()
    state.zero_()
    state.copy_(torch.from_numpy(saved))
    cont = labs.decode_results(labs.mts_resume(labs.make_params(N, K, max_generations=G, variant=variant),
                                               5, 100, R, state, resume=True), N, 100)
    assert [key(r) for r in cont] == [key(r) for r in straight]


def test_resume_equals_oracle_and_continues_again(labs, orc):
    N, K, R = 50, 40, 6
    state = torch.empty(R * labs.mts_state_bytes(N, K), dtype=torch.uint8, device="cuda")
    for i, G in enumerate((3, 9, 20)):
        res = labs.decode_results(labs.mts_resume(labs.make_params(N, K, max_generations=G), 8, 0, R, state,
                                                  resume=i > 0), N)
        for r, g in enumerate(res):
            o, _, _ = orc.mts_run(orc.make_params(N, K, max_generations=G), 8, r)
            assert g["E"] == o["E"] and g["seq"] == [int(x) for x in o["seq"]]
            assert g["generations"] == o["generations"] == G and g["steps"] == o["steps"]


def test_resume_with_target_and_nothing_left(labs):
    N, K, R = 40, 30, 8
    state = torch.empty(R * labs.mts_state_bytes(N, K), dtype=torch.uint8, device="cuda")
    a = labs.decode_results(labs.mts_resume(labs.make_params(N, K, max_generations=30), 1, 0, R, state,
                                            resume=False), N)
    # same budget again: nothing left to do, the results repeat
    b = labs.decode_results(labs.mts_resume(labs.make_params(N, K, max_generations=30), 1, 0, R, state,
                                            resume=True), N)
    assert [key(r) for r in a] == [key(r) for r in b]
    # a target every replica already meets stops each one at once
    t = max(r["E"] for r in a)
    c = labs.decode_results(labs.mts_resume(labs.make_params(N, K, max_generations=1000, target_E=t), 1, 0, R,
                                            state, resume=True), N)
    assert all(r["status"] == labs.RUN_REACHED and r["generations"] == 30 for r in c)


def test_records_of_another_run_are_refused(labs):
    N, K, R = 33, 20, 8
    nb = labs.mts_state_bytes(N, K)
    state = torch.empty(R * nb, dtype=torch.uint8, device="cuda")
    labs.mts_resume(labs.make_params(N, K, max_generations=2), 4, 0, R, state, resume=False)
    before = state.cpu().numpy().copy()
    for P, seed, first in ((labs.make_params(N, K, max_generations=4), 5, 0),            # other seed
                           (labs.make_params(N, K, max_generations=4), 4, 1),            # other instances
                           (labs.make_params(N, K, max_generations=4, variant=1), 4, 0),  # other variant
                           (labs.make_params(N - 2, K, max_generations=4), 4, 0)):       # other N, same size
        res = labs.decode_results(labs.mts_resume(P, seed, first, R, state, resume=True), P.N, first)
        assert all(r["status"] == labs.RUN_BADSTATE and r["generations"] == 0 and r["E"] == -1 and
                   r["F"] == 0.0 and r["flip_evals"] == 0 for r in res)
        assert np.array_equal(state.cpu().numpy(), before)
    # a fresh start rewrites them
    res = labs.decode_results(labs.mts_resume(labs.make_params(N, K, max_generations=4), 5, 0, R, state,
                                              resume=False), N)
    assert all(r["status"] == labs.RUN_BUDGET for r in res)
