"""d(S) of Appendix A on the GPU: the d column of Table II and the oracle on
random and patterned sequences of odd and even lengths."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def test_table2_d_column(labs, orc):
    import tests.test_oracle_pins as pins

    for N, _, _, hx, d in pins.table2_rows():
        w = orc.hex_to_words(hx, N)[None, :]
        assert int(labs.skew_deviation_batch(dev(w), N)[0]) == d


@pytest.mark.parametrize("N", [3, 4, 5, 6, 31, 32, 33, 63, 64, 65, 96, 99, 128, 129, 190, 255, 256])
def test_matches_oracle(labs, orc, N):
    from paper_2504_00987_gb300 import workloads

    seqs = np.concatenate([workloads.random_sequences(N, 23, seed=N), workloads.sequence_edge_cases(N)])
    got = labs.skew_deviation_batch(dev(seqs), N).cpu().numpy()
    for b in range(len(seqs)):
        assert got[b] == orc.skew_deviation(seqs[b], N)


def test_skew_symmetric_sequences_have_zero_deviation(labs):
    rng = np.random.default_rng(0)
    for N in [7, 63, 121, 255]:
        n = (N + 1) // 2
        s = np.zeros(N, dtype=np.int64)
        s[:n] = rng.choice([-1, 1], n)
        for i in range(1, n):
            s[n + i - 1] = (-1) ** i * s[n - i - 1]
        w = np.zeros((1, (N + 63) // 64), dtype=np.uint64)
        for i in range(N):
            if s[i] > 0:
                w[0, i // 64] |= np.uint64(1) << np.uint64(i % 64)
        assert int(labs.skew_deviation_batch(dev(w), N)[0]) == 0
