"""The device generator against the oracle's: Philox4x32-10 words of the
randomness contract at 10^6 random counters (and at the structured counters
the kernels use) are identical, and their bits are uniform (chi-square of
the top byte of every word)."""
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


def gpu_words(labs, ctr, seed):
    d = torch.from_numpy(ctr.view(np.int32)).cuda()
    return labs.philox_batch(d, seed).cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEF12345678, (1 << 64) - 1])
def test_philox_million_random_counters(labs, orc, seed):
    rng = np.random.default_rng(seed % 1000)
    ctr = rng.integers(0, 1 << 32, size=(1_000_000, 4), dtype=np.uint64).astype(np.uint32)
    g = gpu_words(labs, ctr, seed)
    assert np.array_equal(g, orc.philox4x32_batch(ctr, seed))
    top = (g >> 24).ravel()
    counts = np.bincount(top, minlength=256)
    expect = top.size / 256
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    from scipy import stats

    assert stats.chi2.sf(chi2, 255) > 1e-6


def test_philox_contract_counters(labs, orc):
    """The counters the kernels draw at: members, generations, mutation
    blocks, steps and crossover blocks of several instances."""
    rows = []
    for inst in (0, 1, 1023, (1 << 32) - 1):
        for a in range(0, 3000, 97):
            for b in (0, 1, 2, 31, 64):
                for purpose in (1, 2, 3, 4, 5):
                    rows.append((inst, a, b, purpose))
    ctr = np.array(rows, dtype=np.uint32)
    assert np.array_equal(gpu_words(labs, ctr, 77), orc.philox4x32_batch(ctr, 77))


def test_philox_empty_and_errors(labs):
    from paper_2504_00987_gb300 import _native as nat

    empty = torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    assert labs.philox_batch(empty, 3).shape == (0, 4)
    with pytest.raises(ValueError):
        labs.philox_batch(torch.zeros((4, 3), dtype=torch.int32, device="cuda"), 0)
    host = torch.zeros((4, 4), dtype=torch.int32)
    assert nat.load().labs_philox_batch(0, host.data_ptr(), 4, host.data_ptr(), None) == nat.LABS_EINVAL
