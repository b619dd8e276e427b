"""Pins for the CPU oracle against facts that do not come from the oracle itself:
the values printed in the paper (Table II), closed forms, textbook special
cases (Barker sequences), invariances of Eq. 2 stated in Sec. II.B/II.C,
library routines (numpy's correlate and numpy's Philox4x64-10), and brute
force on tiny inputs.  Every test here runs on CPU."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_new_records.txt")


def table2_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            N, E, MF, hx, d = line.split()
            rows.append((int(N), int(E), float(MF), hx, int(d)))
    return rows


def np_energy(s):
    """Eq. 1-2 through numpy.correlate (a library autocorrelation)."""
    s = np.asarray(s, dtype=np.int64)
    N = len(s)
    C = np.correlate(s, s, mode="full")[N:]
    return int(np.dot(C, C)), C


def rand_spins(rng, N):
    return rng.choice(np.array([-1, 1]), size=N)


# --------------------------------------------------------------------------- RNG


def test_philox4x64_matches_numpy(orc):
    """The oracle's Philox construction, instantiated on 64-bit words, equals
    numpy.random.Philox (which increments its counter before each block)."""
    rng = np.random.default_rng(123)
    for _ in range(20):
        key = rng.integers(0, 2**63, size=2, dtype=np.int64).astype(np.uint64)
        ctr0 = int(rng.integers(0, 2**62))
        bg = np.random.Philox(key=key, counter=np.array([ctr0, 0, 0, 0], dtype=np.uint64))
        raw = bg.random_raw(8)
        a = orc.philox4x64_10([ctr0 + 1, 0, 0, 0], key)
        b = orc.philox4x64_10([ctr0 + 2, 0, 0, 0], key)
        assert list(raw) == list(a) + list(b)


def _weyl(w: int) -> tuple[int, int]:
    """The Weyl key increments of Philox (SC'11) from their definitions:
    floor((phi - 1) 2^w) and floor((sqrt(3) - 1) 2^w), in exact integer arithmetic."""
    import math

    s5 = math.isqrt(5 << (2 * w))    # floor(sqrt(5) 2^w)
    s3 = math.isqrt(3 << (2 * w))    # floor(sqrt(3) 2^w)
    return (s5 - (1 << w)) >> 1, s3 - (1 << w)


def _philox_naive(w: int, mult: tuple[int, int], ctr, key, rounds: int = 10) -> list[int]:
    """Philox4xW (Salmon, Moraes, Dror, Shaw, SC'11) with Python integers: each
    round multiplies counter words 0 and 2 by the two multipliers into
    double-width products and emits (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2),
    hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)); the key gains the Weyl increments
    before every round but the first."""
    mask = (1 << w) - 1
    w0, w1 = _weyl(w)
    x = [int(c) & mask for c in ctr]
    k0, k1 = int(key[0]) & mask, int(key[1]) & mask
    for r in range(rounds):
        if r:
            k0, k1 = (k0 + w0) & mask, (k1 + w1) & mask
        p0, p1 = mult[0] * x[0], mult[1] * x[2]
        x = [(p1 >> w) ^ x[1] ^ k0, p1 & mask, (p0 >> w) ^ x[3] ^ k1, p0 & mask]
    return x


def test_philox4x64_naive_matches_numpy():
    """The naive round structure and key schedule, on 64-bit words, equal numpy.random.Philox."""
    mult64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
    rng = np.random.default_rng(7)
    for _ in range(10):
        key = rng.integers(0, 2**63, size=2, dtype=np.int64).astype(np.uint64)
        ctr0 = int(rng.integers(0, 2**62))
        raw = np.random.Philox(key=key, counter=np.array([ctr0, 0, 0, 0], dtype=np.uint64)).random_raw(4)
        assert list(map(int, raw)) == _philox_naive(64, mult64, [ctr0 + 1, 0, 0, 0], key)


def test_philox4x32_matches_naive_definition(orc):
    """The oracle's Philox4x32-10 equals the naive big-integer one (same
    structure as the numpy-checked 64-bit form, Weyl increments derived from
    phi and sqrt 3, the 32-bit multipliers of SC'11) on 10^4 random counters
    and keys, so a wrong digit in any of its constants fails here."""
    mult32 = (0xD2511F53, 0xCD9E8D57)
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 1 << 32, size=(10_000, 4), dtype=np.uint64)
    keys = rng.integers(0, 1 << 32, size=(10_000, 2), dtype=np.uint64)
    for i in range(10_000):
        c, k = [int(v) for v in ctr[i]], [int(v) for v in keys[i]]
        assert list(map(int, orc.philox4x32_10(c, k))) == _philox_naive(32, mult32, c, k), i


def test_philox_batch_equals_single_calls(orc):
    """The batched oracle generator is the single-counter one at every row."""
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 1 << 32, size=(200, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0x0123456789ABCDEF
    out = orc.philox4x32_batch(ctr, seed)
    for r in range(200):
        assert list(out[r]) == list(orc.philox4x32_10(list(ctr[r]), [seed & 0xFFFFFFFF, seed >> 32]))


def test_philox4x32_statistics(orc):
    """Uniformity and independence of the 32-bit variant over a counter sweep."""
    outs = np.array([orc.philox4x32_10([i, 3, 0, 4], [5, 0]) for i in range(4096)], dtype=np.uint64)
    flat = outs.ravel()
    # bit balance: each of 32 bits is set in ~50% of 16384 words
    bits = np.array([(flat >> np.uint64(b)) & np.uint64(1) for b in range(32)], dtype=np.float64)
    frac = bits.mean(axis=1)
    assert np.all(np.abs(frac - 0.5) < 0.02)
    # chi-square over 64 buckets of the top 6 bits
    hist = np.bincount((flat >> np.uint64(26)).astype(np.int64), minlength=64)
    chi2 = ((hist - len(flat) / 64) ** 2 / (len(flat) / 64)).sum()
    assert chi2 < 120  # 63 dof: p ~ 1e-5
    # distinct counters and distinct keys give distinct blocks
    assert len({tuple(o) for o in outs.tolist()}) == 4096
    assert list(orc.philox4x32_10([0, 0, 0, 0], [0, 0])) != list(orc.philox4x32_10([0, 0, 0, 0], [1, 0]))


# --------------------------------------------------------------------- Energy


def test_table2_energies_and_merit_factors(orc):
    """All 17 rows of Table II: decoded MSB-first, E matches and N^2/(2E) rounds to MF."""
    for N, E, MF, hx, _ in table2_rows():
        w = orc.hex_to_words(hx, N)
        assert orc.energy(w, N) == E
        assert round(N * N / (2 * E), 2) == pytest.approx(MF)


def test_energy_matches_numpy_correlate(orc):
    rng = np.random.default_rng(1)
    for N in [3, 4, 5, 17, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256]:
        for _ in range(4):
            s = rand_spins(rng, N)
            E, C = orc.energy(orc.spins_to_words(s), N, with_C=True)
            E2, C2 = np_energy(s)
            assert E == E2
            assert list(C) == list(C2)


def test_energy_closed_forms(orc):
    """All-equal and alternating sequences: |C_k| = N - k, so
    E = sum_{m=1}^{N-1} m^2 = (N-1) N (2N-1) / 6."""
    for N in [3, 10, 64, 99, 128, 256]:
        closed = (N - 1) * N * (2 * N - 1) // 6
        for s in (np.ones(N), -np.ones(N), np.array([(-1) ** i for i in range(N)])):
            assert orc.energy(orc.spins_to_words(s), N) == closed


BARKER = {  # textbook Barker sequences: every |C_k| <= 1
    7: "+++--+-",
    11: "+++---+--+-",
    13: "+++++--++-+-+",
}


def test_barker_sequences(orc):
    for N, txt in BARKER.items():
        s = np.array([1 if c == "+" else -1 for c in txt])
        E, C = orc.energy(orc.spins_to_words(s), N, with_C=True)
        assert np.all(np.abs(C) <= 1)
        assert E == N // 2  # C_k has the parity of N - k


def test_energy_invariances(orc):
    """Sec. II.B: complementation and reversal preserve E.  Alternating sign
    s_i -> (-1)^i s_i maps C_k -> (-1)^k C_k, so E is preserved as well."""
    rng = np.random.default_rng(2)
    for N in [5, 31, 64, 92, 150, 256]:
        s = rand_spins(rng, N)
        E, C = orc.energy(orc.spins_to_words(s), N, with_C=True)
        alt = np.array([(-1) ** i for i in range(N)])
        assert orc.energy(orc.spins_to_words(-s), N) == E
        assert orc.energy(orc.spins_to_words(s[::-1]), N) == E
        E3, C3 = orc.energy(orc.spins_to_words(s * alt), N, with_C=True)
        assert E3 == E
        assert list(C3) == [(-1) ** k * C[k - 1] for k in range(1, N)]


def test_skew_symmetric_odd_correlations_vanish(orc):
    """Eq. 4: for N = 2n - 1, s_{n+i} = (-1)^i s_{n-i} implies C_k = 0 for odd k."""
    rng = np.random.default_rng(3)
    for N in [5, 21, 63, 99, 119, 255]:
        n = (N + 1) // 2
        s = np.zeros(N, dtype=np.int64)
        s[: n] = rand_spins(rng, n)  # s_1 .. s_n free
        for i in range(1, n):
            s[n + i - 1] = (-1) ** i * s[n - i - 1]
        _, C = orc.energy(orc.spins_to_words(s), N, with_C=True)
        assert all(C[k - 1] == 0 for k in range(1, N, 2))
        assert orc.non_skew_pairs(orc.spins_to_words(s), N) == 0


def test_correlation_parity(orc):
    rng = np.random.default_rng(4)
    for N in [6, 7, 64, 65]:
        _, C = orc.energy(orc.spins_to_words(rand_spins(rng, N)), N, with_C=True)
        assert all((C[k - 1] - (N - k)) % 2 == 0 for k in range(1, N))


def test_neighbour_energies_definition(orc):
    rng = np.random.default_rng(5)
    for N in [3, 8, 33, 64, 70]:
        s = rand_spins(rng, N)
        got = orc.neighbour_energies(orc.spins_to_words(s), N)
        for j in range(N):
            t = s.copy()
            t[j] = -t[j]
            assert got[j] == np_energy(t)[0]


# ----------------------------------------------------------------- Brute force


def test_bruteforce_barker_lengths(orc):
    """E >= floor(N/2) always (parity of C_k); equality holds exactly at the
    Barker lengths 3, 4, 5, 7, 11, 13 among N = 3..20."""
    barker = {3, 4, 5, 7, 11, 13}
    for N in range(3, 21):
        E, n, arg = orc.bruteforce(N)
        assert orc.energy(arg, N) == E
        assert (E == N // 2) == (N in barker)
        assert E >= N // 2
        assert n % 4 == 0 or N <= 2  # complement x reversal orbits (size 2 or 4, paired)


def test_bruteforce_matches_exhaustive_numpy(orc):
    """Exhaustive numpy enumeration (matrix of all 2^N sequences) for N <= 14."""
    for N in range(3, 15):
        idx = np.arange(1 << N, dtype=np.int64)
        S = np.where(((idx[:, None] >> np.arange(N)) & 1) == 1, 1, -1)
        Es = np.zeros(len(idx), dtype=np.int64)
        for k in range(1, N):
            Ck = (S[:, : N - k] * S[:, k:]).sum(axis=1)
            Es += Ck * Ck
        E, n, _ = orc.bruteforce(N)
        assert E == Es.min()
        assert n == int((Es == E).sum())


# ---------------------------------------------------------------- d(S), App. A


def test_table2_skew_deviation(orc):
    """Appendix A, Eq. 9, under the reading: odd N -> rotations only; even N ->
    rotation then one deletion.  Reproduces the d column of all 17 rows."""
    for N, _, _, hx, d in table2_rows():
        assert orc.skew_deviation(orc.hex_to_words(hx, N), N) == d


# ---------------------------------------------------------------- Tabu search


def skew_complete(s):
    """Sec. II.C, 1-based: for N = 2n - 1, s_{n+i} = (-1)^i s_{n-i}, i = 1..n-1."""
    s = np.array(s)
    N = len(s)
    n = (N + 1) // 2
    for i in range(1, n):
        s[(n + i) - 1] = (-1) ** i * s[(n - i) - 1]
    return s


def is_skew(s):
    N = len(s)
    n = (N + 1) // 2
    return N % 2 == 1 and all(s[n + i - 1] == (-1) ** i * s[n - i - 1] for i in range(1, n))


def replay_tabu(orc, start_s, N, trace, seed, instance, g, max_iter, fix_first=False, skew=False):
    """Brute-force replay of one tabu search: every neighbour energy from
    numpy.correlate, the admissible set and its minima enumerated directly,
    the random picks taken from the (pinned) Philox draws.  skew: the moves
    are the free spins 1..n of Sec. II.C, each flipped with its partner."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    s = skew_complete(start_s) if skew else np.array(start_s)
    E_best = np_energy(s)[0]
    best = s.copy()
    moves = (N + 1) // 2 if skew else N
    tabu = np.zeros(moves, dtype=np.int64)
    min_t, max_t = max_iter // 10, (12 * max_iter) // 100

    def flipped(u, i):
        u = u.copy()
        u[i] = -u[i]
        if skew and i != N - 1 - i:
            u[N - 1 - i] = -u[N - 1 - i]
        return u

    for (gg, t, j, E) in trace:
        assert gg == g
        Ej = [np_energy(flipped(s, i))[0] for i in range(moves)]
        adm = [i for i in range(1 if fix_first else 0, moves) if tabu[i] < t or Ej[i] < E_best]
        m = min(Ej[i] for i in adm)
        ties = [i for i in adm if Ej[i] == m]
        x, y, _, _ = orc.philox4x32_10([instance, g, t, 4], key)
        assert j == ties[(int(x) * len(ties)) >> 32]
        assert E == m
        s = flipped(s, j)
        if skew:
            assert is_skew(s)
        tabu[j] = t + min_t + ((int(y) * (max_t - min_t + 1)) >> 32)
        if E < E_best:  # Algorithm 2: bestSeqTS moves only on a strictly lower energy
            E_best, best = E, s.copy()
    return E_best, best


@pytest.mark.parametrize("N", [5, 8, 11, 16])
def test_tabu_brute_force_replay(orc, N):
    rng = np.random.default_rng(N)
    for trial in range(3):
        s = rand_spins(rng, N)
        seed, inst, g = 1000 + trial, trial, 7
        best, bestE, steps, tr = orc.tabu_run(orc.spins_to_words(s), N, seed, inst, g, trace_cap=1000)
        x = orc.philox4x32_10([inst, g, 1, 2], [seed, 0])[3]
        max_iter = N // 2 + ((int(x) * (N + 1)) >> 32)
        assert steps == max_iter == len(tr)
        E_rep, best_rep = replay_tabu(orc, s, N, tr, seed, inst, g, max_iter)
        assert E_rep == bestE
        assert np.array_equal(orc.words_to_spins(best, N), best_rep)
        assert orc.energy(best, N) == bestE
        assert bestE == min([np_energy(s)[0]] + [int(r[3]) for r in tr])


@pytest.mark.parametrize("N", [3, 4, 7, 20, 64, 65, 128])
def test_tabu_incremental_equals_from_scratch(orc, N):
    rng = np.random.default_rng(100 + N)
    for trial in range(2):
        w = orc.spins_to_words(rand_spins(rng, N))
        a = orc.tabu_run(w, N, 5, trial, 3, incremental=True, trace_cap=4 * N)
        b = orc.tabu_run(w, N, 5, trial, 3, incremental=False, trace_cap=4 * N)
        assert a[1] == b[1] and a[2] == b[2]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])


def test_tabu_fixed_length_and_budget(orc):
    N = 30
    w = orc.spins_to_words(rand_spins(np.random.default_rng(9), N))
    _, _, steps, tr = orc.tabu_run(w, N, 1, 0, 0, max_iter=50, trace_cap=100)
    assert steps == 50 and [int(r[1]) for r in tr] == list(range(1, 51))
    _, _, steps, tr = orc.tabu_run(w, N, 1, 0, 0, max_iter=50, step_budget=17, trace_cap=100)
    assert steps == 17
    _, E0, steps, _ = orc.tabu_run(w, N, 1, 0, 0, max_iter=0)
    assert steps == 0 and E0 == orc.energy(w, N)


# ----------------------------------------------------------------- Memetic-Tabu


def replay_mts(orc, P, seed, inst, res, genlog):
    """Replays Algorithm 1 from the generation log: initial population from
    the INIT draws, tournaments, crossover, mutation draws, the energy of
    every child (numpy), best tracking and replacement."""
    N, K, W = P.N, P.K, orc.words_for(P.N)
    key = [seed & 0xFFFFFFFF, seed >> 32]

    def draw(a, b, purpose, which):
        return int(orc.philox4x32_10([inst, a, b, purpose], key)[which])

    def ri(lo, hi, u):
        return lo + ((u * (hi - lo + 1)) >> 32)

    uniform = bool(P.variant & orc.VARIANT_UNIFORM_CROSSOVER)
    fix = bool(P.variant & orc.VARIANT_FIX_FIRST_SPIN)
    skew = bool(P.variant & orc.VARIANT_SKEW)
    nf = (N + 1) // 2 if skew else N  # spins that crossover and mutation act on
    sym = skew_complete if skew else (lambda v: np.array(v))
    pop = []
    for p in range(K):
        bits = []
        for w in range(W):
            word = draw(p, w, 1, 0) | (draw(p, w, 1, 1) << 32)
            bits += [1 if (word >> b) & 1 else -1 for b in range(64)]
        member = sym(bits[:N])
        if fix and member[0] < 0:  # Sec. II.B: complement so that s_1 = +1
            member = -member
        pop.append(member)
    popE = [np_energy(s)[0] for s in pop]
    bestE = min(popE)
    best = pop[popE.index(bestE)]  # lowest index among the minima
    for L in genlog:
        g = L.g
        pre_mut = orc.words_to_spins(list(L.pre_mut)[:W], N)
        if draw(g, 0, 2, 0) < P.p_comb_u32:
            a, b = ri(0, K - 1, draw(g, 0, 2, 1)), ri(0, K - 1, draw(g, 0, 2, 2))
            c, d = ri(0, K - 1, draw(g, 0, 2, 3)), ri(0, K - 1, draw(g, 1, 2, 0))
            win = lambda x, y: x if (popE[x], x) <= (popE[y], y) else y
            assert L.crossover == 1 and L.p1 == win(a, b) and L.p2 == win(c, d)
            if uniform:
                take2 = np.array([i < nf and draw(g, i // 4, 5, i % 4) < (1 << 31) for i in range(N)])
                expect = sym(np.where(take2, pop[L.p2], pop[L.p1]))
            else:
                cut = ri(1, nf - 1, draw(g, 1, 2, 1))
                assert L.cut == cut
                expect = sym(np.concatenate([pop[L.p1][:cut], pop[L.p2][cut:]]))
        else:
            assert L.crossover == 0 and L.p1 == ri(0, K - 1, draw(g, 1, 2, 2))
            expect = pop[L.p1]
        assert np.array_equal(pre_mut, expect)
        flips = np.array([-1 if j < nf and draw(g, j // 4, 3, j % 4) < P.p_mut_u32 and not (fix and j == 0)
                          else 1 for j in range(N)])
        pre_tabu = orc.words_to_spins(list(L.pre_tabu)[:W], N)
        assert np.array_equal(pre_tabu, sym(pre_mut * flips))
        mi = P.max_iter if P.max_iter >= 0 else nf // 2 + ri(0, nf, draw(g, 1, 2, 3))
        assert L.max_iter == mi and L.min_tabu == mi // 10 and L.max_tabu == (12 * mi) // 100
        child = orc.words_to_spins(list(L.post_tabu)[:W], N)
        assert np_energy(child)[0] == L.E_child <= np_energy(pre_tabu)[0]
        if fix:
            assert child[0] == 1 and pre_tabu[0] == 1
        if skew:
            assert is_skew(child) and is_skew(pre_tabu)
        if L.E_child < bestE:  # Alg. 1: bestSeq changes only on a strictly lower energy
            bestE, best = L.E_child, child
        if P.replace_policy == 0:
            slot = ri(0, K - 1, draw(g, 2, 2, 0))
        else:
            slot = max(range(K), key=lambda p: (popE[p], -p))
        assert L.replace == slot
        pop[slot], popE[slot] = child, L.E_child
    assert res["E"] == bestE == np_energy(orc.words_to_spins(res["seq"], N))[0]
    assert np.array_equal(orc.words_to_spins(res["seq"], N), best)
    assert res["generations"] == len(genlog)
    assert res["steps"] == sum(L.steps for L in genlog)


@pytest.mark.parametrize("policy", [0, 1])
@pytest.mark.parametrize("N,K", [(7, 4), (13, 10), (40, 30), (70, 12)])
def test_mts_replay(orc, N, K, policy):
    P = orc.make_params(N, K, replace_policy=policy, max_generations=30)
    res, tr, gl = orc.mts_run(P, seed=42, instance=3, trace_cap=100000, genlog_cap=100)
    replay_mts(orc, P, 42, 3, res, gl)
    assert res["status"] == orc.STATUS_BUDGET


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("N,K", [(9, 6), (40, 30), (70, 12)])
def test_mts_variants_replay(orc, N, K, variant):
    """Uniform crossover (bit j from P2 iff its CROSS draw < 2^31) and s_1 = +1
    fixed (Sec. II.B): replayed generation by generation; with s_1 fixed no tabu
    step ever flips bit 0."""
    P = orc.make_params(N, K, max_generations=25, variant=variant)
    res, tr, gl = orc.mts_run(P, seed=5, instance=2, trace_cap=100000, genlog_cap=100)
    replay_mts(orc, P, 5, 2, res, gl)
    if variant & orc.VARIANT_FIX_FIRST_SPIN:
        assert all(int(r[2]) != 0 for r in tr if r[1] > 0)
        assert orc.words_to_spins(res["seq"], N)[0] == 1


@pytest.mark.parametrize("N", [6, 11, 16])
def test_tabu_fixed_first_spin_replay(orc, N):
    rng = np.random.default_rng(40 + N)
    s = rand_spins(rng, N)
    best, bestE, steps, tr = orc.tabu_run(orc.spins_to_words(s), N, 7, 1, 2, trace_cap=1000, variant=2)
    x = orc.philox4x32_10([1, 2, 1, 2], [7, 0])[3]
    max_iter = N // 2 + ((int(x) * (N + 1)) >> 32)
    E_rep, best_rep = replay_tabu(orc, s, N, tr, 7, 1, 2, max_iter, fix_first=True)
    assert E_rep == bestE and np.array_equal(orc.words_to_spins(best, N), best_rep)


@pytest.mark.parametrize("N", [3, 5, 9, 15, 21])
@pytest.mark.parametrize("fix", [False, True])
def test_tabu_skew_replay(orc, N, fix):
    """Skew-restricted tabu search (Sec. II.C): pairs of spins flipped together,
    every step replayed by brute force; maxIter = floor(n/2) + randInt(0, n)."""
    rng = np.random.default_rng(70 + N)
    n = (N + 1) // 2
    for trial in range(2):
        s = rand_spins(rng, N)  # the oracle completes it from its free half
        variant = orc.VARIANT_SKEW | (orc.VARIANT_FIX_FIRST_SPIN if fix else 0)
        best, bestE, steps, tr = orc.tabu_run(orc.spins_to_words(s), N, 11, trial, 4, trace_cap=1000,
                                              variant=variant)
        x = orc.philox4x32_10([trial, 4, 1, 2], [11, 0])[3]
        max_iter = n // 2 + ((int(x) * (n + 1)) >> 32)
        assert steps == max_iter == len(tr)
        E_rep, best_rep = replay_tabu(orc, s, N, tr, 11, trial, 4, max_iter, fix_first=fix, skew=True)
        assert E_rep == bestE and np.array_equal(orc.words_to_spins(best, N), best_rep)
        assert is_skew(best_rep)
        C = np_energy(best_rep)[1]
        assert all(C[k - 1] == 0 for k in range(1, N, 2))  # Eq. 4: odd lags vanish


@pytest.mark.parametrize("variant", [4, 5, 6, 7])
@pytest.mark.parametrize("N,K", [(7, 5), (25, 20), (71, 10)])
def test_mts_skew_replay(orc, N, K, variant):
    P = orc.make_params(N, K, max_generations=20, variant=variant)
    assert P.p_mut_u32 == (1 << 32) // ((N + 1) // 2)
    res, tr, gl = orc.mts_run(P, seed=6, instance=3, trace_cap=100000, genlog_cap=100)
    replay_mts(orc, P, 6, 3, res, gl)
    assert is_skew(orc.words_to_spins(res["seq"], N))


def skew_optimum(N):
    """min E over all 2^n skew-symmetric sequences (numpy enumeration)."""
    n = (N + 1) // 2
    codes = np.arange(1 << n, dtype=np.int64)
    free = np.where((codes[:, None] >> np.arange(n)) & 1, 1, -1)
    full = np.empty((len(codes), N), dtype=np.int64)
    full[:, :n] = free
    for i in range(1, n):
        full[:, n + i - 1] = (-1) ** i * full[:, n - i - 1]
    E = np.zeros(len(codes), dtype=np.int64)
    for k in range(1, N):
        E += np.sum(full[:, : N - k] * full[:, k:], axis=1) ** 2
    return int(E.min())


def test_bruteforce_threads_match_single_thread(orc):
    """The chunked exhaustive search gives the single-threaded walk's minimum
    and number of minimisers, whatever the thread count."""
    for N in (8, 13, 20, 24):
        E, n, _ = orc.bruteforce(N)
        for threads in (1, 3, 8):
            assert orc.bruteforce_mt(N, threads) == (E, n)


def test_bruteforce_skew_matches_enumeration(orc):
    """The oracle's exhaustive skew optimum equals the numpy enumeration, and
    its count of minimisers equals the count among all 2^N sequences
    filtered by the skew condition (N = 13, 15, 17)."""
    for N in (3, 5, 7, 9, 11, 13, 19, 21, 25):
        assert orc.bruteforce_skew(N)[0] == skew_optimum(N)
    for N in (13, 15, 17):
        codes = np.arange(1 << N, dtype=np.int64)
        S = np.where((codes[:, None] >> np.arange(N)) & 1, 1, -1)
        n = (N + 1) // 2
        keep = np.ones(len(codes), dtype=bool)
        for i in range(1, n):
            keep &= S[:, n + i - 1] == (-1) ** i * S[:, n - i - 1]
        E = np.array([np_energy(x)[0] for x in S[keep]])
        assert orc.bruteforce_skew(N) == (int(E.min()), int((E == E.min()).sum()))
    with pytest.raises(ValueError):
        orc.bruteforce_skew(20)


def test_skew_optimum_by_filtering():
    """skew_optimum() equals the minimum over all 2^N sequences filtered by the
    skew condition, for N = 13..19."""
    for N in (13, 15, 17, 19):
        codes = np.arange(1 << N, dtype=np.int64)
        S = np.where((codes[:, None] >> np.arange(N)) & 1, 1, -1)
        n = (N + 1) // 2
        keep = np.ones(len(codes), dtype=bool)
        for i in range(1, n):
            keep &= S[:, n + i - 1] == (-1) ** i * S[:, n - i - 1]
        S = S[keep]
        assert len(S) == 1 << n
        assert skew_optimum(N) == min(np_energy(x)[0] for x in S)


@pytest.mark.parametrize("N", [13, 19, 25])
def test_mts_skew_reaches_skew_optimum(orc, N):
    """The restricted search reaches the exhaustive skew-symmetric optimum,
    which is never below the exhaustive unrestricted optimum: equal at N = 13
    (the skew-symmetric Barker length), strictly above it at N = 19 and 25,
    odd lengths whose optima are not skew-symmetric (Sec. II.C)."""
    E_skew = skew_optimum(N)
    E_all = orc.bruteforce(N)[0]
    if N == 13:
        assert E_skew == E_all == 6
    else:
        assert E_skew > E_all
    P = orc.make_params(N, 20, target_E=E_skew, max_generations=3000, variant=orc.VARIANT_SKEW)
    res, _, _ = orc.mts_run(P, seed=2)
    assert res["E"] == E_skew and res["status"] == orc.STATUS_REACHED


def test_skew_variant_refuses_even_N(orc):
    with pytest.raises(Exception):
        orc.mts_run(orc.make_params(20, 5, max_generations=1, variant=orc.VARIANT_SKEW), 0)
    with pytest.raises(Exception):
        orc.tabu_run(orc.spins_to_words(np.ones(20, dtype=np.int64)), 20, 0, 0, variant=orc.VARIANT_SKEW)


@pytest.mark.parametrize("N", [5, 12, 33, 66])
def test_mts_incremental_equals_from_scratch(orc, N):
    P = orc.make_params(N, 8, max_generations=12)
    a = orc.mts_run(P, seed=9, instance=1, incremental=True, trace_cap=100000)
    b = orc.mts_run(P, seed=9, instance=1, incremental=False, trace_cap=100000)
    assert a[0]["E"] == b[0]["E"] and np.array_equal(a[0]["seq"], b[0]["seq"])
    assert np.array_equal(a[1], b[1])


def test_mts_step_budget_and_target(orc):
    N = 40
    P = orc.make_params(N, 20, max_steps=777)
    res, tr, gl = orc.mts_run(P, seed=1, trace_cap=100000, genlog_cap=1000)
    assert res["steps"] == 777 == sum(1 for r in tr if r[1] > 0)
    replay_mts(orc, P, 1, 0, res, gl)
    # a target already met by the initial population: zero generations
    P1 = orc.make_params(N, 20, target_E=10**6)
    r1, _, _ = orc.mts_run(P1, seed=1)
    assert r1["generations"] == 0 and r1["status"] == orc.STATUS_REACHED
    # a reachable target stops at the first generation whose child meets it
    target = res["E"]
    P2 = orc.make_params(N, 20, target_E=target, max_steps=10**7)
    r2, _, gl2 = orc.mts_run(P2, seed=1, genlog_cap=10**5)
    assert r2["status"] == orc.STATUS_REACHED and r2["E"] <= target
    assert gl2[-1].E_child <= target
    assert all(L.E_child > target for L in gl2[:-1])


@pytest.mark.slow
def test_plain_n24_reaches_bruteforce_optimum(orc):
    """N=24, K=100, seed 0, 2,000 generations: the best E equals the exhaustive optimum."""
    E_opt, _, _ = orc.bruteforce(24)
    P = orc.make_params(24, 100, max_generations=2000)
    res, _, _ = orc.mts_run(P, seed=0)
    assert res["E"] == E_opt
