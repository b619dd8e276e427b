"""Planted mistakes: each is a plausible error in the oracle (a wrong sign,
index, bound, constant or rule) planted in a copy of labs_oracle.c; the
copy is compiled and the oracle's pins (tests/test_oracle_pins.py) are run
against it in a child process with LABS_ORACLE_LIB pointing at it.  Every
mutant must make at least one pin fail, so a pin set that would let such a
mistake through is caught here.  CPU only; the mutants run in parallel."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

pytestmark = pytest.mark.slow

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "labs_oracle.c")

# (name, text in labs_oracle.c, replacement, occurrences to replace: 1 = first, 0 = all)
MUTANTS = [
    ("philox multiplier M0", "M0 = 0xD2511F53u", "M0 = 0xD2511F55u", 1),
    ("philox multiplier M1", "M1 = 0xCD9E8D57u", "M1 = 0xCD9E8D47u", 1),
    ("philox Weyl W0", "W0 = 0x9E3779B9u", "W0 = 0x9E3779B8u", 1),
    ("philox Weyl W1", "W1 = 0xBB67AE85u", "W1 = 0xBB67AE95u", 1),
    ("philox key words swapped", "uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};",
     "uint32_t key[2] = {(uint32_t)(seed >> 32), (uint32_t)seed};", 1),
    ("dropped boundary term of C_k", "for (int i = 0; i + k < N; ++i) Ck += s[i] * s[i + k];",
     "for (int i = 0; i + k < N - 1; ++i) Ck += s[i] * s[i + k];", 1),
    ("tableC: lower row entry dropped at i = 0", "if (j - k >= 0) c -= 2 * T->table[k][j - k];",
     "if (j - k > 0) c -= 2 * T->table[k][j - k];", 1),
    ("maxIter range one short", "return N / 2 + rand_int(0, N, u);", "return N / 2 + rand_int(0, N - 1, u);", 1),
    ("tenure 0.11 instead of 0.12", "info.max_tabu = (12 * info.max_iter) / 100;",
     "info.max_tabu = (11 * info.max_iter) / 100;", 1),
    ("tabu test <= instead of <", "int adm = tabu_list[j] < t || Ej[j] < E_best;",
     "int adm = tabu_list[j] <= t || Ej[j] < E_best;", 0),
    ("aspiration <= instead of <", "int adm = tabu_list[j] < t || Ej[j] < E_best;",
     "int adm = tabu_list[j] < t || Ej[j] <= E_best;", 0),
    ("reversed tie order", "if (seen == pick) {\n                    i_sel = j;",
     "if (seen == count - 1 - pick) {\n                    i_sel = j;", 1),
    ("non-strict bestSeqTS update", "if (E_pivot < E_best) {", "if (E_pivot <= E_best) {", 1),
    ("tournament ties to the higher index", "return a < b ? a : b;", "return a < b ? b : a;", 1),
    ("cut range starts at 0", "int cut = rand_int(1, nfree - 1,", "int cut = rand_int(0, nfree - 1,", 1),
    ("cut range one too long", "int cut = rand_int(1, nfree - 1,", "int cut = rand_int(1, nfree,", 1),
    ("crossover parents swapped", "child[i] = i < cut ? pop[(size_t)p1 * N + i] : pop[(size_t)p2 * N + i];",
     "child[i] = i < cut ? pop[(size_t)p2 * N + i] : pop[(size_t)p1 * N + i];", 1),
    ("mutation draw counter shifted", "draw(seed, instance, gg, (uint32_t)(j / 4), ORC_PURPOSE_MUT, j % 4)",
     "draw(seed, instance, gg, (uint32_t)(j / 4) + 1, ORC_PURPOSE_MUT, j % 4)", 1),
    ("non-strict bestSeq update", "if (E_child < E_best) {", "if (E_child <= E_best) {", 1),
    ("replacement rules swapped", "if (P->replace_policy == ORC_REPLACE_RANDOM) {\n            slot",
     "if (P->replace_policy != ORC_REPLACE_RANDOM) {\n            slot", 1),
    ("skew completion sign", "s[c + i] = (int8_t)((i & 1) ? -s[c - i] : s[c - i]);",
     "s[c + i] = (int8_t)((i & 1) ? s[c - i] : -s[c - i]);", 1),
    ("skew move without its partner", "if (i_sel < c) pivot[N - 1 - i_sel] = (int8_t)-pivot[N - 1 - i_sel];",
     "", 1),
    ("skew maxIter from N instead of n", "info.max_iter = tabu_len(n, seed,", "info.max_iter = tabu_len(N, seed,", 1),
]


def _mutate(src: str, old: str, new: str, count: int) -> str:
    assert old in src, old
    return src.replace(old, new) if count == 0 else src.replace(old, new, count)


def _caught(name: str, text: str, tmp: str) -> tuple[str, bool, str]:
    d = tempfile.mkdtemp(dir=tmp)
    c, so = os.path.join(d, "labs_oracle.c"), os.path.join(d, "liblabs_oracle.so")
    open(c, "w").write(text)
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-I",
                           os.path.join(ROOT, "oracle"), "-o", so, c])
    env = dict(os.environ, LABS_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True)
    return name, r.returncode != 0, r.stdout[-300:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(SRC).read()
    texts = [(name, _mutate(src, old, new, n)) for name, old, new, n in MUTANTS]
    assert all(t != src for _, t in texts)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda nt: _caught(nt[0], nt[1], str(tmp_path)), texts))
    missed = [(name, tail) for name, caught, tail in results if not caught]
    assert not missed, missed


def test_unmodified_copy_passes_the_pins(tmp_path):
    """The harness itself: the oracle compiled the same way from an unchanged copy passes."""
    name, caught, tail = _caught("unmodified", open(SRC).read(), str(tmp_path))
    assert not caught, tail
