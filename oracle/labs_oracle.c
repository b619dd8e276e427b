/*
 * labs_oracle.c -- CPU oracle for the LABS memetic tabu search (MTS).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.
 *
 * Everything here works on plain int8 spin arrays s[0..N-1] (s[i] is the
 * paper's s_{i+1}) and follows arXiv 2504.00987 step by step; the packed
 * uint64 format only appears at the function boundary.  No blocking, no
 * bit tricks, no reordering of the algorithm's steps.
 */
#include "labs_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 and Philox4x64-10 (Salmon et al., SC'11).                   */
/* A round multiplies counter words 0 and 2 by fixed odd constants, and      */
/* produces (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)). */
/* Between rounds the key is bumped by the Weyl constants (golden ratio and  */
/* sqrt(3) - 1, scaled to the word size).                                    */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t y0 = (uint64_t)(p1 >> 64) ^ x1 ^ k0;
        uint64_t y1 = (uint64_t)p1;
        uint64_t y2 = (uint64_t)(p0 >> 64) ^ x3 ^ k1;
        uint64_t y3 = (uint64_t)p0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

void orc_philox4x32_batch(const uint32_t* ctr, int64_t B, uint64_t seed, uint32_t* out) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < B; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* One draw of the RNG contract: word `which` of Philox4x32-10 at counter
 * (instance, a, b, purpose) under key (seed lo, seed hi). */
static uint32_t draw(uint64_t seed, uint32_t instance, uint32_t a, uint32_t b, uint32_t purpose,
                     int which) {
    uint32_t ctr[4] = {instance, a, b, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[which];
}

/* randInt(lo, hi), inclusive: lo + floor(u * (hi - lo + 1) / 2^32). */
static int32_t rand_int(int32_t lo, int32_t hi, uint32_t u) {
    uint64_t span = (uint64_t)(int64_t)(hi - lo + 1);
    return lo + (int32_t)(((uint64_t)u * span) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Sequences                                                                 */
/* ------------------------------------------------------------------------ */

static int words_for(int32_t N) { return (N + 63) / 64; }

static void unpack(const uint64_t* words, int32_t N, int8_t* s) {
    for (int i = 0; i < N; ++i) s[i] = ((words[i / 64] >> (i % 64)) & 1u) ? 1 : -1;
}

static void pack(const int8_t* s, int32_t N, uint64_t* words) {
    for (int w = 0; w < ORC_MAX_W; ++w) words[w] = 0;
    for (int i = 0; i < N; ++i)
        if (s[i] > 0) words[i / 64] |= (uint64_t)1 << (i % 64);
}

/* Eq. 1: C_k = sum_{i=1}^{N-k} s_i s_{i+k};  Eq. 2: E = sum_{k=1}^{N-1} C_k^2. */
static int64_t energy_spins(const int8_t* s, int32_t N, int32_t* C) {
    int64_t E = 0;
    for (int k = 1; k <= N - 1; ++k) {
        int32_t Ck = 0;
        for (int i = 0; i + k < N; ++i) Ck += s[i] * s[i + k];
        if (C) C[k - 1] = Ck;
        E += (int64_t)Ck * Ck;
    }
    return E;
}

int64_t orc_energy(const uint64_t* words, int32_t N, int32_t* C) {
    if (N < 1 || N > ORC_MAX_N || !words) return -1;
    int8_t s[ORC_MAX_N];
    unpack(words, N, s);
    return energy_spins(s, N, C);
}

int32_t orc_neighbour_energies(const uint64_t* words, int32_t N, int32_t* E_out) {
    if (N < 2 || N > ORC_MAX_N || !words || !E_out) return -1;
    int8_t s[ORC_MAX_N];
    unpack(words, N, s);
    for (int j = 0; j < N; ++j) {
        s[j] = (int8_t)-s[j];
        E_out[j] = (int32_t)energy_spins(s, N, 0);
        s[j] = (int8_t)-s[j];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* tableC / vectorC (Table I): row k holds the products s_i s_{i+k},         */
/* i = 0..N-1-k, and vectorC[k] is the row sum, i.e. C_k.                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t N;
    int8_t table[ORC_MAX_N][ORC_MAX_N]; /* table[k][i], 1 <= k <= N-1 */
    int32_t vec[ORC_MAX_N];             /* vec[k] = C_k */
} tablec;

static void tablec_build(tablec* T, const int8_t* s, int32_t N) {
    T->N = N;
    for (int k = 1; k <= N - 1; ++k) {
        int32_t sum = 0;
        for (int i = 0; i + k < N; ++i) {
            T->table[k][i] = (int8_t)(s[i] * s[i + k]);
            sum += T->table[k][i];
        }
        T->vec[k] = sum;
    }
}

/* E(flip(pivot, j)): flipping s_j negates the two products of row k that
 * contain s_j, namely entries i = j (if j + k < N) and i = j - k (if j >= k). */
static int32_t tablec_flip_energy(const tablec* T, int j) {
    const int32_t N = T->N;
    int64_t E = 0;
    for (int k = 1; k <= N - 1; ++k) {
        int32_t c = T->vec[k];
        if (j + k < N) c -= 2 * T->table[k][j];
        if (j - k >= 0) c -= 2 * T->table[k][j - k];
        E += (int64_t)c * c;
    }
    return (int32_t)E;
}

/* Apply the flip of s_j to tableC / vectorC: O(N), one entry per row changes
 * on each side of the flipped spin. */
static void tablec_flip(tablec* T, int j) {
    const int32_t N = T->N;
    for (int k = 1; k <= N - 1; ++k) {
        if (j + k < N) {
            T->vec[k] -= 2 * T->table[k][j];
            T->table[k][j] = (int8_t)-T->table[k][j];
        }
        if (j - k >= 0) {
            T->vec[k] -= 2 * T->table[k][j - k];
            T->table[k][j - k] = (int8_t)-T->table[k][j - k];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Tabu search, Algorithm 2.                                                 */
/*                                                                           */
/* Readings where the paper is silent or differs between Algorithms 2 and 4: */
/*  - maxIter = floor(N/2) + randInt(0, N) (Algorithm 4; same range as the   */
/*    randInt[N/2, 3N/2] of Sec. III.B);                                     */
/*  - minTabu = floor(maxIter/10), maxTabu = floor(12*maxIter/100), integer  */
/*    arithmetic, tenure drawn inclusive;                                    */
/*  - bit i is admissible at step t iff tabuList[i] < t, or if flipping it   */
/*    gives an energy strictly below E(bestSeqTS) (aspiration);              */
/*  - ties among the admissible minima: the pick-th of them in ascending     */
/*    index order, pick = floor(u * count / 2^32) with u the step's tie draw; */
/*  - bestSeqTS starts as the input and is replaced only on a strictly       */
/*    lower energy.                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t steps;
    int32_t max_iter, min_tabu, max_tabu;
} tabu_info;

static int32_t tabu_len(int32_t N, uint64_t seed, uint32_t instance, uint32_t g, int32_t max_iter) {
    if (max_iter >= 0) return max_iter;
    uint32_t u = draw(seed, instance, g, 1u, ORC_PURPOSE_GEN, 3);
    return N / 2 + rand_int(0, N, u);
}

/* s: in = start sequence, out = bestSeqTS.  *E: in = E(start), out = E(best). */
/* fix_first: s_1 is never flipped (Sec. II.B symmetry break variant). */
static tabu_info tabu_search(int8_t* s, int32_t N, int32_t* E, uint64_t seed, uint32_t instance,
                             uint32_t g, int32_t max_iter_opt, int64_t step_budget,
                             int32_t incremental, int32_t fix_first, int32_t* trace,
                             int64_t trace_cap, int64_t* trace_len) {
    tabu_info info;
    int8_t pivot[ORC_MAX_N], best[ORC_MAX_N];
    int32_t tabu_list[ORC_MAX_N];
    int32_t Ej[ORC_MAX_N];
    static __thread tablec T; /* large; one per thread */

    info.max_iter = tabu_len(N, seed, instance, g, max_iter_opt);
    info.min_tabu = info.max_iter / 10;
    info.max_tabu = (12 * info.max_iter) / 100;
    info.steps = 0;

    memcpy(pivot, s, (size_t)N);
    memcpy(best, s, (size_t)N);
    for (int i = 0; i < N; ++i) tabu_list[i] = 0;
    int32_t E_best = *E;
    if (incremental) tablec_build(&T, pivot, N);

    for (int32_t t = 1; t <= info.max_iter; ++t) {
        if (step_budget >= 0 && info.steps >= step_budget) break;

        /* Energies of all N neighbours of the pivot. */
        for (int j = 0; j < N; ++j) {
            if (incremental) {
                Ej[j] = tablec_flip_energy(&T, j);
            } else {
                pivot[j] = (int8_t)-pivot[j];
                Ej[j] = (int32_t)energy_spins(pivot, N, 0);
                pivot[j] = (int8_t)-pivot[j];
            }
        }
        /* Admissible minimum and its ties, ascending index order. */
        int32_t m = INT32_MAX, count = 0;
        const int j0 = fix_first ? 1 : 0;
        for (int j = j0; j < N; ++j) {
            int adm = tabu_list[j] < t || Ej[j] < E_best;
            if (adm && Ej[j] < m) m = Ej[j];
        }
        for (int j = j0; j < N; ++j) {
            int adm = tabu_list[j] < t || Ej[j] < E_best;
            if (adm && Ej[j] == m) ++count;
        }
        if (count == 0) break; /* cannot happen: maxTabu < N leaves a free bit */
        uint32_t u_tie = draw(seed, instance, g, (uint32_t)t, ORC_PURPOSE_STEP, 0);
        uint32_t u_ten = draw(seed, instance, g, (uint32_t)t, ORC_PURPOSE_STEP, 1);
        int32_t pick = (int32_t)(((uint64_t)u_tie * (uint64_t)count) >> 32);
        int i_sel = -1;
        for (int j = j0, seen = 0; j < N; ++j) {
            int adm = tabu_list[j] < t || Ej[j] < E_best;
            if (adm && Ej[j] == m) {
                if (seen == pick) {
                    i_sel = j;
                    break;
                }
                ++seen;
            }
        }
        /* pivot <- flip(pivot, i); tabuList[i] = t + randInt(minTabu, maxTabu). */
        pivot[i_sel] = (int8_t)-pivot[i_sel];
        if (incremental) tablec_flip(&T, i_sel);
        tabu_list[i_sel] = t + rand_int(info.min_tabu, info.max_tabu, u_ten);
        int32_t E_pivot = m;
        if (E_pivot < E_best) {
            E_best = E_pivot;
            memcpy(best, pivot, (size_t)N);
        }
        ++info.steps;
        if (trace && trace_len && *trace_len < trace_cap) {
            int32_t* r = trace + 4 * (*trace_len);
            r[0] = (int32_t)g;
            r[1] = t;
            r[2] = i_sel;
            r[3] = E_pivot;
            ++*trace_len;
        }
    }
    memcpy(s, best, (size_t)N);
    *E = E_best;
    return info;
}

/* ------------------------------------------------------------------------ */
/* Skew-symmetric restriction (Sec. II.C).  For odd N = 2n - 1 a sequence is */
/* skew-symmetric iff s_{n+i} = (-1)^i s_{n-i} for i = 1..n-1; 0-based with  */
/* centre c = n - 1 that is s[c+i] = (-1)^i s[c-i].  The n spins s[0..c]   */
/* are free and determine the rest.                                          */
/* ------------------------------------------------------------------------ */

/* Rewrites s[c+1..N-1] from the free half s[0..c-1]. */
static void symmetrize(int8_t* s, int32_t N) {
    const int c = (N - 1) / 2;
    for (int i = 1; i <= c; ++i) s[c + i] = (int8_t)((i & 1) ? -s[c - i] : s[c - i]);
}

/* Tabu search over skew-symmetric sequences: move i (0 <= i <= c) flips the
 * free spin s[i] and, for i < c, its partner s[N-1-i], so the pivot stays
 * skew-symmetric.  Everything else is Algorithm 2 as read above, over the n
 * moves: maxIter = floor(n/2) + randInt(0, n) unless given, the tenure
 * bounds from maxIter, tabuList indexed by move, the same admissibility,
 * ties and draws.  Neighbour energies straight from Eq. 2. */
static tabu_info tabu_search_skew(int8_t* s, int32_t N, int32_t* E, uint64_t seed,
                                  uint32_t instance, uint32_t g, int32_t max_iter_opt,
                                  int64_t step_budget, int32_t fix_first, int32_t* trace,
                                  int64_t trace_cap, int64_t* trace_len) {
    tabu_info info;
    const int c = (N - 1) / 2, n = c + 1;
    int8_t pivot[ORC_MAX_N], best[ORC_MAX_N];
    int32_t tabu_list[ORC_MAX_N];
    int32_t Ei[ORC_MAX_N];

    info.max_iter = tabu_len(n, seed, instance, g, max_iter_opt);
    info.min_tabu = info.max_iter / 10;
    info.max_tabu = (12 * info.max_iter) / 100;
    info.steps = 0;

    memcpy(pivot, s, (size_t)N);
    memcpy(best, s, (size_t)N);
    for (int i = 0; i < n; ++i) tabu_list[i] = 0;
    int32_t E_best = *E;

    for (int32_t t = 1; t <= info.max_iter; ++t) {
        if (step_budget >= 0 && info.steps >= step_budget) break;
        /* Energies of the n neighbours: flip s[i] and its partner. */
        for (int i = 0; i < n; ++i) {
            pivot[i] = (int8_t)-pivot[i];
            if (i < c) pivot[N - 1 - i] = (int8_t)-pivot[N - 1 - i];
            Ei[i] = (int32_t)energy_spins(pivot, N, 0);
            pivot[i] = (int8_t)-pivot[i];
            if (i < c) pivot[N - 1 - i] = (int8_t)-pivot[N - 1 - i];
        }
        int32_t m = INT32_MAX, count = 0;
        const int i0 = fix_first ? 1 : 0;
        for (int i = i0; i < n; ++i) {
            int adm = tabu_list[i] < t || Ei[i] < E_best;
            if (adm && Ei[i] < m) m = Ei[i];
        }
        for (int i = i0; i < n; ++i) {
            int adm = tabu_list[i] < t || Ei[i] < E_best;
            if (adm && Ei[i] == m) ++count;
        }
        if (count == 0) break; /* cannot happen while maxTabu < n - 1 */
        uint32_t u_tie = draw(seed, instance, g, (uint32_t)t, ORC_PURPOSE_STEP, 0);
        uint32_t u_ten = draw(seed, instance, g, (uint32_t)t, ORC_PURPOSE_STEP, 1);
        int32_t pick = (int32_t)(((uint64_t)u_tie * (uint64_t)count) >> 32);
        int i_sel = -1;
        for (int i = i0, seen = 0; i < n; ++i) {
            int adm = tabu_list[i] < t || Ei[i] < E_best;
            if (adm && Ei[i] == m) {
                if (seen == pick) {
                    i_sel = i;
                    break;
                }
                ++seen;
            }
        }
        if (i_sel < 0) break; /* unreachable: pick < count */
        pivot[i_sel] = (int8_t)-pivot[i_sel];
        if (i_sel < c) pivot[N - 1 - i_sel] = (int8_t)-pivot[N - 1 - i_sel];
        tabu_list[i_sel] = t + rand_int(info.min_tabu, info.max_tabu, u_ten);
        if (m < E_best) {
            E_best = m;
            memcpy(best, pivot, (size_t)N);
        }
        ++info.steps;
        if (trace && trace_len && *trace_len < trace_cap) {
            int32_t* r = trace + 4 * (*trace_len);
            r[0] = (int32_t)g;
            r[1] = t;
            r[2] = i_sel;
            r[3] = m;
            ++*trace_len;
        }
    }
    memcpy(s, best, (size_t)N);
    *E = E_best;
    return info;
}

int64_t orc_tabu_run(const uint64_t* start, int32_t N, uint64_t seed, uint32_t instance,
                     uint32_t g, int32_t max_iter, int64_t step_budget, int32_t incremental,
                     uint64_t* best_out, int32_t* bestE_out, int32_t* trace, int64_t trace_cap,
                     int64_t* trace_len) {
    return orc_tabu_run_v(start, N, seed, instance, g, max_iter, step_budget, incremental, 0,
                          best_out, bestE_out, trace, trace_cap, trace_len);
}

int64_t orc_tabu_run_v(const uint64_t* start, int32_t N, uint64_t seed, uint32_t instance,
                       uint32_t g, int32_t max_iter, int64_t step_budget, int32_t incremental,
                       int32_t variant, uint64_t* best_out, int32_t* bestE_out, int32_t* trace,
                       int64_t trace_cap, int64_t* trace_len) {
    if (N < 3 || N > ORC_MAX_N || !start) return -1;
    const int skew = (variant & ORC_VARIANT_SKEW) != 0;
    if (skew && N % 2 == 0) return -1;
    int8_t s[ORC_MAX_N];
    unpack(start, N, s);
    if (skew) symmetrize(s, N); /* the start's free half decides */
    int32_t E = (int32_t)energy_spins(s, N, 0);
    if (trace_len) *trace_len = 0;
    const int fix = (variant & ORC_VARIANT_FIX_FIRST_SPIN) != 0;
    tabu_info info = skew ? tabu_search_skew(s, N, &E, seed, instance, g, max_iter, step_budget, fix,
                                             trace, trace_cap, trace_len)
                          : tabu_search(s, N, &E, seed, instance, g, max_iter, step_budget,
                                        incremental, fix, trace, trace_cap, trace_len);
    if (best_out) pack(s, N, best_out);
    if (bestE_out) *bestE_out = E;
    return info.steps;
}

/* ------------------------------------------------------------------------ */
/* Memetic-Tabu, Algorithm 1.                                                */
/*                                                                           */
/* Readings of the steps the paper names but does not define:               */
/*  - initial member p, word w: Philox(instance, p, w, INIT) words 0 and 1   */
/*    as the low and high halves, bits >= N cleared;                         */
/*  - randReal(0,1) < p_comb  <->  coin draw < p_comb_u32;                   */
/*  - selectParents: two binary tournaments with replacement, the lower E   */
/*    wins, equal E goes to the lower index;                                 */
/*  - Combine: one-point crossover, child = P1 bits [0,c) and P2 bits [c,N), */
/*    c = randInt(1, N-1);                                                   */
/*  - Sample: a uniformly drawn member;                                      */
/*  - Mutate: bit j flips iff its draw < p_mut_u32 (floor(2^32/N) ~ 1/N);    */
/*  - bestSeq is replaced only on a strictly lower energy;                   */
/*  - the child replaces a uniformly drawn member (Algorithm 1), or the      */
/*    highest-E member, lowest index on ties (replace-worst variant);        */
/*  - a step budget may end a tabu search early; that generation still      */
/*    completes with the partial bestSeqTS.                                  */
/* Variants: uniform crossover takes bit j from P2 iff word j%4 of           */
/* (instance, g, j/4, CROSS) < 2^31; fixing s_1 = +1 complements the initial */
/* members with s_1 = -1 (E is unchanged, Sec. II.B), never mutates s_1 and  */
/* never flips it in the tabu search.  The skew variant (odd N) keeps every */
/* sequence skew-symmetric: initial members are symmetrized, the cut is     */
/* randInt(1, n-1) and mutation and uniform crossover act on the n free     */
/* spins, the child is symmetrized, and the tabu search is the skew one.    */
/* Draw layout per generation g:                                             */
/*   GEN(g,0): x coin, y tournament a, z tournament b, w tournament c        */
/*   GEN(g,1): x tournament d, y cut, z sample, w maxIter                    */
/*   GEN(g,2): x replacement slot                                            */
/* ------------------------------------------------------------------------ */

static int tournament(const int32_t* E, int a, int b) {
    if (E[a] < E[b]) return a;
    if (E[b] < E[a]) return b;
    return a < b ? a : b;
}

static int params_ok(const orc_params* P) {
    if (!P) return 0;
    if (P->N < 3 || P->N > ORC_MAX_N) return 0;
    if (P->K < 1 || P->K > ORC_MAX_K) return 0;
    if (P->replace_policy != ORC_REPLACE_RANDOM && P->replace_policy != ORC_REPLACE_WORST) return 0;
    if (P->target_E < 0 && P->max_generations < 0 && P->max_steps < 0) return 0;
    if (P->variant & ~(ORC_VARIANT_UNIFORM_CROSSOVER | ORC_VARIANT_FIX_FIRST_SPIN | ORC_VARIANT_SKEW))
        return 0;
    if ((P->variant & ORC_VARIANT_SKEW) && P->N % 2 == 0) return 0;
    return 1;
}

int32_t orc_mts_run(const orc_params* P, uint64_t seed, uint32_t instance, int32_t incremental,
                    orc_result* res, int32_t* trace, int64_t trace_cap, int64_t* trace_len,
                    orc_genlog* genlog, int64_t genlog_cap, int64_t* genlog_len) {
    if (!params_ok(P) || !res) return -1;
    const int32_t N = P->N, K = P->K, W = words_for(N);
    const int skew = (P->variant & ORC_VARIANT_SKEW) != 0;
    const int32_t nfree = skew ? (N + 1) / 2 : N; /* spins crossover and mutation act on */
    int8_t* pop = (int8_t*)malloc((size_t)K * (size_t)N);
    int32_t* popE = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
    if (!pop || !popE) {
        free(pop);
        free(popE);
        return -1;
    }
    if (trace_len) *trace_len = 0;
    if (genlog_len) *genlog_len = 0;

    /* population <- K random binary sequences of length N. */
    for (int p = 0; p < K; ++p) {
        uint64_t words[ORC_MAX_W] = {0, 0, 0, 0};
        for (int w = 0; w < W; ++w) {
            uint32_t lo = draw(seed, instance, (uint32_t)p, (uint32_t)w, ORC_PURPOSE_INIT, 0);
            uint32_t hi = draw(seed, instance, (uint32_t)p, (uint32_t)w, ORC_PURPOSE_INIT, 1);
            words[w] = (uint64_t)lo | ((uint64_t)hi << 32);
        }
        unpack(words, N, pop + (size_t)p * N);
        if (skew) symmetrize(pop + (size_t)p * N, N);
        if ((P->variant & ORC_VARIANT_FIX_FIRST_SPIN) && pop[(size_t)p * N] < 0)
            for (int i = 0; i < N; ++i) pop[(size_t)p * N + i] = (int8_t)-pop[(size_t)p * N + i];
        popE[p] = (int32_t)energy_spins(pop + (size_t)p * N, N, 0);
    }
    /* bestSeq <- the lowest-energy member (lowest index on ties). */
    int best_idx = 0;
    for (int p = 1; p < K; ++p)
        if (popE[p] < popE[best_idx]) best_idx = p;
    int8_t best[ORC_MAX_N];
    memcpy(best, pop + (size_t)best_idx * N, (size_t)N);
    int32_t E_best = popE[best_idx];

    int64_t g = 0, steps = 0;
    int32_t status = ORC_STATUS_BUDGET;
    for (;;) {
        if (P->target_E >= 0 && E_best <= P->target_E) {
            status = ORC_STATUS_REACHED;
            break;
        }
        if (P->max_generations >= 0 && g >= P->max_generations) break;
        if (P->max_steps >= 0 && steps >= P->max_steps) break;

        const uint32_t gg = (uint32_t)g;
        int8_t child[ORC_MAX_N];
        orc_genlog L;
        memset(&L, 0, sizeof L);
        L.g = (int32_t)g;

        uint32_t coin = draw(seed, instance, gg, 0, ORC_PURPOSE_GEN, 0);
        if (coin < P->p_comb_u32) {
            int a = rand_int(0, K - 1, draw(seed, instance, gg, 0, ORC_PURPOSE_GEN, 1));
            int b = rand_int(0, K - 1, draw(seed, instance, gg, 0, ORC_PURPOSE_GEN, 2));
            int c = rand_int(0, K - 1, draw(seed, instance, gg, 0, ORC_PURPOSE_GEN, 3));
            int d = rand_int(0, K - 1, draw(seed, instance, gg, 1, ORC_PURPOSE_GEN, 0));
            int p1 = tournament(popE, a, b);
            int p2 = tournament(popE, c, d);
            int cut = rand_int(1, nfree - 1, draw(seed, instance, gg, 1, ORC_PURPOSE_GEN, 1));
            if (P->variant & ORC_VARIANT_UNIFORM_CROSSOVER) {
                cut = 0;
                for (int i = 0; i < nfree; ++i) {
                    uint32_t u = draw(seed, instance, gg, (uint32_t)(i / 4), ORC_PURPOSE_CROSS, i % 4);
                    child[i] = u < 0x80000000u ? pop[(size_t)p2 * N + i] : pop[(size_t)p1 * N + i];
                }
            } else {
                for (int i = 0; i < N; ++i)
                    child[i] = i < cut ? pop[(size_t)p1 * N + i] : pop[(size_t)p2 * N + i];
            }
            if (skew) symmetrize(child, N);
            L.crossover = 1;
            L.p1 = p1;
            L.p2 = p2;
            L.cut = cut;
        } else {
            int p = rand_int(0, K - 1, draw(seed, instance, gg, 1, ORC_PURPOSE_GEN, 2));
            memcpy(child, pop + (size_t)p * N, (size_t)N);
            L.p1 = p;
        }
        pack(child, N, L.pre_mut);

        /* Mutate(child, p_mutate): independent flip per bit. */
        for (int j = (P->variant & ORC_VARIANT_FIX_FIRST_SPIN) ? 1 : 0; j < nfree; ++j) {
            uint32_t u = draw(seed, instance, gg, (uint32_t)(j / 4), ORC_PURPOSE_MUT, j % 4);
            if (u < P->p_mut_u32) child[j] = (int8_t)-child[j];
        }
        if (skew) symmetrize(child, N);
        pack(child, N, L.pre_tabu);

        /* child <- Tabu-Search(child). */
        int32_t E_child = (int32_t)energy_spins(child, N, 0);
        int64_t budget = P->max_steps >= 0 ? P->max_steps - steps : -1;
        const int fix = (P->variant & ORC_VARIANT_FIX_FIRST_SPIN) != 0;
        tabu_info ti = skew ? tabu_search_skew(child, N, &E_child, seed, instance, gg, P->max_iter,
                                               budget, fix, trace, trace_cap, trace_len)
                            : tabu_search(child, N, &E_child, seed, instance, gg, P->max_iter,
                                          budget, incremental, fix, trace, trace_cap, trace_len);
        steps += ti.steps;
        pack(child, N, L.post_tabu);

        /* update bestSeq to child if E(bestSeq) > E(child). */
        if (E_child < E_best) {
            E_best = E_child;
            memcpy(best, child, (size_t)N);
        }
        /* replace an individual of the population by the child. */
        int slot;
        if (P->replace_policy == ORC_REPLACE_RANDOM) {
            slot = rand_int(0, K - 1, draw(seed, instance, gg, 2, ORC_PURPOSE_GEN, 0));
        } else {
            slot = 0;
            for (int p = 1; p < K; ++p)
                if (popE[p] > popE[slot]) slot = p;
        }
        memcpy(pop + (size_t)slot * N, child, (size_t)N);
        popE[slot] = E_child;

        if (trace && trace_len && *trace_len < trace_cap) {
            int32_t* r = trace + 4 * (*trace_len);
            r[0] = (int32_t)g;
            r[1] = 0;
            r[2] = slot;
            r[3] = E_child;
            ++*trace_len;
        }
        L.max_iter = ti.max_iter;
        L.min_tabu = ti.min_tabu;
        L.max_tabu = ti.max_tabu;
        L.replace = slot;
        L.E_child = E_child;
        L.steps = (int32_t)ti.steps;
        if (genlog && genlog_len && *genlog_len < genlog_cap) genlog[(*genlog_len)++] = L;
        ++g;
    }

    pack(best, N, res->seq);
    res->E = E_best;
    res->status = status;
    res->generations = g;
    res->steps = steps;
    free(pop);
    free(popE);
    return 0;
}

typedef struct {
    const orc_params* P;
    uint64_t seed;
    uint32_t first_instance;
    int32_t replicas, threads, tid;
    orc_result* res;
    int32_t rc;
} many_job;

static void* many_worker(void* arg) {
    many_job* J = (many_job*)arg;
    J->rc = 0;
    for (int r = J->tid; r < J->replicas; r += J->threads)
        if (orc_mts_run(J->P, J->seed, J->first_instance + (uint32_t)r, 1, &J->res[r], 0, 0, 0, 0, 0,
                        0) != 0)
            J->rc = -1;
    return 0;
}

int32_t orc_mts_run_many(const orc_params* P, uint64_t seed, uint32_t first_instance,
                         int32_t replicas, int32_t threads, orc_result* res) {
    if (!params_ok(P) || !res || replicas < 0 || threads < 1) return -1;
    if (threads > replicas) threads = replicas > 0 ? replicas : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    many_job* jobs = (many_job*)malloc(sizeof(many_job) * (size_t)threads);
    if (!th || !jobs) {
        free(th);
        free(jobs);
        return -1;
    }
    for (int i = 0; i < threads; ++i) {
        jobs[i] = (many_job){P, seed, first_instance, replicas, threads, i, res, 0};
        pthread_create(&th[i], 0, many_worker, &jobs[i]);
    }
    int32_t rc = 0;
    for (int i = 0; i < threads; ++i) {
        pthread_join(th[i], 0);
        if (jobs[i].rc) rc = -1;
    }
    free(th);
    free(jobs);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive search (definition of S*, Sec. II).  A reflected Gray code     */
/* visits every sequence with s_N fixed by one flip at a time; C_k is        */
/* brought up to date after each flip from the spins themselves (O(N)).      */
/* Fixing one spin is exact because E is invariant under complementation     */
/* (Sec. II.B).                                                              */
/* ------------------------------------------------------------------------ */

int32_t orc_bruteforce(int32_t N, int32_t* E_min, int64_t* n_min, uint64_t* argmin) {
    if (N < 2 || N > 32 || !E_min) return -1;
    int8_t s[64];
    int32_t C[64];
    for (int i = 0; i < N; ++i) s[i] = 1;
    int64_t E = energy_spins(s, N, C + 1);
    int64_t best = E, count = 1;
    uint64_t best_seq = ((uint64_t)1 << N) - 1;
    const uint64_t total = (uint64_t)1 << (N - 1);
    for (uint64_t step = 1; step < total; ++step) {
        int j = __builtin_ctzll(step); /* Gray code: flip the lowest set bit of step */
        for (int k = 1; k <= N - 1; ++k) {
            int32_t d = 0;
            if (j + k < N) d += s[j + k];
            if (j - k >= 0) d += s[j - k];
            C[k] += -2 * s[j] * d;
        }
        s[j] = (int8_t)-s[j];
        E = 0;
        for (int k = 1; k <= N - 1; ++k) E += (int64_t)C[k] * C[k];
        if (E < best) {
            best = E;
            count = 1;
            best_seq = 0;
            for (int i = 0; i < N; ++i)
                if (s[i] > 0) best_seq |= (uint64_t)1 << i;
        } else if (E == best) {
            ++count;
        }
    }
    *E_min = (int32_t)best;
    /* each minimiser found has its complement outside the enumerated half */
    if (n_min) *n_min = 2 * count;
    if (argmin) *argmin = best_seq;
    return 0;
}

/* The same exhaustive search split over threads: the spins s[N-1-T..N-2]
 * take each of their 2^T values in one chunk (T = 6), and every chunk runs
 * the Gray-code walk above over s[0..N-2-T] from its own start, C_k from
 * scratch.  s[N-1] = +1 as above (complements are equivalent). */
typedef struct {
    int32_t N, T, chunk0, chunks, step;
    int64_t best, count;
} bf_job;

static void* bf_worker(void* arg) {
    bf_job* J = (bf_job*)arg;
    const int32_t N = J->N, low = N - 1 - J->T;
    J->best = -1;
    J->count = 0;
    for (int ch = J->chunk0; ch < J->chunks; ch += J->step) {
        int8_t s[64];
        int32_t C[64];
        for (int i = 0; i < N; ++i) s[i] = 1;
        for (int b = 0; b < J->T; ++b)
            if ((ch >> b) & 1) s[low + b] = -1;
        int64_t E = energy_spins(s, N, C + 1);
        int64_t best = E, count = 1;
        const uint64_t total = (uint64_t)1 << low;
        for (uint64_t step = 1; step < total; ++step) {
            const int j = __builtin_ctzll(step);
            for (int k = 1; k <= N - 1; ++k) {
                int32_t d = 0;
                if (j + k < N) d += s[j + k];
                if (j - k >= 0) d += s[j - k];
                C[k] += -2 * s[j] * d;
            }
            s[j] = (int8_t)-s[j];
            E = 0;
            for (int k = 1; k <= N - 1; ++k) E += (int64_t)C[k] * C[k];
            if (E < best) {
                best = E;
                count = 1;
            } else if (E == best) {
                ++count;
            }
        }
        if (J->best < 0 || best < J->best) {
            J->best = best;
            J->count = count;
        } else if (best == J->best) {
            J->count += count;
        }
    }
    return 0;
}

int32_t orc_bruteforce_mt(int32_t N, int32_t threads, int32_t* E_min, int64_t* n_min) {
    if (N < 8 || N > 40 || threads < 1 || !E_min) return -1;
    const int T = 6, chunks = 1 << T;
    if (threads > chunks) threads = chunks;
    pthread_t th[64];
    bf_job jobs[64];
    for (int i = 0; i < threads; ++i) {
        jobs[i] = (bf_job){N, T, i, chunks, threads, -1, 0};
        pthread_create(&th[i], 0, bf_worker, &jobs[i]);
    }
    int64_t best = -1, count = 0;
    for (int i = 0; i < threads; ++i) {
        pthread_join(th[i], 0);
        if (best < 0 || jobs[i].best < best) {
            best = jobs[i].best;
            count = jobs[i].count;
        } else if (jobs[i].best == best) {
            count += jobs[i].count;
        }
    }
    *E_min = (int32_t)best;
    if (n_min) *n_min = 2 * count;
    return 0;
}

/* Exhaustive minimum of E over the skew-symmetric sequences of odd length N
 * (Sec. II.C): every assignment of the n = (N+1)/2 free spins, completed
 * by symmetrize() and scored from Eq. 2.  n_min counts the minimisers. */
int32_t orc_bruteforce_skew(int32_t N, int32_t* E_min, int64_t* n_min) {
    if (N < 3 || N > 45 || N % 2 == 0 || !E_min) return -1;
    const int n = (N + 1) / 2;
    int8_t s[ORC_MAX_N];
    int64_t best = -1, count = 0;
    for (uint64_t code = 0; code < ((uint64_t)1 << n); ++code) {
        for (int i = 0; i < n; ++i) s[i] = ((code >> i) & 1) ? 1 : -1;
        symmetrize(s, N);
        const int64_t E = energy_spins(s, N, 0);
        if (best < 0 || E < best) {
            best = E;
            count = 1;
        } else if (E == best) {
            ++count;
        }
    }
    *E_min = (int32_t)best;
    if (n_min) *n_min = count;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Appendix A: deviation from skew-symmetry.                                 */
/* Eq. 5: for odd length L = 2n - 1, n_non-skew counts i = 1..n-1 with      */
/*   s_{n+i} != (-1)^i s_{n-i}.                                              */
/* Eq. 6: Rot(S; r) moves the first r spins to the end.                      */
/* Eq. 7, 8: insertion of xi after position i, deletion of position i.      */
/* Eq. 9 reading (odd and even lengths are not separated in the paper):     */
/*   odd N:  min over r of n_non-skew(Rot(S; r));                            */
/*   even N: min over r, i of n_non-skew(Del(Rot(S; r); i)).                 */
/* The mode bits of skew_deviation_mode select the branches explicitly.      */
/* ------------------------------------------------------------------------ */

static int32_t non_skew_spins(const int8_t* s, int32_t L) {
    const int n = (L + 1) / 2; /* L = 2n - 1; s_{m} (1-based) = s[m-1] */
    int32_t cnt = 0;
    for (int i = 1; i <= n - 1; ++i) {
        int sign = (i % 2) ? -1 : 1;
        if (s[n + i - 1] != sign * s[n - i - 1]) ++cnt;
    }
    return cnt;
}

int32_t orc_non_skew_pairs(const uint64_t* words, int32_t N) {
    if (N < 1 || N > ORC_MAX_N || (N % 2) == 0 || !words) return -1;
    int8_t s[ORC_MAX_N];
    unpack(words, N, s);
    return non_skew_spins(s, N);
}

#define SKEW_ROT 1
#define SKEW_INS 2
#define SKEW_DEL 4

int32_t orc_skew_deviation_mode(const uint64_t* words, int32_t N, int32_t mode);

int32_t orc_skew_deviation_mode(const uint64_t* words, int32_t N, int32_t mode) {
    if (N < 2 || N > ORC_MAX_N || !words) return -1;
    int8_t s[ORC_MAX_N], rot[ORC_MAX_N], t[ORC_MAX_N + 1];
    unpack(words, N, s);
    int32_t best = INT32_MAX;
    for (int r = 0; r < N; ++r) {
        for (int i = 0; i < N; ++i) rot[i] = s[(i + r) % N];
        if ((mode & SKEW_ROT) && (N % 2) == 1) {
            int32_t v = non_skew_spins(rot, N);
            if (v < best) best = v;
        }
        if ((mode & SKEW_INS) && (N % 2) == 0) {
            for (int i = 0; i <= N; ++i)
                for (int xi = -1; xi <= 1; xi += 2) {
                    for (int a = 0, b = 0; a <= N; ++a) t[a] = (a == i) ? (int8_t)xi : rot[b++];
                    int32_t v = non_skew_spins(t, N + 1);
                    if (v < best) best = v;
                }
        }
        if ((mode & SKEW_DEL) && (N % 2) == 0) {
            for (int i = 0; i < N; ++i) {
                for (int a = 0, b = 0; b < N; ++b)
                    if (b != i) t[a++] = rot[b];
                int32_t v = non_skew_spins(t, N - 1);
                if (v < best) best = v;
            }
        }
    }
    return best == INT32_MAX ? -1 : best;
}

int32_t orc_skew_deviation(const uint64_t* words, int32_t N) {
    return orc_skew_deviation_mode(words, N, SKEW_ROT | SKEW_DEL);
}
