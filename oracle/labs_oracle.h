/*
 * labs_oracle.h -- CPU oracle for the LABS memetic tabu search (MTS).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * timed CPU baseline of the benchmark may load this library.  The product
 * (the CUDA library and its Python binding) never includes, links or calls
 * anything declared here, and this file includes nothing from the product.
 *
 * What it computes, with the passage of arXiv 2504.00987 it follows:
 *   - C_k and E of a +-1 sequence .......................... Eq. 1, Eq. 2
 *   - merit factor F = N^2 / (2E) ........................... Eq. 3
 *   - Memetic-Tabu (population loop) ........................ Algorithm 1, Sec. III.A
 *   - Tabu-Search ........................................... Algorithm 2, Sec. III.B
 *   - tableC / vectorC incremental neighbour energies ....... Table I, Sec. III.C
 *   - deviation from skew-symmetry d(S) ..................... Appendix A, Eqs. 5-9
 *   - search restricted to skew-symmetric sequences ......... Sec. II.C (variant)
 *   - exhaustive optimum (brute force) for small N .......... Sec. II (definition of S*)
 *
 * Randomness: every random decision is one output word of Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11), written here from that paper's definition, keyed by the 64-bit seed
 * and addressed by a counter (instance, generation-or-member, index, purpose).
 * The counter layout is the contract both sides of the parity tests follow.
 *
 * Sequence format at the interface: N spins s_1..s_N packed LSB-first into
 * ceil(N/64) uint64 words, spin s_{i+1} at bit (i % 64) of word (i / 64),
 * bit 1 <-> s = +1, bits at positions >= N zero.
 */
#ifndef LABS_ORACLE_H
#define LABS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_N 256
#define ORC_MAX_W 4
#define ORC_MAX_K 1024

/* Philox counter word 3: what the draw is for. */
#define ORC_PURPOSE_INIT 1u /* (instance, member p, word w)  -> word bits       */
#define ORC_PURPOSE_GEN 2u  /* (instance, generation g, 0|1|2) -> per-generation */
#define ORC_PURPOSE_MUT 3u  /* (instance, g, j/4)   -> word (j%4) per bit j      */
#define ORC_PURPOSE_STEP 4u /* (instance, g, t)     -> x: tie pick, y: tenure    */
#define ORC_PURPOSE_CROSS 5u /* (instance, g, j/4)  -> word (j%4): uniform crossover */

/* Variants (bit flags of orc_params.variant). */
#define ORC_VARIANT_UNIFORM_CROSSOVER 1 /* Combine: bit j from P2 iff its draw < 2^31 */
#define ORC_VARIANT_FIX_FIRST_SPIN 2    /* s_1 = +1 throughout (Sec. II.B) */
#define ORC_VARIANT_SKEW 4              /* odd N: skew-symmetric sequences only (Sec. II.C) */

#define ORC_REPLACE_RANDOM 0 /* Algorithm 1: replace a random individual */
#define ORC_REPLACE_WORST 1  /* variant: replace the highest-E member     */

#define ORC_STATUS_BUDGET 0  /* stopped by a generation or step budget */
#define ORC_STATUS_REACHED 1 /* E(best) <= target_E                    */

typedef struct orc_params {
    int32_t N;                /* sequence length, 3..256 */
    int32_t K;                /* population size, 1..1024 */
    uint32_t p_comb_u32;      /* crossover iff draw < p_comb_u32 */
    uint32_t p_mut_u32;       /* bit j flips iff draw < p_mut_u32 */
    int32_t replace_policy;   /* ORC_REPLACE_* */
    int32_t target_E;         /* stop when E(best) <= target_E; -1: none */
    int64_t max_generations;  /* -1: none */
    int64_t max_steps;        /* tabu steps per replica; -1: none */
    int32_t max_iter;         /* tabu length; -1: floor(N/2) + randInt(0, N)
                                 (skew variant: n = (N+1)/2 in place of N) */
    int32_t variant;          /* ORC_VARIANT_* flags, 0: Algorithm 1 as read */
} orc_params;

typedef struct orc_result {
    uint64_t seq[ORC_MAX_W]; /* best sequence found */
    int32_t E;               /* its energy */
    int32_t status;          /* ORC_STATUS_* */
    int64_t generations;     /* completed generations */
    int64_t steps;           /* tabu steps taken */
} orc_result;

/* One record per generation, for the oracle's own pin tests. */
typedef struct orc_genlog {
    int32_t g;
    int32_t crossover;   /* 1: tournament + one-point crossover, 0: sample */
    int32_t p1, p2;      /* parents (crossover) or the sampled member (p1) */
    int32_t cut;         /* crossover cut c: child = P1[0,c) | P2[c,N) */
    int32_t max_iter, min_tabu, max_tabu;
    int32_t replace;     /* population slot overwritten by the child */
    int32_t E_child;     /* energy returned by the tabu search */
    int32_t steps;       /* tabu steps taken in this generation */
    int32_t pad;
    uint64_t pre_mut[ORC_MAX_W];  /* child before mutation */
    uint64_t pre_tabu[ORC_MAX_W]; /* child after mutation */
    uint64_t post_tabu[ORC_MAX_W];/* child returned by the tabu search */
} orc_genlog;

/* Philox4x32-10: out = bijection(ctr) under key. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* orc_philox4x32_10 at B counters ctr[4i..4i+3] under key (seed lo, seed hi). */
void orc_philox4x32_batch(const uint32_t* ctr, int64_t B, uint64_t seed, uint32_t* out);
/* Philox4x64-10, same construction on 64-bit words (pinned against numpy). */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Eq. 1 and Eq. 2 on a packed sequence.  C (nullable) receives C_1..C_{N-1}.
 * Returns E, or -1 on bad arguments. */
int64_t orc_energy(const uint64_t* words, int32_t N, int32_t* C);

/* Energy of each of the N one-bit-flip neighbours of a packed sequence,
 * each recomputed from Eq. 2 (O(N^2) per neighbour). */
int32_t orc_neighbour_energies(const uint64_t* words, int32_t N, int32_t* E_out);

/* One tabu search (Algorithm 2) from `start`.  The draws come from
 * (seed, instance, generation g); max_iter < 0 selects the random rule.
 * incremental = 0 recomputes every neighbour energy from Eq. 2;
 * incremental = 1 keeps tableC / vectorC (Table I).
 * step_budget < 0: unlimited.  trace (nullable) receives {g, t, j, E} per
 * step.  Returns the number of steps taken, or -1 on bad arguments. */
int64_t orc_tabu_run(const uint64_t* start, int32_t N, uint64_t seed, uint32_t instance,
                     uint32_t g, int32_t max_iter, int64_t step_budget, int32_t incremental,
                     uint64_t* best_out, int32_t* bestE_out, int32_t* trace, int64_t trace_cap,
                     int64_t* trace_len);
/* The same with variant flags (ORC_VARIANT_FIX_FIRST_SPIN keeps s_1 fixed). */
int64_t orc_tabu_run_v(const uint64_t* start, int32_t N, uint64_t seed, uint32_t instance,
                       uint32_t g, int32_t max_iter, int64_t step_budget, int32_t incremental,
                       int32_t variant, uint64_t* best_out, int32_t* bestE_out, int32_t* trace,
                       int64_t trace_cap, int64_t* trace_len);

/* Algorithm 1 for one replica.  trace (nullable): {g, t, j, E} per tabu
 * step and {g, 0, replace, E_child} at the end of each generation.
 * genlog (nullable): one orc_genlog per generation.  Returns 0 or -1. */
int32_t orc_mts_run(const orc_params* P, uint64_t seed, uint32_t instance, int32_t incremental,
                    orc_result* res, int32_t* trace, int64_t trace_cap, int64_t* trace_len,
                    orc_genlog* genlog, int64_t genlog_cap, int64_t* genlog_len);

/* `replicas` independent replicas (instances first_instance + r), the
 * incremental form, spread over `threads` POSIX threads. */
int32_t orc_mts_run_many(const orc_params* P, uint64_t seed, uint32_t first_instance,
                         int32_t replicas, int32_t threads, orc_result* res);

/* Exhaustive minimum of E over all 2^N sequences (N <= 32).  Returns E_min,
 * the number of minimising sequences and the first one found. */
int32_t orc_bruteforce(int32_t N, int32_t* E_min, int64_t* n_min, uint64_t* argmin);

/* orc_bruteforce split over `threads` POSIX threads, for 8 <= N <= 40
 * (no argmin); *n_min counts all minimisers (complements included). */
int32_t orc_bruteforce_mt(int32_t N, int32_t threads, int32_t* E_min, int64_t* n_min);

/* Exhaustive minimum of E over the 2^((N+1)/2) skew-symmetric sequences of
 * odd length N <= 45 (Sec. II.C); *n_min = number of minimisers. */
int32_t orc_bruteforce_skew(int32_t N, int32_t* E_min, int64_t* n_min);

/* Appendix A: n_non-skew (Eq. 5) of an odd-length sequence, and d(S)
 * under the reading documented in the implementation. */
int32_t orc_non_skew_pairs(const uint64_t* words, int32_t N);
int32_t orc_skew_deviation(const uint64_t* words, int32_t N);

#ifdef __cplusplus
}
#endif
#endif
