/*
 * labs.h -- C ABI of the GB300 (sm_103a) memetic tabu search (MTS) solver for
 * Low Autocorrelation Binary Sequences (LABS), after arXiv 2504.00987.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Sequence format.  A length-N sequence S = s_1 .. s_N, s_i in {-1, +1}
 *   (Sec. II), is packed LSB-first into W = ceil(N/64) uint64 words: s_{i+1}
 *   is bit (i % 64) of word (i / 64), bit 1 <-> +1.  Bits at positions >= N
 *   are ignored by every call (read as zero) and written as zero.
 *   A batch of B sequences is B * W contiguous words (row-major, 8-byte
 *   aligned).  3 <= N <= LABS_MAX_N.
 * Energy (Eq. 1, Eq. 2): C_k = sum_{i=1}^{N-k} s_i s_{i+k}, E = sum_k C_k^2,
 *   exact in int32.  Merit factor (Eq. 3): F = N^2 / (2 E).
 * Memory.  The caller owns every buffer.  "d_" pointers are device memory
 *   (cudaMalloc, cudaMallocAsync or a framework's allocator); "h_" pointers
 *   are host memory.  A pointer of the wrong kind is rejected with
 *   LABS_EINVAL before any launch.
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *   Calls are asynchronous on that stream unless documented as blocking.
 * Errors.  Every entry point returns a LABS_* status.  A non-OK status
 *   leaves a message for labs_last_error() (thread-local).  The library
 *   never aborts, never exits and prints nothing.
 * Randomness.  Every random decision is one 32-bit word of Philox4x32-10
 *   (Salmon et al., SC'11) under key (seed low 32 bits, seed high 32 bits)
 *   at counter (instance, a, b, purpose); see labs_params for the draws.
 *   Results are a pure function of (parameters, seed, instance): the same
 *   instance gives the same trajectory alone, in a batch or after resume.
 */
#ifndef LABS_H
#define LABS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LABS_OK 0
#define LABS_EINVAL 1       /* bad argument (size, pointer kind, alignment, tail bits) */
#define LABS_ENOMEM 2       /* a device or host allocation failed */
#define LABS_ECUDA 3        /* a CUDA runtime call failed; see labs_last_error() */
#define LABS_ETIMEOUT 4     /* a bounded device wait ran out */
#define LABS_EBUSY 5        /* no free slot or queue entry */
#define LABS_ENOTREADY 6    /* result not available yet */
#define LABS_ECANCELED 7    /* request was cancelled */
#define LABS_ENOTFOUND 8    /* unknown ticket */

#define LABS_MAX_N 256
#define LABS_MAX_W 4
#define LABS_MAX_K 1024

/* Replacement rule of the population loop. */
#define LABS_REPLACE_RANDOM 0 /* Algorithm 1: a uniformly drawn member (default) */
#define LABS_REPLACE_WORST 1  /* variant: the highest-E member, lowest index on ties */

/* Variants of the population loop (bit flags; 0 = Algorithm 1 as read). */
#define LABS_VARIANT_UNIFORM_CROSSOVER 1 /* Combine: child bit j from P2 iff draw (i, g, j/4, 5)
                                            word j%4 < 2^31 (instead of one cut) */
#define LABS_VARIANT_FIX_FIRST_SPIN 2    /* s_1 = +1 throughout (Sec. II.B symmetry break):
                                            initial members with s_1 = -1 are complemented,
                                            s_1 is never mutated nor flipped by the tabu search */
#define LABS_VARIANT_SKEW 4              /* odd N only: the search runs over skew-symmetric
                                            sequences s_{n+i} = (-1)^i s_{n-i}, N = 2n-1
                                            (Sec. II.C).  Sequences are completed from their
                                            free half s_1..s_n; the crossover cut is
                                            randInt(1, n-1); mutation (default rate 1/n) acts
                                            on the free half; a tabu move flips a free spin
                                            and its partner; maxIter = floor(n/2) +
                                            randInt(0, n).  labs_mts_launch, labs_mts_run,
                                            labs_mts_run_static and labs_tabu_run (which
                                            completes each start from its free half) take
                                            it; batches and the service refuse it. */

/* Why a replica stopped. */
#define LABS_RUN_BUDGET 0  /* generation or step budget used up */
#define LABS_RUN_REACHED 1 /* E(best) <= target_E */
#define LABS_RUN_STOPPED 2 /* another replica of the same run reached target_E (GLF) */
#define LABS_RUN_BADSTATE 3 /* labs_mts_resume: the state record belongs to another run */
#define LABS_RUN_SYNC_LOST 4 /* a replica mapped on two warps (labs_mapping.warps_per_seq
                                = 2) stopped because one warp waited for the other
                                beyond a bounded number of polls; its record is not a
                                result (never expected; reported instead of waiting) */

typedef void* labs_stream_t; /* a cudaStream_t */

/*
 * Parameters of Memetic-Tabu (Algorithm 1 / Algorithm 3 of the paper).
 *
 * Draws per replica (instance i), generation g, as Philox words (x, y, z, w):
 *   population member p, word w .. (i, p, w, 1): x = low half, y = high half
 *   (i, g, 0, 2) ...................... x coin, y/z/w tournament entrants a, b, c
 *   (i, g, 1, 2) ...................... x entrant d, y crossover cut, z sampled
 *                                       member, w tabu length
 *   (i, g, 2, 2) ...................... x replaced member
 *   (i, g, j/4, 3) .................... word j%4: mutation draw of bit j
 *   (i, g, t, 4) ...................... x tie pick, y tenure of tabu step t
 *   (i, g, j/4, 5) .................... word j%4: uniform-crossover draw of bit j
 *                                       (LABS_VARIANT_UNIFORM_CROSSOVER only)
 * randInt(a, b) = a + floor(u * (b - a + 1) / 2^32).
 * The generation step: with probability p_comb two binary tournaments
 * (lower E wins, lower index on ties) pick P1, P2 and the child is
 * P1 bits [0, c) | P2 bits [c, N), c = randInt(1, N-1); otherwise the child
 * is a copy of member randInt(0, K-1).  Every bit of the child then flips
 * iff its draw < p_mut_u32.  The tabu search (Algorithm 2) runs for
 * maxIter = floor(N/2) + randInt(0, N) steps (or `max_iter`), with tenure
 * randInt(floor(maxIter/10), floor(12 maxIter/100)); a bit is admissible iff
 * its tabu has expired or flipping it beats the search's best (aspiration);
 * ties for the admissible minimum are broken by the tie draw in ascending
 * bit order.  A search with no admissible move stops at that step: this
 * cannot happen under the default maxIter (its tenure bound stays below N),
 * but a user max_iter of about 8N or more lets floor(12 maxIter/100) reach
 * N, and then every bit can be tabu with none aspirating.  The child
 * replaces a member (replace_policy) and the replica's best on a strictly
 * lower energy.
 */
typedef struct labs_params {
    int32_t N;               /* 3 .. LABS_MAX_N */
    int32_t K;               /* population size, 1 .. LABS_MAX_K (paper: 100) */
    uint32_t p_comb_u32;     /* crossover iff coin < p_comb_u32; 0.9 -> 3865470566 */
    uint32_t p_mut_u32;      /* per-bit flip iff draw < p_mut_u32; 0 -> floor(2^32/N) */
    int32_t replace_policy;  /* LABS_REPLACE_* */
    int32_t target_E;        /* stop a replica once E(best) <= target_E; -1: no target */
    int64_t max_generations; /* per replica; -1: unlimited */
    int64_t max_steps;       /* tabu steps per replica; -1: unlimited.  A budget can end a
                                tabu search early; that generation still completes. */
    int32_t max_iter;        /* tabu length; -1: floor(N/2) + randInt(0, N) */
    int32_t glf;             /* nonzero: a replica reaching target_E stops every replica of
                                the run at its next generation boundary (Algorithm 3 GLF) */
    int32_t* d_trace;        /* nullable, device: per replica trace_cap records {g, t, j, E}
                                (t >= 1: tabu step; t == 0: end of generation g with
                                j = replaced member, E = E(child)) */
    int64_t trace_cap;       /* records per replica in d_trace */
    int32_t variant;         /* LABS_VARIANT_* flags */
    int32_t pad;
} labs_params;

/* Per-replica result in device memory (64 bytes). */
typedef struct labs_device_result {
    uint64_t seq[LABS_MAX_W]; /* best sequence of the replica */
    int32_t E;                /* its energy */
    int32_t status;           /* LABS_RUN_* */
    int64_t generations;      /* completed generations */
    int64_t steps;            /* tabu steps taken (flip evaluations = steps * N) */
    int64_t trace_len;        /* records written to the replica's trace */
} labs_device_result;

/* Per-replica result in host memory. */
typedef struct labs_result {
    uint64_t seq[LABS_MAX_W];
    int32_t E;
    int32_t N;
    double F;                 /* merit factor N^2 / (2E), Eq. 3 */
    int64_t generations;
    int64_t steps;
    int64_t flip_evals;       /* steps * N */
    int64_t trace_len;
    uint64_t instance;
    double seconds;           /* wall time of the whole call */
    int32_t status;
    int32_t pad;
} labs_result;

/* Options of a standalone tabu search batch. */
typedef struct labs_tabu_opts {
    int32_t max_iter;        /* steps; -1: floor(N/2) + randInt(0, N) from draw (i, g, 1, 2).w */
    uint32_t generation;     /* g of the draws (a search inside MTS uses its generation) */
    uint64_t first_instance; /* sequence b uses instance first_instance + b */
    int64_t trace_cap;       /* records {g, t, j, E} per sequence in d_trace */
    int32_t variant;         /* LABS_VARIANT_FIX_FIRST_SPIN: bit 0 is never flipped */
    int32_t pad;
} labs_tabu_opts;

/*
 * One Memetic-Tabu instance of a batch (64 bytes, host or device).  The
 * fields mean what the labs_params fields of the same name mean; the run
 * of an instance is a pure function of this record, so it is the same
 * alone, in any batch, under any mapping.  p_mut_u32 == 0 selects
 * floor(2^32 / N).  `instance` (< 2^32) is counter word 0 of its draws.
 */
typedef struct labs_instance {
    int32_t N, K;
    uint32_t p_comb_u32, p_mut_u32;
    int32_t replace_policy, target_E;
    int64_t max_generations, max_steps;
    int32_t max_iter, variant;
    uint64_t seed;
    uint64_t instance;
} labs_instance;

#define LABS_ORDER_LPT 0   /* queue longest instance first (pair-term budget) */
#define LABS_ORDER_GIVEN 1 /* queue in the given order */

/* How a batch is mapped on the GPU. */
typedef struct labs_mapping {
    int32_t warps_per_block; /* warps per CTA: 1, 2, 4 or 8 */
    int32_t blocks_per_sm;   /* resident CTAs per SM of the persistent grid, >= 1 */
    int32_t order;           /* LABS_ORDER_* */
    int32_t warps_per_seq;   /* warps per replica: 1 (or 0), or 2 (warps_per_block 2, 4
                                or 8): the two warps of a replica split every tabu
                                step's neighbours and meet once per step in shared
                                memory, which halves a step's scoring but repeats the
                                move's bookkeeping in both warps (on GB300 slower than
                                one warp for N <= 160; the autotuner times both); a
                                lost step (a bounded wait that runs out) stops the
                                replica with LABS_RUN_SYNC_LOST */
} labs_mapping;

typedef struct labs_batch labs_batch; /* opaque */

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* labs_last_error(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int32_t labs_version(void);

/*
 * labs_energy_batch -- Eq. 1 and Eq. 2 for B sequences.
 *   d_seqs  device, B * W uint64, packed sequences (read only).
 *   N       3 .. LABS_MAX_N.   B >= 0 (B == 0 is a no-op).
 *   d_E     device, B int32: E of each sequence.
 *   d_C     device, nullable, B * (N-1) int32: C_1 .. C_{N-1} of each sequence.
 * Asynchronous on `stream`.
 */
int32_t labs_energy_batch(const uint64_t* d_seqs, int32_t N, int64_t B, int32_t* d_E,
                          int32_t* d_C, labs_stream_t stream);

/*
 * labs_tabu_run -- B independent tabu searches (Algorithm 2 / Algorithm 4),
 * one from each start sequence, each scoring all N one-bit-flip neighbours
 * per step with incremental correlations (Sec. III.C).
 *   d_start  device, B * W uint64 start sequences.
 *   seed     Philox key; sequence b uses instance opts->first_instance + b
 *            and generation opts->generation.
 *   d_best   device, B * W uint64: best sequence visited (bestSeqTS).
 *   d_bestE  device, B int32: its energy.
 *   d_steps  device, nullable, B int64: steps taken.
 *   d_trace  device, nullable, B * trace_cap * 4 int32 records {g, t, j, E}.
 * Asynchronous on `stream`.
 */
int32_t labs_tabu_run(const uint64_t* d_start, int32_t N, int64_t B, uint64_t seed,
                      const labs_tabu_opts* opts, uint64_t* d_best, int32_t* d_bestE,
                      int64_t* d_steps, int32_t* d_trace, labs_stream_t stream);

/*
 * labs_mts_launch -- `replicas` independent Memetic-Tabu replicas (Algorithm
 * 3: one population per replica, all on the device), instances
 * first_instance .. first_instance + replicas - 1.  Asynchronous.
 *   d_out   device, replicas labs_device_result.
 *   d_glf   device, nullable, one uint32 global termination flag shared by
 *           the replicas of this launch; the caller zeroes it.  Required
 *           when P->glf is nonzero.
 * Fails with LABS_EINVAL if no target, generation or step budget bounds the
 * run.
 */
int32_t labs_mts_launch(const labs_params* P, uint64_t seed, uint64_t first_instance,
                        int64_t replicas, labs_device_result* d_out, uint32_t* d_glf,
                        labs_stream_t stream);

/*
 * labs_mts_run -- labs_mts_launch plus the device scratch it needs (results,
 * GLF), the copy of the results to h_out[replicas] and the merit factors.
 * BLOCKING: returns once the results are in host memory.  Allocates and
 * frees its scratch with cudaMallocAsync/cudaFreeAsync on `stream`.
 */
int32_t labs_mts_run(const labs_params* P, uint64_t seed, uint64_t first_instance,
                     int64_t replicas, labs_result* h_out, labs_stream_t stream);

/*
 * labs_results_decode -- the host form of device result records (from
 * labs_mts_launch or labs_mts_resume, copied to host memory by the caller):
 * h_out[r] gets the record's sequence, E, status and counters, the merit
 * factor F = N^2 / (2E) of Eq. 3 (0 when E <= 0), flip_evals = steps * N,
 * instance = first_instance + r and seconds = 0.  E is copied with its
 * sign: a record refused by labs_mts_resume (LABS_RUN_BADSTATE) carries
 * E = -1.  Host memory only (h_in: n records, h_out: n results, both owned
 * by the caller); touches no GPU.  LABS_EINVAL for N outside 3..LABS_MAX_N,
 * n < 0, or a NULL buffer with n > 0.
 */
int32_t labs_results_decode(const labs_device_result* h_in, int64_t n, int32_t N,
                            uint64_t first_instance, labs_result* h_out);

/*
 * Checkpoint and resume.  Between two generations a replica's whole state
 * is its population, their energies, its best sequence and its generation
 * and step counters: every later draw is addressed by (instance,
 * generation, index), so nothing else is needed to continue it exactly.
 *
 * labs_mts_state_bytes -- bytes of one replica's state record for (N, K):
 *   an 80-byte header, then the population and its energies, padded to 16.
 * labs_mts_resume -- labs_mts_launch with a state record per replica.
 *   d_state  device, replicas * labs_mts_state_bytes(N, K) bytes, 16-byte
 *            aligned, owned by the caller (copy it to the host to keep a
 *            checkpoint, and back to continue).
 *   resume   0: every replica starts from its initial population;
 *            nonzero: every replica continues from its record, which must
 *            have been written by this function for the same N, K, variant,
 *            seed and instance (otherwise the record is left as it is and the
 *            replica reports LABS_RUN_BADSTATE without running).
 *   Budgets and the target are totals over the whole run (max_generations
 *   counts from generation 0).  Each replica runs until P's stop condition,
 *   then writes its result to d_out and its record to d_state.  A run
 *   stopped by a generation budget and continued with a larger one equals
 *   the run made straight to the larger budget, bit for bit; a step budget
 *   may end a generation's tabu search early, and the continued run keeps
 *   that shortened generation.  Traces are not recorded (P->d_trace must be
 *   NULL); d_glf as in labs_mts_launch.  Asynchronous on `stream`.
 */
int64_t labs_mts_state_bytes(int32_t N, int32_t K);
int32_t labs_mts_resume(const labs_params* P, uint64_t seed, uint64_t first_instance,
                        int64_t replicas, void* d_state, int32_t resume, labs_device_result* d_out,
                        uint32_t* d_glf, labs_stream_t stream);

/*
 * labs_skew_deviation_batch -- deviation from skew-symmetry d(S) (Appendix A,
 * Eqs. 5-9) of B sequences.  n_non-skew (Eq. 5) counts, for an odd length
 * L = 2n - 1, the i in 1..n-1 with s_{n+i} != (-1)^i s_{n-i}.  d(S) is its
 * minimum over the rotations Rot(S; r) for odd N, and over the rotations
 * followed by one deletion Del(Rot(S; r); i) for even N (the reading that
 * reproduces the d column of Table II).  N >= 3 (even N >= 4).
 *   d_seqs  device, B * W uint64 packed sequences.
 *   d_d     device, B int32 results.
 * Asynchronous on `stream`.
 */
int32_t labs_skew_deviation_batch(const uint64_t* d_seqs, int32_t N, int64_t B, int32_t* d_d,
                                  labs_stream_t stream);

/*
 * labs_philox_batch -- the four words of Philox4x32-10 (Salmon et al., SC'11)
 * under key (seed low 32 bits, seed high 32 bits) at each of B counters,
 * i.e. the draws of the randomness contract above, computed by the device
 * function every kernel draws with (for reproducing a decision, or for
 * checking the generator).
 *   d_ctr  device, B x 4 uint32 counters (instance, a, b, purpose), 16-byte aligned.
 *   d_out  device, B x 4 uint32 words (x, y, z, w), 16-byte aligned.
 * Asynchronous on `stream`.
 */
int32_t labs_philox_batch(uint64_t seed, const uint32_t* d_ctr, int64_t B, uint32_t* d_out,
                          labs_stream_t stream);

/*
 * Batched uneven instances: one persistent launch, captured once in a CUDA
 * graph, in which every replica unit (one warp, or a pair of warps with
 * warps_per_seq = 2) takes the next instance from a device queue and runs
 * it to its stop condition.  Every instance must be bounded by a
 * generation budget or a step budget (with max_iter != 0).
 *
 * labs_autotune      -- picks a mapping for these instances by timing the
 *                       candidate mappings (warps_per_seq x warps_per_block x
 *                       blocks_per_sm within occupancy) on a copy of the
 *                       batch with every budget divided by 8; caches the
 *                       choice per batch signature.  BLOCKING; uses `stream`.
 * labs_batch_create  -- validates and orders the instances (host h_inst[n]),
 *                       uploads them, allocates the results and captures the
 *                       launch in a CUDA graph.  mapping == NULL: autotune.
 *                       Allocates device memory (cudaMalloc); BLOCKING.
 * labs_batch_launch  -- replays the graph on `stream` (asynchronous).  May be
 *                       called again; each launch reruns every instance.
 * labs_batch_device_results -- the device array of n labs_device_result, in
 *                       the original instance order (owned by the batch).
 * labs_batch_results -- copies the results to h_out[n] (original order) and
 *                       fills the merit factors.  BLOCKING on `stream`.
 * labs_batch_get_mapping -- the mapping the batch runs with.
 * labs_batch_destroy -- frees everything; NULL is a no-op.
 * labs_mts_batch_run -- create + launch + results + destroy.  BLOCKING.
 */
int32_t labs_autotune(const labs_instance* h_inst, int64_t n, labs_stream_t stream,
                      labs_mapping* out);
int32_t labs_batch_create(const labs_instance* h_inst, int64_t n, const labs_mapping* mapping,
                          labs_stream_t stream, labs_batch** out);
int32_t labs_batch_launch(labs_batch* b, labs_stream_t stream);
int32_t labs_batch_device_results(const labs_batch* b, labs_device_result** d_out);
int32_t labs_batch_results(labs_batch* b, labs_result* h_out, labs_stream_t stream);
int32_t labs_batch_get_mapping(const labs_batch* b, labs_mapping* out);
int32_t labs_batch_destroy(labs_batch* b);
int32_t labs_mts_batch_run(const labs_instance* h_inst, int64_t n, const labs_mapping* mapping,
                           labs_result* h_out, labs_stream_t stream);

/*
 * Solve service: continuous batching of solve requests on one GPU.
 *
 * A server owns `max_slots` slots and a device arena for the populations.
 * A scheduler thread admits pending requests (FIFO) as slots and memory free
 * up -- a request is admitted when a slot is free, its word class (the
 * kernel's word count for its N) still fits in one resident wave of the
 * quantum kernels, by their shared memory and registers per SM, and the
 * arena has a free extent of its footprint -- and runs quanta: one bounded
 * launch per word class (each with that class's shared memory per warp, on
 * its own stream) in which every admitted request advances by whole
 * generations up to `quantum_steps` tabu steps, its population staying in
 * its arena extent between quanta.  Requests that arrive while a quantum
 * runs join at the next quantum.  A request's result is the same
 * alone, in any mix, under any quantum size (it is the labs_mts_launch run
 * of its instance).  Results carry the request's latency (submit -> result)
 * in labs_result.seconds.
 */
typedef struct labs_serve_opts {
    int32_t max_slots;          /* requests resident on the GPU at once (one warp each) */
    int32_t max_N;              /* largest N accepted, 3 .. LABS_MAX_N */
    int32_t max_K;              /* largest K accepted, 1 .. LABS_MAX_K */
    int32_t warps_per_block;    /* quantum kernel CTA size in warps: 1, 2, 4 or 8 */
    int64_t quantum_steps;      /* tabu steps per slot per quantum (rounded up to a generation) */
    int64_t queue_capacity;     /* pending requests; submit answers LABS_EBUSY beyond it */
    int64_t hbm_budget_bytes;   /* bytes of the device arena holding the resident
                                   populations; a request takes K (nw + 1) 4 bytes of it
                                   (nw = 2, 3, 4, 5, 6, 8 for N up to 64, 96, 128, 160,
                                   192, 256; padded to 16) while it runs, and waits in the
                                   queue while no free extent fits it.  0: max_slots
                                   requests of (max_N, max_K).  LABS_EINVAL if it holds no
                                   (max_N, max_K) request. */
    int64_t quantum_timeout_ms; /* longest wait for one quantum before the server fails with
                                   LABS_ETIMEOUT; 0: 60000 */
    int64_t quantum_us;         /* > 0: a slot also suspends at the first generation boundary
                                   after this many microseconds of the quantum (device clock;
                                   at least one generation per quantum), so slots of every N
                                   share a quantum evenly; 0: steps only */
    int32_t warps_per_request;  /* 0 or 1: one warp per request.  2: a quantum runs each
                                   request whose word count is even on two warps (they split
                                   every tabu step's neighbours) whenever all active requests
                                   fit in one resident wave that way, else on one.  Results
                                   do not depend on it.  On GB300, N <= 160, pairs measured
                                   slower than single warps (the per-step exchange and the
                                   duplicated move bookkeeping cost more than the halved
                                   scoring saves), hence the default. */
    int32_t pad;
} labs_serve_opts;

/* One solve request: an MTS instance; max_steps or max_generations must bound it. */
typedef labs_instance labs_request;

typedef struct labs_serve_stats {
    int64_t submitted, completed, canceled, quanta;
    int64_t running, pending;
    int64_t flip_evals;         /* tabu steps x N of every quantum so far */
    double gpu_seconds;         /* summed quantum durations */
    int32_t failed;             /* LABS_OK or the error that stopped the server */
    int32_t pad;
    /* requests the admission rules held back, each request counted once per
       rule: no free slot; its word class would not fit in one resident wave
       of the quantum kernels (shared memory and registers per SM, from the
       occupancy API; a request is always admitted when nothing runs); no free
       arena extent of its footprint */
    int64_t deferred_slots, deferred_smem, deferred_hbm;
    int64_t arena_bytes, arena_used_bytes;
    int64_t pair_quanta;        /* quanta that ran even-word-count requests on warp pairs */
} labs_serve_stats;

typedef struct labs_server labs_server; /* opaque */

/* Creates a server (allocates its arena and starts its scheduler thread) on
 * the current device; NULL on failure (see labs_last_error()). */
labs_server* labs_serve_create(const labs_serve_opts* opts);
/* Queues a request; *ticket identifies it.  LABS_EBUSY when the queue is full. */
int32_t labs_serve_submit(labs_server* s, const labs_request* req, uint64_t* ticket);
/* LABS_OK with the result (the ticket is then released), LABS_ENOTREADY,
 * LABS_ECANCELED (released), LABS_ENOTFOUND, or the server's failure code. */
int32_t labs_serve_poll(labs_server* s, uint64_t ticket, labs_result* out);
/* Cancels a pending or running request (it leaves the GPU at the next quantum). */
int32_t labs_serve_cancel(labs_server* s, uint64_t ticket);
int32_t labs_serve_stats_get(labs_server* s, labs_serve_stats* out);
/* Stops the scheduler, waits for the quantum in flight and frees everything. */
int32_t labs_serve_destroy(labs_server* s);

/*
 * labs_mts_run_static -- labs_mts_run without any memory allocation (no
 * counterpart in the paper; an interface for callers that cannot allocate).
 * Some callers may not allocate device memory at all: an application that
 * owns the GPU memory budget through its own pool, a latency-critical loop
 * that cannot afford cudaMalloc/cudaFree (which may synchronise the
 * device), or a process under a hard device-memory quota.  This call makes
 * no device or host allocation: its device scratch (one result record per
 * replica and the global termination flag) is a fixed array compiled into
 * the library, sized for LABS_STATIC_MAX_REPLICAS replicas (about 256 KiB),
 * which every GPU that loads the library holds until the process exits.
 *   - replicas > LABS_STATIC_MAX_REPLICAS is rejected with LABS_EINVAL.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress,
 *     a host-side query that allocates nothing) with the caller's device
 *     current, so the address stays right after cudaDeviceReset.  The first
 *     call on a device (and the first after a reset) loads the library's
 *     device code, which places the array: make it before any stream
 *     capture.
 *   - All calls on a device share the one array, which keeps the last
 *     call's contents (each call clears the flag and overwrites the records
 *     it reads): calls whose GPU work overlaps -- on different streams or
 *     from different threads -- race and must be serialised by the caller.
 *   - Arguments, results and errors are those of labs_mts_run.  BLOCKING.
 */
#define LABS_STATIC_MAX_REPLICAS 4096
int32_t labs_mts_run_static(const labs_params* P, uint64_t seed, uint64_t first_instance,
                            int64_t replicas, labs_result* h_out, labs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* LABS_H */
