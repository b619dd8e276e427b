// replica.cuh -- one warp runs one Memetic-Tabu replica (Algorithm 1 /
// Algorithm 3): initial population, the generation step (selection,
// crossover or sampling, mutation, tabu search, best update, replacement)
// and the stop test.  The population (K packed sequences and their
// energies) lives in the warp's slice of shared memory; everything else in
// registers.  The functions are split at generation boundaries so a replica
// can also be suspended and resumed there (the state between generations
// is the population, the best sequence and the counters).
//
// SKEW (compile time; odd N): every sequence is skew-symmetric (Sec. II.C).
// Members and children are completed from their free half b_0..b_c, the
// cut is randInt(1, n-1) with n = c + 1, mutation acts on the free half,
// maxIter = floor(n/2) + randInt(0, n), and the tabu search moves pairs.
#pragma once

#include "tabu_core.cuh"
#include "tabu_skew.cuh"

namespace lgpu {

// Parameters of one replica (an MTS instance under one Philox stream).
struct ReplicaCfg {
    int32_t N, K;
    uint32_t p_comb_u32, p_mut_u32;
    int32_t replace_policy, target_E;
    int64_t max_generations, max_steps;
    int32_t max_iter;
    int32_t variant;  // LABS_VARIANT_* flags
    uint32_t inst;
    uint2 key;
};

// Bit j of `mask` is set iff word j%4 of Philox(inst, g, j/4, purpose) < thr
// (j < N): one Philox block per four bits, nibbles OR-reduced over the warp.
template <int NW>
__device__ __forceinline__ void draw_bit_mask(const ReplicaCfg& a, uint32_t g, uint32_t purpose,
                                              uint32_t thr, int lane, uint32_t (&mask)[NW]) {
#pragma unroll
    for (int w = 0; w < NW; ++w) mask[w] = 0u;
    const int nd = (a.N + 3) / 4;
    for (int base = 0; base < nd; base += 32) {
        const int cidx = base + lane;
        uint32_t nib = 0;
        if (cidx < nd) {
            const uint4 d = draw4(a.key, a.inst, g, static_cast<uint32_t>(cidx), purpose);
            nib = (d.x < thr ? 1u : 0u) | (d.y < thr ? 2u : 0u) | (d.z < thr ? 4u : 0u) |
                  (d.w < thr ? 8u : 0u);
        }
        const int word_of = cidx >> 3;  // 8 nibbles per 32-bit word
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t part = (word_of == w) ? (nib << (4 * (cidx & 7))) : 0u;
            mask[w] |= __reduce_or_sync(kFull, part) & word_lowmask(w, a.N);
        }
    }
}

template <int NW>
struct ReplicaState {
    uint32_t best[NW];
    int32_t E_best;
    int32_t status;
    int64_t g, steps;
};

template <int NW>
__device__ __forceinline__ void load_seq(const uint32_t* __restrict__ src, uint32_t (&v)[NW]) {
#pragma unroll
    for (int w = 0; w < NW; ++w) v[w] = src[w];
}

// Lane w < NW writes word w of a warp-uniform sequence.
template <int NW>
__device__ __forceinline__ void store_seq(uint32_t* __restrict__ dst, const uint32_t (&v)[NW], int lane) {
    if (lane < NW) {
        uint32_t x = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) x = (lane == w) ? v[w] : x;
        dst[lane] = x;
    }
}

// Binary tournament: the lower energy wins, the lower index on ties.
__device__ __forceinline__ int tournament(const int32_t* __restrict__ popE, int a, int b) {
    const int32_t ea = popE[a], eb = popE[b];
    if (ea < eb) return a;
    if (eb < ea) return b;
    return a < b ? a : b;
}

// population <- K random sequences (word w of member p from Philox
// (inst, p, w/2, INIT)); bestSeq <- the lowest energy, lowest index on ties.
template <int NW, bool SKEW = false>
__device__ void replica_init(const ReplicaCfg& a, uint32_t* __restrict__ pop,
                             int32_t* __restrict__ popE, ReplicaState<NW>& st, int lane) {
    const int N = a.N, K = a.K;
    if constexpr (NW & 1) {  // the last 64-bit word keeps only its low half
        constexpr int W64 = (NW + 1) / 2;
        for (int idx = lane; idx < K * W64; idx += 32) {
            const int p = idx / W64, w64 = idx % W64;
            const uint4 d = draw4(a.key, a.inst, static_cast<uint32_t>(p), static_cast<uint32_t>(w64), kPurposeInit);
            pop[p * NW + 2 * w64] = d.x & word_lowmask(2 * w64, N);
            if (2 * w64 + 1 < NW) pop[p * NW + 2 * w64 + 1] = d.y & word_lowmask(2 * w64 + 1, N);
        }
    } else {
        for (int idx = lane; idx < K * (NW / 2); idx += 32) {
            const int p = idx / (NW / 2), w64 = idx % (NW / 2);
            const uint4 d = draw4(a.key, a.inst, static_cast<uint32_t>(p), static_cast<uint32_t>(w64), kPurposeInit);
            pop[p * NW + 2 * w64] = d.x & word_lowmask(2 * w64, N);
            pop[p * NW + 2 * w64 + 1] = d.y & word_lowmask(2 * w64 + 1, N);
        }
    }
    __syncwarp();
    if constexpr (SKEW) {
        for (int p = lane; p < K; p += 32) {
            uint32_t B[NW];
            load_seq<NW>(pop + p * NW, B);
            skew_complete<NW>(B, N);
#pragma unroll
            for (int w = 0; w < NW; ++w) pop[p * NW + w] = B[w];
        }
        __syncwarp();
    }
    if (a.variant & LABS_VARIANT_FIX_FIRST_SPIN) {  // complement members with s_1 = -1 (E unchanged)
        for (int p = lane; p < K; p += 32)
            if ((pop[p * NW] & 1u) == 0u)
#pragma unroll
                for (int w = 0; w < NW; ++w) pop[p * NW + w] ^= word_lowmask(w, N);
        __syncwarp();
    }
    int32_t lbestE = INT_MAX;
    int lbest = INT_MAX;
    for (int p = lane; p < K; p += 32) {
        uint32_t B[NW];
        load_seq<NW>(pop + p * NW, B);
        const int32_t e = thread_energy<NW>(B, N);
        popE[p] = e;
        if (e < lbestE) {
            lbestE = e;
            lbest = p;
        }
    }
    __syncwarp();
    st.E_best = __reduce_min_sync(kFull, lbestE);
    const int best0 = __reduce_min_sync(kFull, lbestE == st.E_best ? lbest : INT_MAX);
    load_seq<NW>(pop + best0 * NW, st.best);
    st.status = LABS_RUN_BUDGET;
    st.g = 0;
    st.steps = 0;
}

// The while-condition of Algorithm 1 plus the budgets and the GLF of
// Algorithm 3.  True if the replica stops before generation st.g.
template <int NW>
__device__ __forceinline__ bool replica_should_stop(const ReplicaCfg& a, ReplicaState<NW>& st,
                                                    const uint32_t* glf) {
    if (st.status == LABS_RUN_SYNC_LOST) return true;
    if (a.target_E >= 0 && st.E_best <= a.target_E) {
        st.status = LABS_RUN_REACHED;
        return true;
    }
    if (a.max_generations >= 0 && st.g >= a.max_generations) return true;
    if (a.max_steps >= 0 && st.steps >= a.max_steps) return true;
    if (glf != nullptr) {
        const uint32_t f = __shfl_sync(kFull, *reinterpret_cast<const volatile uint32_t*>(glf), 0);
        if (f != 0u) {
            st.status = LABS_RUN_STOPPED;
            return true;
        }
    }
    return false;
}

// One generation g = st.g.  Returns the tabu steps it took.
// WPS = 2: this warp is half HALF of a replica on two warps (tabu_search);
// it holds its own copy of the population and takes the same decisions as
// its partner, with which it meets through `link` inside the tabu search.
// The global termination flag is not supported there (glf must be null: the
// two warps could read it at different times).
template <int NW, bool TRACE = false, bool SKEW = false, int WPS = 1, int HALF = 0, bool PERK = false>
__device__ int64_t replica_generation(const ReplicaCfg& a, ReplicaState<NW>& st,
                                      uint32_t* __restrict__ pop, int32_t* __restrict__ popE,
                                      int32_t* __restrict__ Cs, int4* __restrict__ trace,
                                      int64_t trace_cap, int64_t& trace_len, uint32_t* glf,
                                      int lane, PairLink* link = nullptr, uint32_t* xseq = nullptr) {
    static_assert(WPS == 1 || (!SKEW && !TRACE), "two warps per replica: unrestricted, untraced");
    const int N = a.N, K = a.K;
    const uint32_t gg = static_cast<uint32_t>(st.g);
    const uint32_t p_mut = a.p_mut_u32;
    // generation draws: lane 0 -> (g,0), lane 1 -> (g,1), lane 2 -> (g,2)
    const uint4 gd = draw4(a.key, a.inst, gg, static_cast<uint32_t>(lane < 3 ? lane : 0), kPurposeGen);
    const uint32_t coin = __shfl_sync(kFull, gd.x, 0);
    const uint32_t ua = __shfl_sync(kFull, gd.y, 0), ub = __shfl_sync(kFull, gd.z, 0);
    const uint32_t uc = __shfl_sync(kFull, gd.w, 0), ud = __shfl_sync(kFull, gd.x, 1);
    const uint32_t ucut = __shfl_sync(kFull, gd.y, 1), usamp = __shfl_sync(kFull, gd.z, 1);
    const uint32_t uiter = __shfl_sync(kFull, gd.w, 1), urep = __shfl_sync(kFull, gd.x, 2);

    uint32_t child[NW];
    if (coin < a.p_comb_u32) {
        const int p1 = tournament(popE, rand_int(0, K - 1, ua), rand_int(0, K - 1, ub));
        const int p2 = tournament(popE, rand_int(0, K - 1, uc), rand_int(0, K - 1, ud));
        if (a.variant & LABS_VARIANT_UNIFORM_CROSSOVER) {
            uint32_t m2[NW];  // bits taken from P2
            draw_bit_mask<NW>(a, gg, kPurposeCross, 0x80000000u, lane, m2);
#pragma unroll
            for (int w = 0; w < NW; ++w) child[w] = (pop[p1 * NW + w] & ~m2[w]) | (pop[p2 * NW + w] & m2[w]);
        } else {
            const int cut = rand_int(1, (SKEW ? (N + 1) / 2 : N) - 1, ucut);
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t lm = word_lowmask(w, cut);
                child[w] = (pop[p1 * NW + w] & lm) | (pop[p2 * NW + w] & ~lm);
            }
        }
    } else {
        load_seq<NW>(pop + rand_int(0, K - 1, usamp) * NW, child);
    }
    // Mutate: bit j flips iff word j%4 of (inst, g, j/4, MUT) < p_mut.
    {
        uint32_t mm[NW];
        draw_bit_mask<NW>(a, gg, kPurposeMut, p_mut, lane, mm);
        if (a.variant & LABS_VARIANT_FIX_FIRST_SPIN) mm[0] &= ~1u;
#pragma unroll
        for (int w = 0; w < NW; ++w) child[w] ^= mm[w];
        // (bits above the free half are rewritten by the completion)
        if constexpr (SKEW) skew_complete<NW>(child, N);
    }
    // child <- Tabu-Search(child)
    const int nmov = SKEW ? (N + 1) / 2 : N;  // tabu moves
    const int max_iter = a.max_iter >= 0 ? a.max_iter : nmov / 2 + rand_int(0, nmov, uiter);
    const int64_t budget = a.max_steps >= 0 ? a.max_steps - st.steps : -1;
    TabuOut to;
    if constexpr (SKEW) {
        to = (a.variant & LABS_VARIANT_FIX_FIRST_SPIN)
                 ? tabu_search_skew<NW, TRACE, true>(child, N, a.key, a.inst, gg, max_iter, budget, Cs,
                                                     trace, trace_cap, trace_len, lane)
                 : tabu_search_skew<NW, TRACE, false>(child, N, a.key, a.inst, gg, max_iter, budget, Cs,
                                                      trace, trace_cap, trace_len, lane);
    } else {
        to = (a.variant & LABS_VARIANT_FIX_FIRST_SPIN)
                 ? tabu_search<NW, TRACE, true, WPS, HALF, PERK>(child, N, a.key, a.inst, gg, max_iter, budget,
                                                                 Cs, trace, trace_cap, trace_len, lane, link, xseq)
                 : tabu_search<NW, TRACE, false, WPS, HALF, PERK>(child, N, a.key, a.inst, gg, max_iter, budget,
                                                                  Cs, trace, trace_cap, trace_len, lane, link, xseq);
    }
    if (to.fault) {  // the pair lost step: stop the replica, report it
        st.status = LABS_RUN_SYNC_LOST;
        return to.steps;
    }
    st.steps += to.steps;
    if (to.E_best < st.E_best) {
        st.E_best = to.E_best;
#pragma unroll
        for (int w = 0; w < NW; ++w) st.best[w] = child[w];
    }
    // replace a member of the population by the child
    int slot;
    if (a.replace_policy == LABS_REPLACE_RANDOM) {
        slot = rand_int(0, K - 1, urep);
    } else {
        int32_t lmax = INT_MIN;
        for (int p = lane; p < K; p += 32) lmax = max(lmax, popE[p]);
        const int32_t emax = __reduce_max_sync(kFull, lmax);
        int lidx = INT_MAX;
        for (int p = lane; p < K; p += 32)
            if (popE[p] == emax) {
                lidx = p;
                break;
            }
        slot = __reduce_min_sync(kFull, lidx);
    }
    __syncwarp();
    store_seq<NW>(pop + slot * NW, child, lane);
    if (lane == 0) popE[slot] = to.E_best;
    __syncwarp();
    if constexpr (TRACE) {
        if (trace_len < trace_cap) {
            if (lane == 0) trace[trace_len] = make_int4(static_cast<int>(st.g), 0, slot, to.E_best);
            ++trace_len;
        }
    }
    ++st.g;
    if (glf != nullptr && a.target_E >= 0 && to.E_best <= a.target_E && lane == 0) atomicExch(glf, 1u);
    return to.steps;
}

template <int NW>
__device__ __forceinline__ void replica_store_result(const ReplicaState<NW>& st, int64_t trace_len,
                                                     labs_device_result* out, int lane) {
    if (lane < 2 * LABS_MAX_W) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) v = (lane == w) ? st.best[w] : v;
        reinterpret_cast<uint32_t*>(out->seq)[lane] = v;
    }
    if (lane == 0) {
        out->E = st.E_best;
        out->status = st.status;
        out->generations = st.g;
        out->steps = st.steps;
        out->trace_len = trace_len;
    }
}

// A whole replica from scratch to its stop condition.  WPS = 2: both warps
// run it (see replica_generation); the lower half stores the result.
template <int NW, bool TRACE = false, bool SKEW = false, int WPS = 1, int HALF = 0, bool PERK = false>
__device__ __forceinline__ void replica_run(const ReplicaCfg& a, uint32_t* pop, int32_t* popE,
                                            int32_t* Cs, int4* trace, int64_t trace_cap,
                                            uint32_t* glf, labs_device_result* out, int lane,
                                            PairLink* link = nullptr, uint32_t* xseq = nullptr) {
    ReplicaState<NW> st;
    int64_t trace_len = 0;
    replica_init<NW, SKEW>(a, pop, popE, st, lane);
    while (!replica_should_stop<NW>(a, st, glf))
        replica_generation<NW, TRACE, SKEW, WPS, HALF, PERK>(a, st, pop, popE, Cs, trace, trace_cap, trace_len,
                                                             glf, lane, link, xseq);
    if (HALF == 0) replica_store_result<NW>(st, trace_len, out, lane);
}

}  // namespace lgpu
