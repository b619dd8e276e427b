// mts_kernels.cuh -- Memetic-Tabu (Algorithm 1 / Algorithm 3) and batched
// tabu search (Algorithm 2 / Algorithm 4) kernels, templated on the word
// count, tracing and the skew-symmetric restriction (Sec. II.C).  One warp
// runs one replica: its population lives in the warp's slice of shared
// memory (K packed sequences and their energies), its pivot, correlations
// and tabu list in registers.  Replicas never synchronise with each other;
// the only cross-replica state is the optional global termination flag.
// mts.cu instantiates the unrestricted kernels, mts_skew.cu the restricted
// ones and mts_resume.cu the resumable ones (both kinds), so each
// translation unit compiles one family.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"
#include "replica.cuh"

namespace lgpu {

template <int NW, bool TRACE, bool SKEW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) mts_kernel(const MtsArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + warp;
    if (r >= a.replicas) return;

    uint32_t* pop = reinterpret_cast<uint32_t*>(smem + static_cast<size_t>(warp) * a.smem_per_warp);
    int32_t* popE = reinterpret_cast<int32_t*>(pop + a.K * NW);
    int32_t* Cs = popE + a.K;
    ReplicaCfg cfg;
    cfg.N = a.N;
    cfg.K = a.K;
    cfg.p_comb_u32 = a.p_comb_u32;
    cfg.p_mut_u32 = a.p_mut_u32;
    cfg.replace_policy = a.replace_policy;
    cfg.target_E = a.target_E;
    cfg.max_generations = a.max_generations;
    cfg.max_steps = a.max_steps;
    cfg.max_iter = a.max_iter;
    cfg.variant = a.variant;
    cfg.inst = static_cast<uint32_t>(a.first_instance + static_cast<uint64_t>(r));
    cfg.key = philox_key(a.seed);
    int4* trace = a.d_trace ? a.d_trace + r * a.trace_cap : nullptr;
    replica_run<NW, TRACE, SKEW>(cfg, pop, popE, Cs, trace, a.trace_cap, a.d_glf, a.d_out + r, lane);
}

// Memetic-Tabu with resumable state: each replica starts from its initial
// population or from its record in ra.d_state, runs to its stop condition
// and writes its record back (population, energies, best, counters).  The
// draws are addressed by (instance, generation, index), so a run continued
// from a record at a generation boundary equals the uninterrupted run.  A
// record of another run (N, K, variant, seed or instance) is left untouched
// and the replica reports LABS_RUN_BADSTATE.
template <int NW, bool SKEW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) mts_resume_kernel(const ResumeArgs ra) {
    extern __shared__ __align__(16) unsigned char smem[];
    const MtsArgs& a = ra.m;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + warp;
    if (r >= a.replicas) return;

    uint32_t* pop = reinterpret_cast<uint32_t*>(smem + static_cast<size_t>(warp) * a.smem_per_warp);
    int32_t* popE = reinterpret_cast<int32_t*>(pop + a.K * NW);
    int32_t* Cs = popE + a.K;
    ReplicaCfg cfg;
    cfg.N = a.N;
    cfg.K = a.K;
    cfg.p_comb_u32 = a.p_comb_u32;
    cfg.p_mut_u32 = a.p_mut_u32;
    cfg.replace_policy = a.replace_policy;
    cfg.target_E = a.target_E;
    cfg.max_generations = a.max_generations;
    cfg.max_steps = a.max_steps;
    cfg.max_iter = a.max_iter;
    cfg.variant = a.variant;
    cfg.inst = static_cast<uint32_t>(a.first_instance + static_cast<uint64_t>(r));
    cfg.key = philox_key(a.seed);

    unsigned char* rec = ra.d_state + static_cast<size_t>(r) * ra.state_bytes;
    ResumeHeader* h = reinterpret_cast<ResumeHeader*>(rec);
    uint32_t* hpop = reinterpret_cast<uint32_t*>(rec + sizeof(ResumeHeader));
    int32_t* hpopE = reinterpret_cast<int32_t*>(hpop + a.K * NW);
    ReplicaState<NW> st;
    if (ra.resume) {
        const bool match = h->N == a.N && h->K == a.K && h->variant == a.variant &&
                           h->instance == cfg.inst && h->seed == a.seed;
        if (!match) {
            if (lane == 0) {
                labs_device_result* o = a.d_out + r;
                for (int w = 0; w < LABS_MAX_W; ++w) o->seq[w] = 0;
                o->E = -1;
                o->status = LABS_RUN_BADSTATE;
                o->generations = 0;
                o->steps = 0;
                o->trace_len = 0;
            }
            return;
        }
        for (int x = lane; x < a.K * NW; x += 32) pop[x] = hpop[x];
        for (int x = lane; x < a.K; x += 32) popE[x] = hpopE[x];
#pragma unroll
        for (int w = 0; w < NW; ++w) st.best[w] = h->best[w];
        st.E_best = h->E_best;
        st.status = LABS_RUN_BUDGET;
        st.g = h->g;
        st.steps = h->steps;
        __syncwarp();
    } else {
        replica_init<NW, SKEW>(cfg, pop, popE, st, lane);
    }
    int64_t trace_len = 0;
    while (!replica_should_stop<NW>(cfg, st, a.d_glf))
        replica_generation<NW, false, SKEW>(cfg, st, pop, popE, Cs, nullptr, 0, trace_len, a.d_glf, lane);
    replica_store_result<NW>(st, 0, a.d_out + r, lane);
    __syncwarp();
    for (int x = lane; x < a.K * NW; x += 32) hpop[x] = pop[x];
    for (int x = lane; x < a.K; x += 32) hpopE[x] = popE[x];
    if (lane < 2 * LABS_MAX_W) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) v = (lane == w) ? st.best[w] : v;
        h->best[lane] = v;
    }
    if (lane == 0) {
        h->E_best = st.E_best;
        h->status = st.status;
        h->g = st.g;
        h->steps = st.steps;
        h->N = a.N;
        h->K = a.K;
        h->variant = a.variant;
        h->instance = cfg.inst;
        h->seed = a.seed;
    }
}

template <int NW, bool TRACE, bool SKEW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) tabu_kernel(const TabuArgs a) {
    __shared__ int32_t Cs_all[kWarpsPerBlock][64 * NW];  // two buffers of C_k
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t b = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + warp;
    if (b >= a.B) return;
    const int N = a.N;
    const uint2 key = philox_key(a.seed);
    const uint32_t inst = static_cast<uint32_t>(a.first_instance + static_cast<uint64_t>(b));
    constexpr int ROW = (NW + 1) & ~1;  // 32-bit words per row: whole 64-bit words
    uint32_t seq[NW];
    load_seq<NW>(reinterpret_cast<const uint32_t*>(a.d_start) + b * ROW, seq);
#pragma unroll
    for (int w = 0; w < NW; ++w) seq[w] &= word_lowmask(w, N);  // bits >= N are ignored
    if constexpr (SKEW) skew_complete<NW>(seq, N);              // the free half decides
    const int nmov = SKEW ? (N + 1) / 2 : N;
    int max_iter = a.max_iter;
    if (max_iter < 0) {
        const uint4 d = draw4(key, inst, a.generation, 1u, kPurposeGen);
        max_iter = nmov / 2 + rand_int(0, nmov, d.w);
    }
    int4* trace = a.d_trace ? a.d_trace + b * a.trace_cap : nullptr;
    int64_t trace_len = 0;
    const bool fix = (a.variant & LABS_VARIANT_FIX_FIRST_SPIN) != 0;
    TabuOut to;
    if constexpr (SKEW) {
        to = fix ? tabu_search_skew<NW, TRACE, true>(seq, N, key, inst, a.generation, max_iter, -1,
                                                     Cs_all[warp], trace, a.trace_cap, trace_len, lane)
                 : tabu_search_skew<NW, TRACE, false>(seq, N, key, inst, a.generation, max_iter, -1,
                                                      Cs_all[warp], trace, a.trace_cap, trace_len, lane);
    } else {
        to = fix ? tabu_search<NW, TRACE, true>(seq, N, key, inst, a.generation, max_iter, -1,
                                                Cs_all[warp], trace, a.trace_cap, trace_len, lane)
                 : tabu_search<NW, TRACE, false>(seq, N, key, inst, a.generation, max_iter, -1,
                                                 Cs_all[warp], trace, a.trace_cap, trace_len, lane);
    }
    if (lane < ROW) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) v = (lane == w) ? seq[w] : v;
        reinterpret_cast<uint32_t*>(a.d_best)[b * ROW + lane] = v;
    }
    if (lane == 0) {
        a.d_bestE[b] = to.E_best;
        if (a.d_steps) a.d_steps[b] = to.steps;
    }
}

template <int NW, bool TRACE, bool SKEW>
cudaError_t launch_mts_t(const MtsArgs& a, cudaStream_t stream) {
    const size_t smem = a.smem_per_warp * kWarpsPerBlock;
    cudaError_t e = cudaFuncSetAttribute(mts_kernel<NW, TRACE, SKEW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t blocks = (a.replicas + kWarpsPerBlock - 1) / kWarpsPerBlock;
    mts_kernel<NW, TRACE, SKEW><<<static_cast<unsigned>(blocks), kWarpsPerBlock * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

// 32-bit words per sequence in registers: whole 64-bit words, except three
// for 64 < N <= 96 and five for 128 < N <= 160 (less work per step than the
// next whole 64-bit word count).
inline int word_count(int N) {
    return N <= 64 ? 2 : N <= 96 ? 3 : N <= 128 ? 4 : N <= 160 ? 5 : N <= 192 ? 6 : 8;
}

template <bool SKEW>
cudaError_t launch_mts_family(const MtsArgs& a, cudaStream_t stream) {
    const bool tr = a.d_trace != nullptr;
    switch (word_count(a.N)) {
        case 2: return tr ? launch_mts_t<2, true, SKEW>(a, stream) : launch_mts_t<2, false, SKEW>(a, stream);
        case 3: return tr ? launch_mts_t<3, true, SKEW>(a, stream) : launch_mts_t<3, false, SKEW>(a, stream);
        case 4: return tr ? launch_mts_t<4, true, SKEW>(a, stream) : launch_mts_t<4, false, SKEW>(a, stream);
        case 5: return tr ? launch_mts_t<5, true, SKEW>(a, stream) : launch_mts_t<5, false, SKEW>(a, stream);
        case 6: return tr ? launch_mts_t<6, true, SKEW>(a, stream) : launch_mts_t<6, false, SKEW>(a, stream);
        default: return tr ? launch_mts_t<8, true, SKEW>(a, stream) : launch_mts_t<8, false, SKEW>(a, stream);
    }
}

template <int NW, bool SKEW>
cudaError_t launch_resume_w(const ResumeArgs& a, cudaStream_t stream) {
    const size_t smem = a.m.smem_per_warp * kWarpsPerBlock;
    cudaError_t e = cudaFuncSetAttribute(mts_resume_kernel<NW, SKEW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t blocks = (a.m.replicas + kWarpsPerBlock - 1) / kWarpsPerBlock;
    mts_resume_kernel<NW, SKEW><<<static_cast<unsigned>(blocks), kWarpsPerBlock * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

template <bool SKEW>
cudaError_t launch_resume_family(const ResumeArgs& a, cudaStream_t stream) {
    switch (word_count(a.m.N)) {
        case 2: return launch_resume_w<2, SKEW>(a, stream);
        case 3: return launch_resume_w<3, SKEW>(a, stream);
        case 4: return launch_resume_w<4, SKEW>(a, stream);
        case 5: return launch_resume_w<5, SKEW>(a, stream);
        case 6: return launch_resume_w<6, SKEW>(a, stream);
        default: return launch_resume_w<8, SKEW>(a, stream);
    }
}

template <int NW, bool SKEW>
cudaError_t launch_tabu_w(const TabuArgs& a, cudaStream_t stream) {
    const int64_t blocks = (a.B + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (a.d_trace)
        tabu_kernel<NW, true, SKEW><<<static_cast<unsigned>(blocks), kWarpsPerBlock * 32, 0, stream>>>(a);
    else
        tabu_kernel<NW, false, SKEW><<<static_cast<unsigned>(blocks), kWarpsPerBlock * 32, 0, stream>>>(a);
    return cudaGetLastError();
}

template <bool SKEW>
cudaError_t launch_tabu_family(const TabuArgs& a, cudaStream_t stream) {
    switch (word_count(a.N)) {
        case 2: return launch_tabu_w<2, SKEW>(a, stream);
        case 3: return launch_tabu_w<3, SKEW>(a, stream);
        case 4: return launch_tabu_w<4, SKEW>(a, stream);
        case 5: return launch_tabu_w<5, SKEW>(a, stream);
        case 6: return launch_tabu_w<6, SKEW>(a, stream);
        default: return launch_tabu_w<8, SKEW>(a, stream);
    }
}

}  // namespace lgpu
