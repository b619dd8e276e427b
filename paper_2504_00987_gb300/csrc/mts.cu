// mts.cu -- Memetic-Tabu (Algorithm 1 / Algorithm 3) and batched tabu search
// (Algorithm 2 / Algorithm 4) kernels.  One warp runs one replica: its
// population lives in the warp's slice of shared memory (K packed
// sequences and their energies), its pivot, correlations and tabu list in
// registers (tabu_core.cuh).  Replicas never synchronise with each other;
// the only cross-replica state is the optional global termination flag.
#include <cuda_runtime.h>

#include "kernels.h"
#include "tabu_core.cuh"

namespace lgpu {

template <int NW>
__device__ __forceinline__ void load_seq(const uint32_t* __restrict__ src, uint32_t (&v)[NW]) {
#pragma unroll
    for (int w = 0; w < NW; ++w) v[w] = src[w];
}

// Energy of member p computed by one thread.
template <int NW>
__device__ __forceinline__ int32_t member_energy(const uint32_t* __restrict__ pop, int p, int N) {
    uint32_t B[NW];
    load_seq<NW>(pop + p * NW, B);
    return thread_energy<NW>(B, N);
}

// Binary tournament: the lower energy wins, the lower index on ties.
__device__ __forceinline__ int tournament(const int32_t* __restrict__ popE, int a, int b) {
    const int32_t ea = popE[a], eb = popE[b];
    if (ea < eb) return a;
    if (eb < ea) return b;
    return a < b ? a : b;
}

template <int NW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) mts_kernel(const MtsArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + warp;
    if (r >= a.replicas) return;

    const int N = a.N, K = a.K;
    uint32_t* pop = reinterpret_cast<uint32_t*>(smem + static_cast<size_t>(warp) * a.smem_per_warp);
    int32_t* popE = reinterpret_cast<int32_t*>(pop + K * NW);
    int32_t* Cs = popE + K;
    const uint2 key = philox_key(a.seed);
    const uint32_t inst = static_cast<uint32_t>(a.first_instance + static_cast<uint64_t>(r));
    int4* trace = a.d_trace ? a.d_trace + r * a.trace_cap : nullptr;
    int64_t trace_len = 0;

    // population <- K random sequences: word w of member p from (inst, p, w/2, INIT).
    for (int idx = lane; idx < K * (NW / 2); idx += 32) {
        const int p = idx / (NW / 2), w64 = idx % (NW / 2);
        const uint4 d = draw4(key, inst, static_cast<uint32_t>(p), static_cast<uint32_t>(w64), kPurposeInit);
        pop[p * NW + 2 * w64] = d.x & word_lowmask(2 * w64, N);
        pop[p * NW + 2 * w64 + 1] = d.y & word_lowmask(2 * w64 + 1, N);
    }
    __syncwarp();
    // energies; bestSeq <- lowest energy, lowest index on ties
    int32_t lbestE = INT_MAX;
    int lbest = INT_MAX;
    for (int p = lane; p < K; p += 32) {
        const int32_t e = member_energy<NW>(pop, p, N);
        popE[p] = e;
        if (e < lbestE) {
            lbestE = e;
            lbest = p;
        }
    }
    __syncwarp();
    int32_t E_best = __reduce_min_sync(kFull, lbestE);
    const int best0 = __reduce_min_sync(kFull, lbestE == E_best ? lbest : INT_MAX);
    uint32_t best[NW];
    load_seq<NW>(pop + best0 * NW, best);

    const uint32_t p_mut = a.p_mut_u32;
    int64_t g = 0, steps = 0;
    int status = LABS_RUN_BUDGET;
    const int nmut = (N + 3) / 4;  // mutation draws: one Philox block per 4 bits
    for (;;) {
        if (a.target_E >= 0 && E_best <= a.target_E) {
            status = LABS_RUN_REACHED;
            break;
        }
        if (a.max_generations >= 0 && g >= a.max_generations) break;
        if (a.max_steps >= 0 && steps >= a.max_steps) break;
        if (a.d_glf != nullptr) {
            const uint32_t f = __shfl_sync(kFull, *reinterpret_cast<volatile uint32_t*>(a.d_glf), 0);
            if (f != 0u) {
                status = LABS_RUN_STOPPED;
                break;
            }
        }
        const uint32_t gg = static_cast<uint32_t>(g);
        // generation draws: lane 0 -> (g,0), lane 1 -> (g,1), lane 2 -> (g,2)
        const uint4 gd = draw4(key, inst, gg, static_cast<uint32_t>(lane < 3 ? lane : 0), kPurposeGen);
        const uint32_t coin = __shfl_sync(kFull, gd.x, 0);
        const uint32_t ua = __shfl_sync(kFull, gd.y, 0), ub = __shfl_sync(kFull, gd.z, 0);
        const uint32_t uc = __shfl_sync(kFull, gd.w, 0), ud = __shfl_sync(kFull, gd.x, 1);
        const uint32_t ucut = __shfl_sync(kFull, gd.y, 1), usamp = __shfl_sync(kFull, gd.z, 1);
        const uint32_t uiter = __shfl_sync(kFull, gd.w, 1), urep = __shfl_sync(kFull, gd.x, 2);

        uint32_t child[NW];
        if (coin < a.p_comb_u32) {
            const int p1 = tournament(popE, rand_int(0, K - 1, ua), rand_int(0, K - 1, ub));
            const int p2 = tournament(popE, rand_int(0, K - 1, uc), rand_int(0, K - 1, ud));
            const int cut = rand_int(1, N - 1, ucut);
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t lm = word_lowmask(w, cut);
                child[w] = (pop[p1 * NW + w] & lm) | (pop[p2 * NW + w] & ~lm);
            }
        } else {
            load_seq<NW>(pop + rand_int(0, K - 1, usamp) * NW, child);
        }
        // Mutate: bit j flips iff word j%4 of (inst, g, j/4, MUT) < p_mut.
        for (int base = 0; base < nmut; base += 32) {
            const int cidx = base + lane;
            uint32_t nib = 0;
            if (cidx < nmut) {
                const uint4 d = draw4(key, inst, gg, static_cast<uint32_t>(cidx), kPurposeMut);
                nib = (d.x < p_mut ? 1u : 0u) | (d.y < p_mut ? 2u : 0u) | (d.z < p_mut ? 4u : 0u) |
                      (d.w < p_mut ? 8u : 0u);
            }
            const int word_of = cidx >> 3;  // 8 nibbles per 32-bit word
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t part = (word_of == w) ? (nib << (4 * (cidx & 7))) : 0u;
                child[w] ^= __reduce_or_sync(kFull, part) & word_lowmask(w, N);
            }
        }
        // child <- Tabu-Search(child)
        const int max_iter = a.max_iter >= 0 ? a.max_iter : N / 2 + rand_int(0, N, uiter);
        const int64_t budget = a.max_steps >= 0 ? a.max_steps - steps : -1;
        const TabuOut to = tabu_search<NW>(child, N, key, inst, gg, max_iter, budget, Cs, trace,
                                           a.trace_cap, trace_len, lane);
        steps += to.steps;
        if (to.E_best < E_best) {
            E_best = to.E_best;
#pragma unroll
            for (int w = 0; w < NW; ++w) best[w] = child[w];
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
        if (lane < NW) {
            uint32_t v = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) v = (lane == w) ? child[w] : v;
            pop[slot * NW + lane] = v;
        }
        if (lane == 0) popE[slot] = to.E_best;
        __syncwarp();
        if (trace != nullptr && trace_len < a.trace_cap) {
            if (lane == 0) trace[trace_len] = make_int4(static_cast<int>(g), 0, slot, to.E_best);
            ++trace_len;
        }
        ++g;
        if (a.d_glf != nullptr && a.target_E >= 0 && to.E_best <= a.target_E && lane == 0)
            atomicExch(a.d_glf, 1u);
    }

    labs_device_result* out = a.d_out + r;
    if (lane < 2 * LABS_MAX_W) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) v = (lane == w) ? best[w] : v;
        reinterpret_cast<uint32_t*>(out->seq)[lane] = v;
    }
    if (lane == 0) {
        out->E = E_best;
        out->status = status;
        out->generations = g;
        out->steps = steps;
        out->trace_len = trace_len;
    }
}

template <int NW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) tabu_kernel(const TabuArgs a) {
    __shared__ int32_t Cs_all[kWarpsPerBlock][32 * NW];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t b = static_cast<int64_t>(blockIdx.x) * kWarpsPerBlock + warp;
    if (b >= a.B) return;
    const int N = a.N;
    const uint2 key = philox_key(a.seed);
    const uint32_t inst = static_cast<uint32_t>(a.first_instance + static_cast<uint64_t>(b));
    uint32_t seq[NW];
    load_seq<NW>(reinterpret_cast<const uint32_t*>(a.d_start) + b * NW, seq);
#pragma unroll
    for (int w = 0; w < NW; ++w) seq[w] &= word_lowmask(w, N);  // bits >= N are ignored
    int max_iter = a.max_iter;
    if (max_iter < 0) {
        const uint4 d = draw4(key, inst, a.generation, 1u, kPurposeGen);
        max_iter = N / 2 + rand_int(0, N, d.w);
    }
    int4* trace = a.d_trace ? a.d_trace + b * a.trace_cap : nullptr;
    int64_t trace_len = 0;
    const TabuOut to = tabu_search<NW>(seq, N, key, inst, a.generation, max_iter, -1,
                                       Cs_all[warp], trace, a.trace_cap, trace_len, lane);
    if (lane < NW) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) v = (lane == w) ? seq[w] : v;
        reinterpret_cast<uint32_t*>(a.d_best)[b * NW + lane] = v;
    }
    if (lane == 0) {
        a.d_bestE[b] = to.E_best;
        if (a.d_steps) a.d_steps[b] = to.steps;
    }
}

size_t mts_smem_per_warp(int N, int K) {
    const int NW = 2 * ((N + 63) / 64);
    const size_t bytes = static_cast<size_t>(K) * NW * 4 + static_cast<size_t>(K) * 4 + 32u * NW * 4;
    return (bytes + 15) & ~static_cast<size_t>(15);
}

template <int NW>
static cudaError_t launch_mts_w(const MtsArgs& a, cudaStream_t stream) {
    const size_t smem = a.smem_per_warp * kWarpsPerBlock;
    cudaError_t e = cudaFuncSetAttribute(mts_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t blocks = (a.replicas + kWarpsPerBlock - 1) / kWarpsPerBlock;
    mts_kernel<NW><<<static_cast<unsigned>(blocks), kWarpsPerBlock * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mts(const MtsArgs& a, cudaStream_t stream) {
    switch ((a.N + 63) / 64) {
        case 1: return launch_mts_w<2>(a, stream);
        case 2: return launch_mts_w<4>(a, stream);
        case 3: return launch_mts_w<6>(a, stream);
        default: return launch_mts_w<8>(a, stream);
    }
}

template <int NW>
static cudaError_t launch_tabu_w(const TabuArgs& a, cudaStream_t stream) {
    const int64_t blocks = (a.B + kWarpsPerBlock - 1) / kWarpsPerBlock;
    tabu_kernel<NW><<<static_cast<unsigned>(blocks), kWarpsPerBlock * 32, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tabu(const TabuArgs& a, cudaStream_t stream) {
    switch ((a.N + 63) / 64) {
        case 1: return launch_tabu_w<2>(a, stream);
        case 2: return launch_tabu_w<4>(a, stream);
        case 3: return launch_tabu_w<6>(a, stream);
        default: return launch_tabu_w<8>(a, stream);
    }
}

}  // namespace lgpu
