// serve.cu -- the quantum kernel of the solve service.  Every active slot
// (one admitted request) gets one warp: the warp resumes the slot's replica
// from its device-resident state (population and energies in the slot's
// extent of the HBM arena, best sequence and counters in the slot record),
// runs whole generations until the replica stops or the quantum's step
// allowance is used, and suspends it again.  Suspension only ever happens
// at a generation boundary, where the replica's state is exactly
// (population, best, g, steps), so a request's trajectory does not depend
// on the quantum size or on which other requests share the launch.  The
// kernel never waits on anything: it is bounded by the quantum and one
// generation.  The quantum is a step count, and optionally a device-time
// budget, so that slots of small N are not held to the pace of the largest
// one.  One launch serves one word-count class (serve_class_nw), so its
// shared memory per warp is that class's, not the largest N's.
#include <cuda_runtime.h>

#include "kernels.h"
#include "replica.cuh"

namespace lgpu {

__device__ __forceinline__ ReplicaCfg serve_cfg(const labs_instance& in) {
    ReplicaCfg c;
    c.N = in.N;
    c.K = in.K;
    c.p_comb_u32 = in.p_comb_u32;
    c.p_mut_u32 = in.p_mut_u32;
    c.replace_policy = in.replace_policy;
    c.target_E = in.target_E;
    c.max_generations = in.max_generations;
    c.max_steps = in.max_steps;
    c.max_iter = in.max_iter;
    c.variant = in.variant;
    c.inst = static_cast<uint32_t>(in.instance);
    c.key = philox_key(in.seed);
    return c;
}

// Device time in nanoseconds (the %globaltimer register), read by lane 0 and
// broadcast so that every lane takes the same decision.
__device__ __forceinline__ uint64_t warp_globaltimer(int lane) {
    uint64_t t = 0;
    if (lane == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return __shfl_sync(kFull, t, 0);
}

// One slot's quantum.  WPS = 2: two warps run the slot's replica (each on its
// own copy of the state, splitting every tabu step's neighbours); the lower
// one takes the device-time decisions and writes the state back, and the
// pair shakes hands after loading so that the write-back cannot overtake the
// other warp's load.
template <int NW, int WPS, int HALF>
__device__ void serve_slot(const ServeArgs& a, int i, int slot, const labs_instance& in,
                           unsigned char* base, int lane, PairLink* link) {
    const ReplicaCfg cfg = serve_cfg(in);
    const int K = cfg.K;
    uint32_t* pop = reinterpret_cast<uint32_t*>(base);
    int32_t* popE = reinterpret_cast<int32_t*>(pop + K * NW);
    int32_t* Cs = popE + K;
    uint32_t* hpop = a.pop + a.pop_off[slot];
    int32_t* hpopE = reinterpret_cast<int32_t*>(hpop + K * NW);
    ServeState* S = a.state + slot;
    uint32_t xseq = 1;

    ReplicaState<NW> st;
    if (S->phase == kSlotFresh) {
        replica_init<NW>(cfg, pop, popE, st, lane);
    } else {
        for (int x = lane; x < K * NW; x += 32) pop[x] = hpop[x];
        for (int x = lane; x < K; x += 32) popE[x] = hpopE[x];
#pragma unroll
        for (int w = 0; w < NW; ++w) st.best[w] = S->best[w];
        st.E_best = S->E_best;
        st.status = S->status;
        st.g = S->g;
        st.steps = S->steps;
        __syncwarp();
    }
    if constexpr (WPS == 2) {
        uint64_t o = 0;
        if (!pair_exchange(link, HALF, xseq++, 0u, o, lane)) st.status = LABS_RUN_SYNC_LOST;
    }
    int64_t used = 0, trace_len = 0;
    bool finished = false;
    const uint64_t t0 = a.quantum_ns ? warp_globaltimer(lane) : 0;
    for (int gens = 0;; ++gens) {
        if (replica_should_stop<NW>(cfg, st, nullptr)) {
            finished = true;
            break;
        }
        if (used >= a.quantum_steps) break;
        if (a.quantum_ns && gens > 0) {
            bool over = HALF == 0 && warp_globaltimer(lane) - t0 >= a.quantum_ns;
            if constexpr (WPS == 2) {  // the lower warp's clock decides for both
                uint64_t o = 0;
                if (!pair_exchange(link, HALF, xseq++, over ? 1u : 0u, o, lane)) {
                    st.status = LABS_RUN_SYNC_LOST;
                    continue;  // stops at the test above
                }
                over = o != 0 || (HALF == 0 && over);
            }
            if (over) break;
        }
        // correlations updated per k (PERK): a request's warp mostly runs alone on its sub-partition
        used += replica_generation<NW, false, false, WPS, HALF, true>(cfg, st, pop, popE, Cs, nullptr, 0,
                                                                      trace_len, nullptr, lane, link, &xseq);
    }
    if (HALF != 0) return;
    if (finished) {
        replica_store_result<NW>(st, 0, a.out + i, lane);
    } else {
        for (int x = lane; x < K * NW; x += 32) hpop[x] = pop[x];
        for (int x = lane; x < K; x += 32) hpopE[x] = popE[x];
    }
    if (lane < NW) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) v = (lane == w) ? st.best[w] : v;
        S->best[lane] = v;
    }
    if (lane == 0) {
        S->E_best = st.E_best;
        S->status = st.status;
        S->g = st.g;
        S->steps = st.steps;
        S->phase = finished ? kSlotDone : kSlotSuspended;
        a.done[i] = finished ? 1 : 0;
        a.quantum_used[i] = used;
    }
}

// Pairs take as many registers as they need (at most one CTA per SM is
// promised, which spares them spills); single warps keep the default budget.
template <int NW, int WPS>
__global__ void __launch_bounds__(256, WPS == 2 ? 1 : 0) serve_quantum_kernel(const ServeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PairLink links[WPS == 2 ? 4 : 1];  // one per pair of an 8-warp CTA
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    PairLink* link = WPS == 2 ? &links[warp >> 1] : nullptr;
    if constexpr (WPS == 2) {
        if (lane < 4) reinterpret_cast<unsigned long long*>(link->slot)[lane] = 0ull;
        __syncthreads();  // every link word is zero before either warp of a pair publishes
    }
    const int i = (blockIdx.x * (blockDim.x >> 5) + warp) / WPS;
    if (i >= a.n_active) return;
    unsigned char* base = smem + static_cast<size_t>(warp) * a.smem_per_warp;
    const int slot = a.active[i];
    const labs_instance in = a.cfg[slot];
    if (WPS == 2 && (warp & 1))
        serve_slot<NW, WPS, WPS - 1>(a, i, slot, in, base, lane, link);
    else
        serve_slot<NW, WPS, 0>(a, i, slot, in, base, lane, link);
}

int serve_class_nw(int N) { return N <= 64 ? 2 : N <= 96 ? 3 : N <= 128 ? 4 : N <= 160 ? 5 : N <= 192 ? 6 : 8; }

size_t serve_smem_per_warp(int nw, int K) {
    // population (K x nw words), energies (K), two buffers of C_k (64 nw)
    const size_t bytes = (static_cast<size_t>(K) * nw + static_cast<size_t>(K) + 64u * nw) * 4u;
    return (bytes + 15) & ~static_cast<size_t>(15);
}

// Two warps per slot need an even word count (the halves of every step).
static const void* serve_fn(int nw, int wps) {
    if (wps == 2) {
        switch (nw) {
            case 2: return reinterpret_cast<const void*>(&serve_quantum_kernel<2, 2>);
            case 4: return reinterpret_cast<const void*>(&serve_quantum_kernel<4, 2>);
            case 6: return reinterpret_cast<const void*>(&serve_quantum_kernel<6, 2>);
            case 8: return reinterpret_cast<const void*>(&serve_quantum_kernel<8, 2>);
            default: break;
        }
    }
    switch (nw) {
        case 2: return reinterpret_cast<const void*>(&serve_quantum_kernel<2, 1>);
        case 3: return reinterpret_cast<const void*>(&serve_quantum_kernel<3, 1>);
        case 4: return reinterpret_cast<const void*>(&serve_quantum_kernel<4, 1>);
        case 5: return reinterpret_cast<const void*>(&serve_quantum_kernel<5, 1>);
        case 6: return reinterpret_cast<const void*>(&serve_quantum_kernel<6, 1>);
        default: return reinterpret_cast<const void*>(&serve_quantum_kernel<8, 1>);
    }
}

int serve_pairs_supported(int nw) { return nw % 2 == 0 ? 1 : 0; }

cudaError_t serve_blocks_per_sm(int nw, int wps, int warps_per_block, size_t smem_per_warp, int* blocks) {
    const void* fn = serve_fn(nw, wps);
    const size_t smem = smem_per_warp * warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, warps_per_block * 32, smem);
}

cudaError_t launch_serve_quantum(const ServeArgs& a, int nw, int wps, int warps_per_block, cudaStream_t stream) {
    if (a.n_active <= 0) return cudaSuccess;
    if (wps == 2 && (nw % 2 != 0 || warps_per_block % 2 != 0)) return cudaErrorInvalidValue;
    const size_t smem = a.smem_per_warp * warps_per_block;
    const int slots_per_block = warps_per_block / wps;
    const int blocks = (a.n_active + slots_per_block - 1) / slots_per_block;
    const void* fn = serve_fn(nw, wps);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(static_cast<unsigned>(warps_per_block * 32));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    void* args[] = {const_cast<ServeArgs*>(&a)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace lgpu
