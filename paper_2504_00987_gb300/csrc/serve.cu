// serve.cu -- the quantum kernel of the solve service.  Every active slot
// (one admitted request) gets one warp: the warp resumes the slot's replica
// from its device-resident state (population and energies in the HBM
// arena, best sequence and counters in the slot record), runs whole
// generations until the replica stops or the quantum's step allowance is
// used, and suspends it again.  Suspension only ever happens at a
// generation boundary, where the replica's state is exactly (population,
// best, g, steps), so a request's trajectory does not depend on the quantum
// size or on which other requests share the launch.  The kernel never waits
// on anything: it is bounded by the quantum and one generation.  The quantum
// is a step count, and optionally a device-time budget, so that slots of
// small N are not held to the pace of the largest one.
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

template <int NW>
__device__ void serve_slot(const ServeArgs& a, int i, int slot, const labs_instance& in,
                           unsigned char* base, int lane) {
    const ReplicaCfg cfg = serve_cfg(in);
    const int K = cfg.K;
    uint32_t* pop = reinterpret_cast<uint32_t*>(base);
    int32_t* popE = reinterpret_cast<int32_t*>(pop + K * NW);
    int32_t* Cs = popE + K;
    uint32_t* hpop = a.pop + static_cast<size_t>(slot) * a.pop_stride_words;
    int32_t* hpopE = reinterpret_cast<int32_t*>(hpop + K * NW);
    ServeState* S = a.state + slot;

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
    int64_t used = 0, trace_len = 0;
    bool finished = false;
    const uint64_t t0 = a.quantum_ns ? warp_globaltimer(lane) : 0;
    for (int gens = 0;; ++gens) {
        if (replica_should_stop<NW>(cfg, st, nullptr)) {
            finished = true;
            break;
        }
        if (used >= a.quantum_steps) break;
        if (a.quantum_ns && gens > 0 && warp_globaltimer(lane) - t0 >= a.quantum_ns) break;
        used += replica_generation<NW>(cfg, st, pop, popE, Cs, nullptr, 0, trace_len, nullptr, lane);
    }
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

template <int NWMAX>
__global__ void __launch_bounds__(256) serve_quantum_kernel(const ServeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= a.n_active) return;
    unsigned char* base = smem + static_cast<size_t>(warp) * a.smem_per_warp;
    const int slot = a.active[i];
    const labs_instance in = a.cfg[slot];
    const int W = (in.N + 63) / 64;
    if (W == 1) {
        serve_slot<2>(a, i, slot, in, base, lane);
    } else if (W == 2) {  // three 32-bit words up to N = 96
        if constexpr (NWMAX >= 4) {
            if (in.N <= 96)
                serve_slot<3>(a, i, slot, in, base, lane);
            else
                serve_slot<4>(a, i, slot, in, base, lane);
        }
    } else if (W == 3) {  // five 32-bit words up to N = 160
        if constexpr (NWMAX >= 6) {
            if (in.N <= 160)
                serve_slot<5>(a, i, slot, in, base, lane);
            else
                serve_slot<6>(a, i, slot, in, base, lane);
        }
    } else {
        if constexpr (NWMAX >= 8) serve_slot<8>(a, i, slot, in, base, lane);
    }
}

cudaError_t launch_serve_quantum(const ServeArgs& a, int nwmax, int warps_per_block, cudaStream_t stream) {
    if (a.n_active <= 0) return cudaSuccess;
    const size_t smem = a.smem_per_warp * warps_per_block;
    const int blocks = (a.n_active + warps_per_block - 1) / warps_per_block;
    const void* fn;
    switch (nwmax) {
        case 2: fn = reinterpret_cast<const void*>(&serve_quantum_kernel<2>); break;
        case 4: fn = reinterpret_cast<const void*>(&serve_quantum_kernel<4>); break;
        case 6: fn = reinterpret_cast<const void*>(&serve_quantum_kernel<6>); break;
        default: fn = reinterpret_cast<const void*>(&serve_quantum_kernel<8>); break;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    switch (nwmax) {
        case 2: serve_quantum_kernel<2><<<blocks, warps_per_block * 32, smem, stream>>>(a); break;
        case 4: serve_quantum_kernel<4><<<blocks, warps_per_block * 32, smem, stream>>>(a); break;
        case 6: serve_quantum_kernel<6><<<blocks, warps_per_block * 32, smem, stream>>>(a); break;
        default: serve_quantum_kernel<8><<<blocks, warps_per_block * 32, smem, stream>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace lgpu
