// batch.cu -- many independent MTS instances of uneven N, K and budget in
// one persistent launch.  The grid is sized to stay resident (blocks_per_sm
// CTAs of warps_per_block warps on every SM); each replica unit (one warp,
// or with warps_per_seq = 2 a pair of warps that split every step's
// neighbours) takes the next instance from a device-wide queue (one
// atomicAdd per instance, ordered longest first by the host), runs it to
// its stop condition with the replica engine and writes its result at the
// instance's original index.  Instances of different word counts share the
// launch: the unit dispatches on W = ceil(N/64) per instance.  Per-instance
// results do not depend on the mapping or on the other instances (every
// draw is keyed by the instance's own seed and instance number).
#include <cuda_runtime.h>

#include "kernels.h"
#include "replica.cuh"

namespace lgpu {

__device__ __forceinline__ ReplicaCfg cfg_from_instance(const labs_instance& in) {
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

template <int NW, int WPS, int HALF>
__device__ __forceinline__ void run_instance(const ReplicaCfg& cfg, unsigned char* base,
                                             labs_device_result* out, int lane, PairLink* link,
                                             uint32_t* xseq) {
    uint32_t* pop = reinterpret_cast<uint32_t*>(base);
    int32_t* popE = reinterpret_cast<int32_t*>(pop + cfg.K * NW);
    int32_t* Cs = popE + cfg.K;
    // correlations updated per k (PERK): the batch's warps run alone on their SM sub-partitions
    replica_run<NW, false, false, WPS, HALF, true>(cfg, pop, popE, Cs, nullptr, 0, nullptr, out, lane, link, xseq);
}

// The queue loop of one unit.  WPS = 2: half 0 takes the instance and tells
// half 1 through the pair's link; both then run it.
template <int NWMAX, int WPS, int HALF>
__device__ __forceinline__ void batch_unit(const BatchArgs& a, unsigned char* base, int lane, PairLink* link) {
    uint32_t xseq = 1;  // exchange 0 would match the zeroed link words
    for (;;) {
        unsigned long long idx = 0;
        if (HALF == 0) {
            if (lane == 0) idx = atomicAdd(a.queue, 1ull);
            idx = __shfl_sync(kFull, idx, 0);
        }
        if constexpr (WPS == 2) {
            uint64_t o = 0;
            if (!pair_exchange(link, HALF, xseq++, HALF == 0 ? idx : 0u, o, lane)) {
                // the pair lost step: the instance this warp took is reported, not run
                if (HALF == 0 && lane == 0 && idx < static_cast<unsigned long long>(a.n)) {
                    labs_device_result* out = a.out + a.order[idx];
                    for (int w = 0; w < LABS_MAX_W; ++w) out->seq[w] = 0;
                    out->E = -1;
                    out->status = LABS_RUN_SYNC_LOST;
                    out->generations = 0;
                    out->steps = 0;
                    out->trace_len = 0;
                }
                break;
            }
            if (HALF == 1) idx = o;
        }
        if (idx >= static_cast<unsigned long long>(a.n)) break;
        const labs_instance in = a.inst[idx];
        const ReplicaCfg cfg = cfg_from_instance(in);
        labs_device_result* out = a.out + a.order[idx];
        const int W = (in.N + 63) / 64;
        if (W == 1) {
            run_instance<2, WPS, HALF>(cfg, base, out, lane, link, &xseq);
        } else if (W == 2) {
            // four words up to N = 128: a three-word path in this kernel cost the
            // four-word one its registers (172 -> 128) and the batch's makespan,
            // which the longest (largest-N) instances set, 12 % on GB300
            if constexpr (NWMAX >= 4) run_instance<4, WPS, HALF>(cfg, base, out, lane, link, &xseq);
        } else if (W == 3) {
            if constexpr (NWMAX >= 6) run_instance<6, WPS, HALF>(cfg, base, out, lane, link, &xseq);
        } else {
            if constexpr (NWMAX >= 8) run_instance<8, WPS, HALF>(cfg, base, out, lane, link, &xseq);
        }
        __syncwarp();
    }
}

// Pairs take as many registers as they need (see serve_quantum_kernel).
template <int NWMAX, int WPS>
__global__ void __launch_bounds__(256, WPS == 2 ? 1 : 0) batch_kernel(const BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PairLink links[WPS == 2 ? 4 : 1];  // one per pair of an 8-warp CTA
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* base = smem + static_cast<size_t>(warp) * a.smem_per_warp;
    if constexpr (WPS == 1) {
        batch_unit<NWMAX, 1, 0>(a, base, lane, nullptr);
    } else {
        PairLink* link = &links[warp >> 1];
        if (lane < 4) reinterpret_cast<unsigned long long*>(link->slot)[lane] = 0ull;
        __syncthreads();  // every link word is zero before either warp of a pair publishes
        if (warp & 1)
            batch_unit<NWMAX, 2, 1>(a, base, lane, link);
        else
            batch_unit<NWMAX, 2, 0>(a, base, lane, link);
    }
}

static const void* batch_fn(int nwmax, int wps) {
    if (wps == 2) {
        switch (nwmax) {
            case 2: return reinterpret_cast<const void*>(&batch_kernel<2, 2>);
            case 4: return reinterpret_cast<const void*>(&batch_kernel<4, 2>);
            case 6: return reinterpret_cast<const void*>(&batch_kernel<6, 2>);
            default: return reinterpret_cast<const void*>(&batch_kernel<8, 2>);
        }
    }
    switch (nwmax) {
        case 2: return reinterpret_cast<const void*>(&batch_kernel<2, 1>);
        case 4: return reinterpret_cast<const void*>(&batch_kernel<4, 1>);
        case 6: return reinterpret_cast<const void*>(&batch_kernel<6, 1>);
        default: return reinterpret_cast<const void*>(&batch_kernel<8, 1>);
    }
}

cudaError_t batch_prepare(int nwmax, int wps, int warps_per_block, size_t smem_per_warp, int* max_blocks_per_sm) {
    const void* fn = batch_fn(nwmax, wps);
    const size_t smem = smem_per_warp * warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, fn, warps_per_block * 32, smem);
}

cudaError_t launch_batch(const BatchArgs& a, int nwmax, int wps, int blocks, int warps_per_block,
                         cudaStream_t stream) {
    if (wps == 2 && warps_per_block % 2 != 0) return cudaErrorInvalidValue;
    const size_t smem = a.smem_per_warp * warps_per_block;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(static_cast<unsigned>(warps_per_block * 32));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    void* args[] = {const_cast<BatchArgs*>(&a)};
    return cudaLaunchKernelExC(&cfg, batch_fn(nwmax, wps), args);
}

}  // namespace lgpu
