// batch.cu -- many independent MTS instances of uneven N, K and budget in
// one persistent launch.  The grid is sized to stay resident (blocks_per_sm
// CTAs of warps_per_block warps on every SM); each warp takes the next
// instance from a device-wide queue (one atomicAdd per instance, ordered
// longest first by the host), runs it to its stop condition with the
// replica engine and writes its result at the instance's original index.
// Instances of different word counts share the launch: the warp dispatches
// on W = ceil(N/64) per instance.  Per-instance results do not depend on
// the mapping or on the other instances (every draw is keyed by the
// instance's own seed and instance number).
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

template <int NW>
__device__ __forceinline__ void run_instance(const ReplicaCfg& cfg, unsigned char* base,
                                             labs_device_result* out, int lane) {
    uint32_t* pop = reinterpret_cast<uint32_t*>(base);
    int32_t* popE = reinterpret_cast<int32_t*>(pop + cfg.K * NW);
    int32_t* Cs = popE + cfg.K;
    replica_run<NW>(cfg, pop, popE, Cs, nullptr, 0, nullptr, out, lane);
}

template <int NWMAX>
__global__ void __launch_bounds__(256) batch_kernel(const BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char* base = smem + static_cast<size_t>(warp) * a.smem_per_warp;
    for (;;) {
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(a.queue, 1ull);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= static_cast<unsigned long long>(a.n)) break;
        const labs_instance in = a.inst[idx];
        const ReplicaCfg cfg = cfg_from_instance(in);
        labs_device_result* out = a.out + a.order[idx];
        const int W = (in.N + 63) / 64;
        if (W == 1) {
            run_instance<2>(cfg, base, out, lane);
        } else if (W == 2) {
            // four words up to N = 128: a three-word path in this kernel cost the
            // four-word one its registers (172 -> 128) and the batch's makespan,
            // which the longest (largest-N) instances set, 12 % on GB300
            if constexpr (NWMAX >= 4) run_instance<4>(cfg, base, out, lane);
        } else if (W == 3) {
            if constexpr (NWMAX >= 6) run_instance<6>(cfg, base, out, lane);
        } else {
            if constexpr (NWMAX >= 8) run_instance<8>(cfg, base, out, lane);
        }
        __syncwarp();
    }
}

static const void* batch_fn(int nwmax) {
    switch (nwmax) {
        case 2: return reinterpret_cast<const void*>(&batch_kernel<2>);
        case 4: return reinterpret_cast<const void*>(&batch_kernel<4>);
        case 6: return reinterpret_cast<const void*>(&batch_kernel<6>);
        default: return reinterpret_cast<const void*>(&batch_kernel<8>);
    }
}

cudaError_t batch_prepare(int nwmax, int warps_per_block, size_t smem_per_warp, int* max_blocks_per_sm) {
    const void* fn = batch_fn(nwmax);
    const size_t smem = smem_per_warp * warps_per_block;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, fn, warps_per_block * 32, smem);
}

cudaError_t launch_batch(const BatchArgs& a, int nwmax, int blocks, int warps_per_block, cudaStream_t stream) {
    const size_t smem = a.smem_per_warp * warps_per_block;
    switch (nwmax) {
        case 2: batch_kernel<2><<<blocks, warps_per_block * 32, smem, stream>>>(a); break;
        case 4: batch_kernel<4><<<blocks, warps_per_block * 32, smem, stream>>>(a); break;
        case 6: batch_kernel<6><<<blocks, warps_per_block * 32, smem, stream>>>(a); break;
        default: batch_kernel<8><<<blocks, warps_per_block * 32, smem, stream>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace lgpu
