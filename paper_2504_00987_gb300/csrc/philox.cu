// philox.cu -- labs_philox_batch: the words of the randomness contract
// (Philox4x32-10 under key (seed low, seed high), counter (instance, a, b,
// purpose)) for B given counters, computed by the same device function the
// kernels draw with.  One thread per counter: 16 B read, 16 B written.
#include <cuda_runtime.h>

#include "capi_util.h"
#include "labs_device.cuh"

namespace lgpu {

__global__ void __launch_bounds__(256) philox_kernel(uint2 key, const uint4* __restrict__ ctr, int64_t B,
                                                     uint4* __restrict__ out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint4 c = ctr[i];
    out[i] = draw4(key, c.x, c.y, c.z, c.w);
}

}  // namespace lgpu

extern "C" int32_t labs_philox_batch(uint64_t seed, const uint32_t* d_ctr, int64_t B, uint32_t* d_out,
                                     labs_stream_t stream) {
    using namespace lcapi;
    if (B < 0) return fail(LABS_EINVAL, "B < 0");
    if (B == 0) return ok();
    if (B > (int64_t{1} << 36)) return fail(LABS_EINVAL, "B too large");
    LABS_TRY(check_dev(d_ctr, 16, "d_ctr", false));
    LABS_TRY(check_dev(d_out, 16, "d_out", false));
    const int64_t blocks = (B + 255) / 256;
    lgpu::philox_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)), reinterpret_cast<const uint4*>(d_ctr),
        B, reinterpret_cast<uint4*>(d_out));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "philox kernel launch");
    return ok();
}
