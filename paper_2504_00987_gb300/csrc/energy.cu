// energy.cu -- labs_energy_batch: C_k (Eq. 1) and E (Eq. 2) of B packed
// sequences.  C_k = (N - k) - 2 popc(b_i xor b_{i+k}, i < N - k): one
// funnel-shifted window, an xor and a popcount per 32 products.
//  - E only: one thread per sequence (W words in registers), reads W*8 B
//    and writes 4 B per sequence.
//  - E and C: one warp per sequence, lane l computes C_k for k = l + 32q,
//    so each row of C is written by consecutive lanes (coalesced).
#include <cuda_runtime.h>

#include "kernels.h"
#include "tabu_core.cuh"

namespace lgpu {

template <int NW>
__global__ void __launch_bounds__(256) energy_thread_kernel(const uint32_t* __restrict__ seqs, int N,
                                                            int64_t B, int32_t* __restrict__ E) {
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= B) return;
    uint32_t s[NW];
    const uint2* src = reinterpret_cast<const uint2*>(seqs + b * NW);  // 8-byte aligned rows
#pragma unroll
    for (int v = 0; v < NW / 2; ++v) {
        const uint2 x = __ldg(src + v);
        s[2 * v] = x.x;
        s[2 * v + 1] = x.y;
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) s[w] &= word_lowmask(w, N);
    E[b] = thread_energy<NW>(s, N);
}

template <int NW>
__global__ void __launch_bounds__(256) energy_warp_kernel(const uint32_t* __restrict__ seqs, int N,
                                                          int64_t B, int32_t* __restrict__ E,
                                                          int32_t* __restrict__ C) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (b >= B) return;
    uint32_t s[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) s[w] = __ldg(seqs + b * NW + w) & word_lowmask(w, N);
    int32_t c[NW];
    correlations<NW>(s, N, lane, c);
    int32_t sq = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        sq += c[q] * c[q];
        const int k = lane + 32 * q;
        if (k >= 1 && k <= N - 1) C[b * (N - 1) + (k - 1)] = c[q];
    }
    sq = __reduce_add_sync(kFull, sq);
    if (lane == 0) E[b] = sq;
}

template <int NW>
static cudaError_t launch_energy_w(const uint64_t* d_seqs, int N, int64_t B, int32_t* d_E,
                                   int32_t* d_C, cudaStream_t stream) {
    const uint32_t* seqs = reinterpret_cast<const uint32_t*>(d_seqs);
    if (d_C == nullptr) {
        const int64_t blocks = (B + 255) / 256;
        energy_thread_kernel<NW><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(seqs, N, B, d_E);
    } else {
        const int64_t blocks = (B + 7) / 8;
        energy_warp_kernel<NW><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(seqs, N, B, d_E, d_C);
    }
    return cudaGetLastError();
}

cudaError_t launch_energy(const uint64_t* d_seqs, int N, int64_t B, int32_t* d_E, int32_t* d_C,
                          cudaStream_t stream) {
    switch ((N + 63) / 64) {
        case 1: return launch_energy_w<2>(d_seqs, N, B, d_E, d_C, stream);
        case 2: return launch_energy_w<4>(d_seqs, N, B, d_E, d_C, stream);
        case 3: return launch_energy_w<6>(d_seqs, N, B, d_E, d_C, stream);
        default: return launch_energy_w<8>(d_seqs, N, B, d_E, d_C, stream);
    }
}

}  // namespace lgpu
