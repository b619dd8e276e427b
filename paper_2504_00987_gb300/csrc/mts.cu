// mts.cu -- the unrestricted Memetic-Tabu and tabu-search kernels
// (mts_kernels.cuh) and their launchers; skew-symmetric requests go to the
// restricted family compiled in mts_skew.cu.
#include "mts_kernels.cuh"

namespace lgpu {

size_t mts_smem_per_warp(int N, int K) {
    const int NW = 2 * ((N + 63) / 64);
    const size_t bytes = static_cast<size_t>(K) * NW * 4 + static_cast<size_t>(K) * 4 + 64u * NW * 4;
    return (bytes + 15) & ~static_cast<size_t>(15);
}

cudaError_t launch_mts(const MtsArgs& a, cudaStream_t stream) {
    if (a.variant & LABS_VARIANT_SKEW) return launch_mts_skew(a, stream);
    return launch_mts_family<false>(a, stream);
}

cudaError_t launch_tabu(const TabuArgs& a, cudaStream_t stream) {
    if (a.variant & LABS_VARIANT_SKEW) return launch_tabu_skew(a, stream);
    return launch_tabu_family<false>(a, stream);
}

}  // namespace lgpu
