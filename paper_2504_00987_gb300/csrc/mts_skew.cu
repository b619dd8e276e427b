// mts_skew.cu -- the Memetic-Tabu and tabu-search kernels restricted to
// skew-symmetric sequences of odd length (Sec. II.C; mts_kernels.cuh with
// SKEW = true, tabu_skew.cuh for the pair moves).
#include "mts_kernels.cuh"

namespace lgpu {

cudaError_t launch_mts_skew(const MtsArgs& a, cudaStream_t stream) { return launch_mts_family<true>(a, stream); }

cudaError_t launch_tabu_skew(const TabuArgs& a, cudaStream_t stream) { return launch_tabu_family<true>(a, stream); }

}  // namespace lgpu
