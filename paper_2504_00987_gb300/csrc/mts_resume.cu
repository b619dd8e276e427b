// mts_resume.cu -- the resumable Memetic-Tabu kernels (mts_resume_kernel in
// mts_kernels.cuh), unrestricted and skew-symmetric, in a translation unit of
// their own so the build compiles them beside the other kernel families.
#include "mts_kernels.cuh"

namespace lgpu {

cudaError_t launch_mts_resume(const ResumeArgs& a, cudaStream_t stream) {
    if (a.m.variant & LABS_VARIANT_SKEW) return launch_resume_family<true>(a, stream);
    return launch_resume_family<false>(a, stream);
}

}  // namespace lgpu
