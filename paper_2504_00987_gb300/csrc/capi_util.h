// capi_util.h -- argument checks and error reporting shared by the C ABI
// translation units (internal; not installed).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>

#include "labs.h"

namespace lgpu {
struct MtsArgs;
}

namespace lcapi {

int32_t fail(int32_t code, const char* fmt, ...);
int32_t ok();
int32_t cuda_fail(cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
int32_t check_dev(const void* p, size_t align, const char* name, bool nullable);
int32_t check_N(int32_t N);
// Validates the run parameters shared by labs_params and labs_instance.
int32_t check_run(int32_t N, int32_t K, int32_t replace_policy, int32_t target_E,
                  int64_t max_generations, int64_t max_steps, int32_t max_iter, uint64_t first_instance,
                  int64_t count, const char* who);
// Unknown flags, and LABS_VARIANT_SKEW with even N or where it is not served.
int32_t check_variant(int32_t variant, int32_t N, bool skew_allowed, const char* who);
// The given threshold, or floor(2^32 / spins mutated) if 0.
uint32_t default_p_mut(int32_t N, uint32_t p_mut_u32, int32_t variant);
int sm_count();
// An NVTX range for the scope (host-side phases: quanta, batch launches,
// autotuning, blocking runs); costs nothing unless a profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
// Validates P and fills the Memetic-Tabu kernel arguments of labs_mts_launch,
// labs_mts_run and labs_mts_run_static (everything except the device pointers).
int32_t make_mts_args(const labs_params* P, uint64_t seed, uint64_t first_instance,
                      int64_t replicas, lgpu::MtsArgs* a);
void fill_host_result(const labs_device_result& d, int32_t N, uint64_t instance, double seconds,
                      labs_result* o);

}  // namespace lcapi

#define LABS_TRY(expr)                  \
    do {                                \
        const int32_t rc_ = (expr);     \
        if (rc_ != LABS_OK) return rc_; \
    } while (0)
