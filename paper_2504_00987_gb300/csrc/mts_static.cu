// mts_static.cu -- labs_mts_run_static: the blocking Memetic-Tabu run of
// labs_mts_run with no memory allocation of any kind.
//
// Who needs it: callers that must not allocate device memory themselves or
// through the library -- a host application that owns the whole GPU memory
// budget through its own pool and forbids other allocators, a
// latency-critical loop where cudaMalloc/cudaFree (which can synchronise the
// device) or a pool that may have to grow is not acceptable, or a process
// running under a hard device-memory quota.
//
// The device scratch labs_mts_run allocates per call (one 64-byte result
// record per replica and the global termination flag) lives here in one
// file-scope __device__ array of fixed size, sized for at most
// LABS_STATIC_MAX_REPLICAS replicas (256 KiB of results plus the flag).
// Every GPU that loads the library holds this array until the process
// exits.  Host code only ever sees a host-side stand-in for the array's
// name, so every call looks up the array's device address with
// cudaGetSymbolAddress, with the caller's device current, and passes that
// address to the kernel.  The lookup is a host-side table query that
// allocates nothing; repeating it on every call keeps the address right
// after a cudaDeviceReset, which reloads the module and may place the array
// elsewhere (a cached address would then point at freed memory).  The first
// call on a device, and the first after a reset, loads the library's device
// code, which is when the array is placed: make that call before any stream
// capture.  The results are copied straight into the caller's h_out array
// and widened to labs_result in place, so the host side allocates nothing
// either.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>

#include "capi_util.h"
#include "kernels.h"
#include "labs.h"

namespace {

constexpr int64_t kMaxReplicas = LABS_STATIC_MAX_REPLICAS;
constexpr size_t kResultBytes = sizeof(labs_device_result) * static_cast<size_t>(kMaxReplicas);
constexpr size_t kFlagOffset = kResultBytes;  // a multiple of 256
constexpr size_t kScratchBytes = kResultBytes + 256;

static_assert(kFlagOffset % 256 == 0, "flag must keep the array's alignment");
static_assert(sizeof(labs_result) >= sizeof(labs_device_result), "in-place widening needs room");

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_mts_static_scratch[kScratchBytes];

// Device address of the scratch array on the current device.
int32_t scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_mts_static_scratch);
    if (e != cudaSuccess) return lcapi::cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    *out = p;
    return LABS_OK;
}

}  // namespace

extern "C" int32_t labs_mts_run_static(const labs_params* P, uint64_t seed, uint64_t first_instance,
                                       int64_t replicas, labs_result* h_out, labs_stream_t stream) {
    using namespace lcapi;
    const auto t0 = std::chrono::steady_clock::now();
    lgpu::MtsArgs a;
    LABS_TRY(make_mts_args(P, seed, first_instance, replicas, &a));
    if (replicas > kMaxReplicas)
        return fail(LABS_EINVAL, "replicas=%lld exceeds the static scratch maximum of %lld",
                    static_cast<long long>(replicas), static_cast<long long>(kMaxReplicas));
    if (replicas == 0) return ok();
    if (h_out == nullptr) return fail(LABS_EINVAL, "h_out is NULL");

    void* base = nullptr;
    LABS_TRY(scratch_address(&base));
    labs_device_result* d_out = static_cast<labs_device_result*>(base);
    uint32_t* d_flag = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) + kFlagOffset);
    a.d_out = d_out;
    a.d_glf = P->glf ? d_flag : nullptr;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The flag keeps the previous call's value: clear it before the launch.
    cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = lgpu::launch_mts(a, s);
    // Raw records into the front of the caller's array, widened in place below.
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_out, d_out, sizeof(labs_device_result) * static_cast<size_t>(replicas),
                            cudaMemcpyDeviceToHost, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "labs_mts_run_static");
    if (es != cudaSuccess) return cuda_fail(es, "labs_mts_run_static synchronize");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    // Record r sits at byte 64 r and goes to byte 96 r: walking backwards,
    // every record is read before anything is written over it.
    const unsigned char* raw = reinterpret_cast<const unsigned char*>(h_out);
    for (int64_t r = replicas - 1; r >= 0; --r) {
        labs_device_result d;
        memcpy(&d, raw + sizeof(labs_device_result) * static_cast<size_t>(r), sizeof d);
        fill_host_result(d, P->N, first_instance + static_cast<uint64_t>(r), secs, &h_out[r]);
    }
    return ok();
}
