// capi.cu -- the extern "C" boundary of liblabs.so (declared in labs.h):
// argument and pointer-kind checks, error strings, launches, and the
// blocking labs_mts_run wrapper with its device scratch.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "capi_util.h"
#include "kernels.h"
#include "labs.h"

namespace lcapi {

thread_local char g_err[512] = {0};

int32_t fail(int32_t code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int32_t ok() {
    g_err[0] = 0;
    return LABS_OK;
}

int32_t cuda_fail(cudaError_t e, const char* what) {
    return fail(LABS_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// True if p is device (or managed) memory of the current context.
bool is_device_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error state of the failed query
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int32_t check_dev(const void* p, size_t align, const char* name, bool nullable) {
    if (p == nullptr) return nullable ? LABS_OK : fail(LABS_EINVAL, "%s is NULL", name);
    if (!is_device_ptr(p)) return fail(LABS_EINVAL, "%s is not device memory", name);
    if (!aligned(p, align)) return fail(LABS_EINVAL, "%s is not %zu-byte aligned", name, align);
    return LABS_OK;
}

int32_t check_N(int32_t N) {
    if (N < 3 || N > LABS_MAX_N) return fail(LABS_EINVAL, "N=%d outside 3..%d", N, LABS_MAX_N);
    return LABS_OK;
}

int32_t check_run(int32_t N, int32_t K, int32_t replace_policy, int32_t target_E,
                  int64_t max_generations, int64_t max_steps, int32_t max_iter, uint64_t first_instance,
                  int64_t count, const char* who) {
    if (N < 3 || N > LABS_MAX_N) return fail(LABS_EINVAL, "%s: N=%d outside 3..%d", who, N, LABS_MAX_N);
    if (K < 1 || K > LABS_MAX_K) return fail(LABS_EINVAL, "%s: K=%d outside 1..%d", who, K, LABS_MAX_K);
    if (replace_policy != LABS_REPLACE_RANDOM && replace_policy != LABS_REPLACE_WORST)
        return fail(LABS_EINVAL, "%s: unknown replace_policy %d", who, replace_policy);
    if (max_iter < -1 || max_iter > (1 << 20))
        return fail(LABS_EINVAL, "%s: max_iter=%d outside -1..2^20", who, max_iter);
    if (target_E < -1) return fail(LABS_EINVAL, "%s: target_E=%d (use -1 for none)", who, target_E);
    if (max_generations < -1 || max_steps < -1)
        return fail(LABS_EINVAL, "%s: budgets must be -1 (unlimited) or >= 0", who);
    // Every run must end: a generation budget, or a step budget with steps
    // that advance.  Generation numbers index the Philox counter (32 bits).
    const bool gen_bound = max_generations >= 0;
    const bool step_bound = max_steps >= 0 && max_iter != 0;
    if (!gen_bound && !step_bound)
        return fail(LABS_EINVAL,
                    "%s: unbounded run: set max_generations, or max_steps with max_iter != 0", who);
    if ((gen_bound ? max_generations : max_steps) > 0xFFFFFFFFll)
        return fail(LABS_EINVAL, "%s: more than 2^32 - 1 generations possible", who);
    if (count < 0) return fail(LABS_EINVAL, "%s: negative count", who);
    if (first_instance + static_cast<uint64_t>(count) > 0x100000000ull)
        return fail(LABS_EINVAL, "%s: instances beyond 2^32 - 1", who);
    if (lgpu::mts_smem_per_warp(N, K) > 227u * 1024u)
        return fail(LABS_EINVAL, "%s: population does not fit in shared memory (N=%d, K=%d)", who, N, K);
    return LABS_OK;
}

int32_t check_variant(int32_t variant, int32_t N, bool skew_allowed, const char* who) {
    if (variant & ~(LABS_VARIANT_UNIFORM_CROSSOVER | LABS_VARIANT_FIX_FIRST_SPIN | LABS_VARIANT_SKEW))
        return fail(LABS_EINVAL, "%s: unknown variant flags 0x%x", who, variant);
    if (variant & LABS_VARIANT_SKEW) {
        if (!skew_allowed)
            return fail(LABS_EINVAL,
                        "%s: LABS_VARIANT_SKEW runs through labs_mts_launch/run/run_static and "
                        "labs_tabu_run only", who);
        if (N % 2 == 0) return fail(LABS_EINVAL, "%s: LABS_VARIANT_SKEW needs odd N (N=%d)", who, N);
    }
    return LABS_OK;
}

uint32_t default_p_mut(int32_t N, uint32_t p_mut_u32, int32_t variant) {
    if (p_mut_u32 != 0) return p_mut_u32;
    const int32_t free_spins = (variant & LABS_VARIANT_SKEW) ? (N + 1) / 2 : N;  // 1 / (spins mutated)
    return static_cast<uint32_t>((1ull << 32) / free_spins);
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

void fill_host_result(const labs_device_result& d, int32_t N, uint64_t instance, double seconds,
                      labs_result* o) {
    memcpy(o->seq, d.seq, sizeof o->seq);
    o->E = d.E;
    o->N = N;
    o->F = d.E > 0 ? static_cast<double>(N) * N / (2.0 * d.E) : 0.0;
    o->generations = d.generations;
    o->steps = d.steps;
    o->flip_evals = d.steps * N;
    o->trace_len = d.trace_len;
    o->instance = instance;
    o->seconds = seconds;
    o->status = d.status;
    o->pad = 0;
}

// Validates P and fills the kernel arguments (everything except pointers).
int32_t make_mts_args(const labs_params* P, uint64_t seed, uint64_t first_instance,
                      int64_t replicas, lgpu::MtsArgs* a) {
    if (P == nullptr) return fail(LABS_EINVAL, "params is NULL");
    LABS_TRY(check_run(P->N, P->K, P->replace_policy, P->target_E, P->max_generations, P->max_steps,
                       P->max_iter, first_instance, replicas, "params"));
    if (replicas > (static_cast<int64_t>(1) << 31) * lgpu::kWarpsPerBlock / 2)
        return fail(LABS_EINVAL, "too many replicas for one launch");
    if (P->trace_cap < 0) return fail(LABS_EINVAL, "trace_cap < 0");
    if (P->d_trace != nullptr) LABS_TRY(check_dev(P->d_trace, 16, "d_trace", false));
    LABS_TRY(check_variant(P->variant, P->N, true, "params"));
    const size_t per_warp = lgpu::mts_smem_per_warp(P->N, P->K);
    if (per_warp * lgpu::kWarpsPerBlock > 227u * 1024u)
        return fail(LABS_EINVAL, "population does not fit in shared memory (N=%d, K=%d)", P->N, P->K);

    a->N = P->N;
    a->K = P->K;
    a->p_comb_u32 = P->p_comb_u32;
    a->p_mut_u32 = default_p_mut(P->N, P->p_mut_u32, P->variant);
    a->replace_policy = P->replace_policy;
    a->target_E = P->target_E;
    a->max_generations = P->max_generations;
    a->max_steps = P->max_steps;
    a->max_iter = P->max_iter;
    a->variant = P->variant;
    a->seed = seed;
    a->first_instance = first_instance;
    a->replicas = replicas;
    a->d_out = nullptr;
    a->d_glf = nullptr;
    a->d_trace = reinterpret_cast<int4*>(P->d_trace);
    a->trace_cap = P->d_trace ? P->trace_cap : 0;
    a->smem_per_warp = per_warp;
    return LABS_OK;
}

}  // namespace lcapi

using namespace lcapi;

extern "C" {

const char* labs_last_error(void) { return lcapi::g_err; }

int32_t labs_version(void) { return 100; }

int32_t labs_energy_batch(const uint64_t* d_seqs, int32_t N, int64_t B, int32_t* d_E, int32_t* d_C,
                          labs_stream_t stream) {
    LABS_TRY(check_N(N));
    if (B < 0) return fail(LABS_EINVAL, "B < 0");
    if (B == 0) return ok();
    if (B > (static_cast<int64_t>(1) << 36)) return fail(LABS_EINVAL, "B too large");
    LABS_TRY(check_dev(d_seqs, 8, "d_seqs", false));
    LABS_TRY(check_dev(d_E, 4, "d_E", false));
    LABS_TRY(check_dev(d_C, 4, "d_C", true));
    const cudaError_t e =
        lgpu::launch_energy(d_seqs, N, B, d_E, d_C, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "energy kernel launch");
    return ok();
}

int32_t labs_tabu_run(const uint64_t* d_start, int32_t N, int64_t B, uint64_t seed,
                      const labs_tabu_opts* opts, uint64_t* d_best, int32_t* d_bestE,
                      int64_t* d_steps, int32_t* d_trace, labs_stream_t stream) {
    LABS_TRY(check_N(N));
    if (opts == nullptr) return fail(LABS_EINVAL, "opts is NULL");
    if (B < 0) return fail(LABS_EINVAL, "B < 0");
    if (opts->max_iter < -1 || opts->max_iter > (1 << 20))
        return fail(LABS_EINVAL, "max_iter=%d outside -1..2^20", opts->max_iter);
    if (opts->trace_cap < 0) return fail(LABS_EINVAL, "trace_cap < 0");
    LABS_TRY(check_variant(opts->variant, N, true, "opts"));
    if (opts->first_instance + static_cast<uint64_t>(B) > 0x100000000ull)
        return fail(LABS_EINVAL, "instances beyond 2^32 - 1");
    if (B == 0) return ok();
    if (B > (static_cast<int64_t>(1) << 31)) return fail(LABS_EINVAL, "B too large");
    LABS_TRY(check_dev(d_start, 8, "d_start", false));
    LABS_TRY(check_dev(d_best, 8, "d_best", false));
    LABS_TRY(check_dev(d_bestE, 4, "d_bestE", false));
    LABS_TRY(check_dev(d_steps, 8, "d_steps", true));
    LABS_TRY(check_dev(d_trace, 16, "d_trace", true));
    lgpu::TabuArgs a;
    a.d_start = d_start;
    a.N = N;
    a.B = B;
    a.seed = seed;
    a.first_instance = opts->first_instance;
    a.generation = opts->generation;
    a.max_iter = opts->max_iter;
    a.variant = opts->variant;
    a.d_best = d_best;
    a.d_bestE = d_bestE;
    a.d_steps = d_steps;
    a.d_trace = reinterpret_cast<int4*>(d_trace);
    a.trace_cap = d_trace ? opts->trace_cap : 0;
    const cudaError_t e = lgpu::launch_tabu(a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "tabu kernel launch");
    return ok();
}

int32_t labs_mts_launch(const labs_params* P, uint64_t seed, uint64_t first_instance,
                        int64_t replicas, labs_device_result* d_out, uint32_t* d_glf,
                        labs_stream_t stream) {
    lgpu::MtsArgs a;
    LABS_TRY(make_mts_args(P, seed, first_instance, replicas, &a));
    if (replicas == 0) return ok();
    LABS_TRY(check_dev(d_out, 16, "d_out", false));
    LABS_TRY(check_dev(d_glf, 4, "d_glf", !P->glf));
    a.d_out = d_out;
    a.d_glf = P->glf ? d_glf : nullptr;
    const cudaError_t e = lgpu::launch_mts(a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "mts kernel launch");
    return ok();
}

int64_t labs_mts_state_bytes(int32_t N, int32_t K) {
    if (N < 3 || N > LABS_MAX_N || K < 1 || K > LABS_MAX_K) {
        fail(LABS_EINVAL, "N=%d or K=%d out of range", N, K);
        return -1;
    }
    ok();
    return static_cast<int64_t>(lgpu::resume_state_bytes(N, K));
}

int32_t labs_mts_resume(const labs_params* P, uint64_t seed, uint64_t first_instance, int64_t replicas,
                        void* d_state, int32_t resume, labs_device_result* d_out, uint32_t* d_glf,
                        labs_stream_t stream) {
    lgpu::ResumeArgs ra;
    LABS_TRY(make_mts_args(P, seed, first_instance, replicas, &ra.m));
    if (P->d_trace != nullptr) return fail(LABS_EINVAL, "labs_mts_resume records no trace (d_trace must be NULL)");
    if (replicas == 0) return ok();
    LABS_TRY(check_dev(d_state, 16, "d_state", false));
    LABS_TRY(check_dev(d_out, 16, "d_out", false));
    LABS_TRY(check_dev(d_glf, 4, "d_glf", !P->glf));
    ra.m.d_out = d_out;
    ra.m.d_glf = P->glf ? d_glf : nullptr;
    ra.d_state = static_cast<unsigned char*>(d_state);
    ra.state_bytes = lgpu::resume_state_bytes(P->N, P->K);
    ra.resume = resume != 0 ? 1 : 0;
    const cudaError_t e = lgpu::launch_mts_resume(ra, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "mts resume kernel launch");
    return ok();
}

int32_t labs_mts_run(const labs_params* P, uint64_t seed, uint64_t first_instance,
                     int64_t replicas, labs_result* h_out, labs_stream_t stream) {
    const auto t0 = std::chrono::steady_clock::now();
    lgpu::MtsArgs a;
    LABS_TRY(make_mts_args(P, seed, first_instance, replicas, &a));
    if (replicas == 0) return ok();
    if (h_out == nullptr) return fail(LABS_EINVAL, "h_out is NULL");
    NvtxRange range("labs mts run");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    labs_device_result* d_out = nullptr;
    uint32_t* d_glf = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_out),
                                    sizeof(labs_device_result) * static_cast<size_t>(replicas), s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(LABS_ENOMEM, "result buffer")
                                                                 : cuda_fail(e, "cudaMallocAsync");
    e = cudaMallocAsync(reinterpret_cast<void**>(&d_glf), sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_glf, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        a.d_out = d_out;
        a.d_glf = P->glf ? d_glf : nullptr;
        e = lgpu::launch_mts(a, s);
    }
    std::vector<labs_device_result> host(static_cast<size_t>(replicas));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host.data(), d_out, sizeof(labs_device_result) * host.size(),
                            cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_out, s);
    if (d_glf) cudaFreeAsync(d_glf, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "labs_mts_run");
    if (es != cudaSuccess) return cuda_fail(es, "labs_mts_run synchronize");
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int64_t r = 0; r < replicas; ++r)
        fill_host_result(host[static_cast<size_t>(r)], P->N, first_instance + static_cast<uint64_t>(r),
                         secs, &h_out[r]);
    return ok();
}

int32_t labs_results_decode(const labs_device_result* h_in, int64_t n, int32_t N,
                            uint64_t first_instance, labs_result* h_out) {
    LABS_TRY(check_N(N));
    if (n < 0) return fail(LABS_EINVAL, "labs_results_decode: negative count");
    if (n == 0) return ok();
    if (h_in == nullptr || h_out == nullptr) return fail(LABS_EINVAL, "labs_results_decode: NULL buffer");
    for (int64_t r = 0; r < n; ++r)
        fill_host_result(h_in[r], N, first_instance + static_cast<uint64_t>(r), 0.0, &h_out[r]);
    return ok();
}

}  // extern "C"
