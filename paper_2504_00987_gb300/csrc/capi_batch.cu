// capi_batch.cu -- host side of the batched persistent launch (labs.h:
// labs_autotune, labs_batch_*, labs_mts_batch_run).
//
// A batch uploads its instances once, in queue order (longest pair-term
// budget first by default, so the long instances start first and the short
// ones fill in behind them), and captures [reset queue counter, persistent
// kernel] in a CUDA graph that every launch replays.  The autotuner times
// the candidate mappings on a copy of the batch with every budget divided by
// 8 and remembers the winner per batch signature.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "capi_util.h"
#include "kernels.h"
#include "labs.h"

using namespace lcapi;

struct labs_batch {
    int device = 0;
    int64_t n = 0;
    labs_mapping map{};
    int nwmax = 2;
    int blocks = 0;
    size_t smem_per_warp = 0;
    std::vector<labs_instance> h_inst;  // original order
    labs_instance* d_inst = nullptr;    // queue order
    int32_t* d_order = nullptr;
    labs_device_result* d_out = nullptr;
    unsigned long long* d_queue = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int32_t validate_instances(const labs_instance* h, int64_t n) {
    if (n < 0) return fail(LABS_EINVAL, "n < 0");
    if (n > 0 && h == nullptr) return fail(LABS_EINVAL, "instances are NULL");
    if (n > (int64_t{1} << 31) - 1) return fail(LABS_EINVAL, "too many instances");
    for (int64_t i = 0; i < n; ++i) {
        const labs_instance& x = h[i];
        char who[48];
        snprintf(who, sizeof who, "instance %lld", static_cast<long long>(i));
        LABS_TRY(check_run(x.N, x.K, x.replace_policy, x.target_E, x.max_generations, x.max_steps,
                           x.max_iter, x.instance, 1, who));
        LABS_TRY(check_variant(x.variant, x.N, false, who));
    }
    return LABS_OK;
}

// Pair-term budget of an instance: the cost the queue order sorts by.
double instance_cost(const labs_instance& x) {
    const double per_step = static_cast<double>(x.N) * (x.N - 1);
    double steps;
    if (x.max_steps >= 0)
        steps = static_cast<double>(x.max_steps);
    else
        steps = static_cast<double>(x.max_generations) * (x.max_iter >= 0 ? x.max_iter : 1.5 * x.N);
    if (x.max_steps >= 0 && x.max_generations >= 0)
        steps = std::min(steps, static_cast<double>(x.max_generations) *
                                    (x.max_iter >= 0 ? x.max_iter : 1.5 * x.N));
    return steps * per_step;
}

int nwmax_of(const labs_instance* h, int64_t n) {
    int w = 1;
    for (int64_t i = 0; i < n; ++i) w = std::max(w, (h[i].N + 63) / 64);
    return 2 * w;
}

size_t smem_of(const labs_instance* h, int64_t n) {
    size_t s = 16;
    for (int64_t i = 0; i < n; ++i) s = std::max(s, lgpu::mts_smem_per_warp(h[i].N, h[i].K));
    return s;
}

std::vector<int32_t> queue_order(const labs_instance* h, int64_t n, int order) {
    std::vector<int32_t> idx(static_cast<size_t>(n));
    std::iota(idx.begin(), idx.end(), 0);
    if (order == LABS_ORDER_LPT)
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
            return instance_cost(h[a]) > instance_cost(h[b]);
        });
    return idx;
}

int wps_of(const labs_mapping& m) { return m.warps_per_seq == 2 ? 2 : 1; }

int32_t check_mapping(const labs_mapping& m) {
    if (m.warps_per_block != 1 && m.warps_per_block != 2 && m.warps_per_block != 4 &&
        m.warps_per_block != 8)
        return fail(LABS_EINVAL, "warps_per_block must be 1, 2, 4 or 8");
    if (m.warps_per_seq < 0 || m.warps_per_seq > 2)
        return fail(LABS_EINVAL, "warps_per_seq must be 1 (or 0) or 2");
    if (m.warps_per_seq == 2 && m.warps_per_block == 1)
        return fail(LABS_EINVAL, "warps_per_seq = 2 needs warps_per_block 2, 4 or 8");
    if (m.blocks_per_sm < 1 || m.blocks_per_sm > 64) return fail(LABS_EINVAL, "blocks_per_sm outside 1..64");
    if (m.order != LABS_ORDER_LPT && m.order != LABS_ORDER_GIVEN) return fail(LABS_EINVAL, "unknown order");
    return LABS_OK;
}

// Device copies of a batch in queue order (shared by the batch and the tuner).
struct DeviceBatch {
    labs_instance* inst = nullptr;
    int32_t* order = nullptr;
    labs_device_result* out = nullptr;
    unsigned long long* queue = nullptr;
    void release() {
        cudaFree(inst);
        cudaFree(order);
        cudaFree(out);
        cudaFree(queue);
        inst = nullptr;
        order = nullptr;
        out = nullptr;
        queue = nullptr;
    }
};

cudaError_t upload(const std::vector<labs_instance>& h, const std::vector<int32_t>& ord, DeviceBatch* d) {
    const size_t n = h.size();
    std::vector<labs_instance> q(n);
    for (size_t i = 0; i < n; ++i) {
        q[i] = h[static_cast<size_t>(ord[i])];
        q[i].p_mut_u32 = default_p_mut(q[i].N, q[i].p_mut_u32, q[i].variant);
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d->inst), sizeof(labs_instance) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&d->order), sizeof(int32_t) * std::max<size_t>(n, 1));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void**>(&d->out), sizeof(labs_device_result) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&d->queue), sizeof(unsigned long long));
    if (e == cudaSuccess && n)
        e = cudaMemcpy(d->inst, q.data(), sizeof(labs_instance) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n) e = cudaMemcpy(d->order, ord.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
    return e;
}

lgpu::BatchArgs args_of(const DeviceBatch& d, int64_t n, size_t smem_per_warp) {
    lgpu::BatchArgs a;
    a.inst = d.inst;
    a.order = d.order;
    a.n = n;
    a.out = d.out;
    a.queue = d.queue;
    a.smem_per_warp = smem_per_warp;
    return a;
}

std::string signature(const labs_instance* h, int64_t n) {
    // word-count histogram, K range and total cost (to 2 significant digits)
    int64_t hist[4] = {0, 0, 0, 0};
    int kmax = 0;
    double cost = 0;
    for (int64_t i = 0; i < n; ++i) {
        hist[(h[i].N + 63) / 64 - 1]++;
        kmax = std::max(kmax, h[i].K);
        cost += instance_cost(h[i]);
    }
    char buf[160];
    snprintf(buf, sizeof buf, "sm%d n%lld w%lld/%lld/%lld/%lld k%d c%.1e", sm_count(),
             static_cast<long long>(n), static_cast<long long>(hist[0]), static_cast<long long>(hist[1]),
             static_cast<long long>(hist[2]), static_cast<long long>(hist[3]), kmax, cost);
    return buf;
}

std::mutex g_tune_mu;
std::map<std::string, labs_mapping> g_tuned;

}  // namespace

extern "C" {

int32_t labs_autotune(const labs_instance* h_inst, int64_t n, labs_stream_t stream, labs_mapping* out) {
    if (out == nullptr) return fail(LABS_EINVAL, "out is NULL");
    LABS_TRY(validate_instances(h_inst, n));
    NvtxRange range("labs autotune");
    labs_mapping best{4, 1, LABS_ORDER_LPT, 1};
    if (n == 0) {
        *out = best;
        return ok();
    }
    const std::string sig = signature(h_inst, n);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(sig);
        if (it != g_tuned.end()) {
            *out = it->second;
            return ok();
        }
    }
    // Tuning copy: every budget divided by 8 (at least one generation).
    std::vector<labs_instance> scaled(h_inst, h_inst + n);
    for (auto& x : scaled) {
        if (x.max_steps >= 0) x.max_steps = std::max<int64_t>(1, x.max_steps / 8);
        if (x.max_generations >= 0) x.max_generations = std::max<int64_t>(1, x.max_generations / 8);
    }
    const int nwmax = nwmax_of(h_inst, n);
    const size_t spw = smem_of(h_inst, n);
    const std::vector<int32_t> ord = queue_order(scaled.data(), n, LABS_ORDER_LPT);
    DeviceBatch d;
    cudaError_t e = upload(scaled, ord, &d);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const lgpu::BatchArgs a = args_of(d, n, spw);
    const int sms = sm_count();
    float best_ms = 1e30f;
    for (int wps : {1, 2}) {
        bool warmed = false;  // each kernel family gets one untimed launch
        for (int wpb : {1, 2, 4, 8}) {
            if (wpb < wps) continue;
            int maxb = 0;
            if (e == cudaSuccess) e = lgpu::batch_prepare(nwmax, wps, wpb, spw, &maxb);
            if (e != cudaSuccess) break;
            for (int bps : {1, 2, 4, 8, 16}) {
                if (bps > maxb) break;
                // more resident replicas than instances x 2 cannot help
                if (bps > 1 && static_cast<int64_t>(sms) * (bps / 2) * (wpb / wps) >= 2 * n) break;
                for (int rep = warmed ? 0 : 1; rep >= 0 && e == cudaSuccess; --rep) {
                    e = cudaMemsetAsync(d.queue, 0, sizeof(unsigned long long), s);
                    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                    if (e == cudaSuccess) e = lgpu::launch_batch(a, nwmax, wps, sms * bps, wpb, s);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                }
                warmed = true;
                float ms = 0;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = labs_mapping{wpb, bps, LABS_ORDER_LPT, wps};
                }
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    d.release();
    if (e != cudaSuccess) return cuda_fail(e, "labs_autotune");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[sig] = best;
    }
    *out = best;
    return ok();
}

int32_t labs_batch_create(const labs_instance* h_inst, int64_t n, const labs_mapping* mapping,
                          labs_stream_t stream, labs_batch** out) {
    if (out == nullptr) return fail(LABS_EINVAL, "out is NULL");
    *out = nullptr;
    LABS_TRY(validate_instances(h_inst, n));
    labs_mapping m;
    if (mapping != nullptr) {
        m = *mapping;
        LABS_TRY(check_mapping(m));
    } else {
        LABS_TRY(labs_autotune(h_inst, n, stream, &m));
    }
    labs_batch* b = new (std::nothrow) labs_batch();
    if (b == nullptr) return fail(LABS_ENOMEM, "batch object");
    cudaGetDevice(&b->device);
    b->n = n;
    b->map = m;
    b->h_inst.assign(h_inst, h_inst + n);
    b->nwmax = nwmax_of(h_inst, n);
    b->smem_per_warp = smem_of(h_inst, n);
    const std::vector<int32_t> ord = queue_order(h_inst, n, m.order);
    DeviceBatch d;
    cudaError_t e = upload(b->h_inst, ord, &d);
    b->d_inst = d.inst;
    b->d_order = d.order;
    b->d_out = d.out;
    b->d_queue = d.queue;
    int maxb = 0;
    if (e == cudaSuccess) e = lgpu::batch_prepare(b->nwmax, wps_of(m), m.warps_per_block, b->smem_per_warp, &maxb);
    if (e == cudaSuccess && maxb < 1) {
        labs_batch_destroy(b);
        return fail(LABS_EINVAL, "mapping does not fit on an SM (warps_per_block=%d)", m.warps_per_block);
    }
    b->blocks = sm_count() * std::min(m.blocks_per_sm, std::max(maxb, 1));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->cap);
        if (le == cudaSuccess)
            le = lgpu::launch_batch(args_of(d, n, b->smem_per_warp), b->nwmax, wps_of(m), b->blocks,
                                    m.warps_per_block, b->cap);
        e = cudaStreamEndCapture(b->cap, &b->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        labs_batch_destroy(b);
        return cuda_fail(e, "labs_batch_create");
    }
    *out = b;
    return ok();
}

int32_t labs_batch_launch(labs_batch* b, labs_stream_t stream) {
    if (b == nullptr) return fail(LABS_EINVAL, "batch is NULL");
    if (b->n == 0) return ok();
    NvtxRange range("labs batch launch");
    const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return ok();
}

int32_t labs_batch_device_results(const labs_batch* b, labs_device_result** d_out) {
    if (b == nullptr || d_out == nullptr) return fail(LABS_EINVAL, "NULL argument");
    *d_out = b->d_out;
    return ok();
}

int32_t labs_batch_get_mapping(const labs_batch* b, labs_mapping* out) {
    if (b == nullptr || out == nullptr) return fail(LABS_EINVAL, "NULL argument");
    *out = b->map;
    return ok();
}

int32_t labs_batch_results(labs_batch* b, labs_result* h_out, labs_stream_t stream) {
    if (b == nullptr) return fail(LABS_EINVAL, "batch is NULL");
    if (b->n == 0) return ok();
    if (h_out == nullptr) return fail(LABS_EINVAL, "h_out is NULL");
    std::vector<labs_device_result> host(static_cast<size_t>(b->n));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(host.data(), b->d_out, sizeof(labs_device_result) * host.size(),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "labs_batch_results");
    for (int64_t i = 0; i < b->n; ++i)
        fill_host_result(host[static_cast<size_t>(i)], b->h_inst[static_cast<size_t>(i)].N,
                         b->h_inst[static_cast<size_t>(i)].instance, 0.0, &h_out[i]);
    return ok();
}

int32_t labs_batch_destroy(labs_batch* b) {
    if (b == nullptr) return ok();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_inst);
    cudaFree(b->d_order);
    cudaFree(b->d_out);
    cudaFree(b->d_queue);
    delete b;
    return ok();
}

int32_t labs_mts_batch_run(const labs_instance* h_inst, int64_t n, const labs_mapping* mapping,
                           labs_result* h_out, labs_stream_t stream) {
    const auto t0 = std::chrono::steady_clock::now();
    labs_batch* b = nullptr;
    LABS_TRY(labs_batch_create(h_inst, n, mapping, stream, &b));
    int32_t rc = labs_batch_launch(b, stream);
    if (rc == LABS_OK) rc = labs_batch_results(b, h_out, stream);
    labs_batch_destroy(b);
    if (rc != LABS_OK) return rc;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int64_t i = 0; i < n; ++i) h_out[i].seconds = secs;
    return ok();
}

}  // extern "C"
