// capi_serve.cu -- host side of the solve service (labs_serve_* in labs.h).
//
// One scheduler thread per server runs the loop
//   admit pending requests into free slots (FIFO; a free slot, the HBM
//   budget and the quantum kernel's shared memory must all have room) ->
//   upload the new slots' records and the active list -> launch one quantum
//   -> wait for it (bounded) -> harvest finished slots, free them.
// Submitting, polling and cancelling only touch host state under the
// server's mutex, so they never wait for the GPU.  Every wait is bounded:
// the scheduler waits for new work with a timeout and for a quantum up to
// quantum_timeout_ms, after which the server stops with LABS_ETIMEOUT and
// every call reports it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "capi_util.h"
#include "kernels.h"
#include "labs.h"

using namespace lcapi;
using Clock = std::chrono::steady_clock;

namespace {

enum TicketState { kPending = 0, kRunning = 1, kDone = 2, kCanceled = 3 };

struct Ticket {
    labs_request req{};
    int state = kPending;
    int32_t slot = -1;
    bool cancel_requested = false;
    labs_result res{};
    Clock::time_point t_submit;
};

int64_t footprint(const labs_request& r) {
    const int64_t nw = 2 * ((r.N + 63) / 64);
    return static_cast<int64_t>(r.K) * nw * 4 + static_cast<int64_t>(r.K) * 4;
}

}  // namespace

struct labs_server {
    labs_serve_opts opts{};
    int device = 0;
    int nwmax = 2;
    size_t pop_stride_words = 0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::vector<int32_t> free_slots;
    std::vector<uint64_t> slot_ticket;  // 0: free
    uint64_t next_ticket = 1;
    bool stop = false;
    int32_t failed = LABS_OK;
    std::string fail_msg;
    int64_t resident_bytes = 0;
    labs_serve_stats stats{};
    std::thread th;

    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    labs_instance* d_cfg = nullptr;
    lgpu::ServeState* d_state = nullptr;
    uint32_t* d_pop = nullptr;
    int32_t* d_active = nullptr;
    labs_device_result* d_out = nullptr;
    int32_t* d_done = nullptr;
    int64_t* d_used = nullptr;
    // pinned staging
    labs_instance* h_cfg = nullptr;
    lgpu::ServeState* h_state = nullptr;
    int32_t* h_active = nullptr;
    labs_device_result* h_out = nullptr;
    int32_t* h_done = nullptr;
    int64_t* h_used = nullptr;
};

namespace {

void free_server(labs_server* s) {
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->d_cfg);
    cudaFree(s->d_state);
    cudaFree(s->d_pop);
    cudaFree(s->d_active);
    cudaFree(s->d_out);
    cudaFree(s->d_done);
    cudaFree(s->d_used);
    cudaFreeHost(s->h_cfg);
    cudaFreeHost(s->h_state);
    cudaFreeHost(s->h_active);
    cudaFreeHost(s->h_out);
    cudaFreeHost(s->h_done);
    cudaFreeHost(s->h_used);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

void set_failed(labs_server* s, int32_t code, const std::string& msg) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed == LABS_OK) {
        s->failed = code;
        s->fail_msg = msg;
        s->stats.failed = code;
    }
    s->cv.notify_all();
}

// Waits for ev1 with a deadline; cudaErrorNotReady until then.
cudaError_t wait_bounded(labs_server* s, int64_t timeout_ms) {
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        const cudaError_t e = cudaEventQuery(s->ev1);
        if (e != cudaErrorNotReady) return e;
        if (Clock::now() > deadline) return cudaErrorNotReady;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

void scheduler(labs_server* s) {
    cudaSetDevice(s->device);
    const int64_t timeout_ms = s->opts.quantum_timeout_ms > 0 ? s->opts.quantum_timeout_ms : 60000;
    std::vector<int32_t> fresh;
    std::vector<int32_t> active;
    for (;;) {
        size_t smem_per_warp = 16;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::milliseconds(20), [&] {
                return s->stop || !s->pending.empty() || s->stats.running > 0;
            });
            if (s->stop || s->failed != LABS_OK) return;
            // cancelled running requests leave their slots at this boundary
            for (size_t slot = 0; slot < s->slot_ticket.size(); ++slot) {
                const uint64_t id = s->slot_ticket[slot];
                if (id == 0) continue;
                Ticket& t = s->tickets[id];
                if (t.cancel_requested) {
                    t.state = kCanceled;
                    s->slot_ticket[slot] = 0;
                    s->free_slots.push_back(static_cast<int32_t>(slot));
                    s->resident_bytes -= footprint(t.req);
                    s->stats.running--;
                    s->stats.canceled++;
                }
            }
            // admission: FIFO while a slot, the HBM budget and shared memory have room
            fresh.clear();
            while (!s->pending.empty() && !s->free_slots.empty()) {
                const uint64_t id = s->pending.front();
                Ticket& t = s->tickets[id];
                const int64_t fp = footprint(t.req);
                if (s->opts.hbm_budget_bytes > 0 && s->resident_bytes + fp > s->opts.hbm_budget_bytes &&
                    s->stats.running > 0)
                    break;
                s->pending.pop_front();
                const int32_t slot = s->free_slots.back();
                s->free_slots.pop_back();
                s->slot_ticket[static_cast<size_t>(slot)] = id;
                t.state = kRunning;
                t.slot = slot;
                s->resident_bytes += fp;
                s->stats.running++;
                s->stats.pending--;
                s->h_cfg[slot] = t.req;
                s->h_cfg[slot].p_mut_u32 = default_p_mut(t.req.N, t.req.p_mut_u32, t.req.variant);
                fresh.push_back(slot);
            }
            active.clear();
            for (size_t slot = 0; slot < s->slot_ticket.size(); ++slot)
                if (s->slot_ticket[slot] != 0) {
                    active.push_back(static_cast<int32_t>(slot));
                    const labs_request& r = s->tickets[s->slot_ticket[slot]].req;
                    smem_per_warp = std::max(smem_per_warp, lgpu::mts_smem_per_warp(r.N, r.K));
                }
        }
        if (active.empty()) continue;
        NvtxRange range("labs serve quantum");
        // upload new slots and the active list
        cudaError_t e = cudaSuccess;
        for (int32_t slot : fresh) {
            memset(&s->h_state[slot], 0, sizeof(lgpu::ServeState));
            s->h_state[slot].phase = lgpu::kSlotFresh;
            e = cudaMemcpyAsync(s->d_cfg + slot, s->h_cfg + slot, sizeof(labs_instance),
                                cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->d_state + slot, s->h_state + slot, sizeof(lgpu::ServeState),
                                    cudaMemcpyHostToDevice, s->stream);
            if (e != cudaSuccess) break;
        }
        const int n = static_cast<int>(active.size());
        std::copy(active.begin(), active.end(), s->h_active);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_active, s->h_active, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s->stream);
        lgpu::ServeArgs a;
        a.cfg = s->d_cfg;
        a.state = s->d_state;
        a.pop = s->d_pop;
        a.pop_stride_words = s->pop_stride_words;
        a.active = s->d_active;
        a.n_active = n;
        a.quantum_steps = s->opts.quantum_steps;
        a.quantum_ns = static_cast<uint64_t>(s->opts.quantum_us) * 1000u;
        a.out = s->d_out;
        a.done = s->d_done;
        a.quantum_used = s->d_used;
        a.smem_per_warp = (smem_per_warp + 15) & ~static_cast<size_t>(15);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev0, s->stream);
        if (e == cudaSuccess) e = lgpu::launch_serve_quantum(a, s->nwmax, s->opts.warps_per_block, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->h_done, s->d_done, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->h_used, s->d_used, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->h_out, s->d_out, sizeof(labs_device_result) * n, cudaMemcpyDeviceToHost,
                                s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev1, s->stream);
        if (e == cudaSuccess) {
            e = wait_bounded(s, timeout_ms);
            if (e == cudaErrorNotReady) {
                set_failed(s, LABS_ETIMEOUT, "quantum did not finish within quantum_timeout_ms");
                return;
            }
        }
        if (e != cudaSuccess) {
            set_failed(s, LABS_ECUDA, std::string("serve quantum: ") + cudaGetErrorString(e));
            return;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, s->ev0, s->ev1);
        // harvest
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.quanta++;
        s->stats.gpu_seconds += ms * 1e-3;
        const auto now = Clock::now();
        for (int i = 0; i < n; ++i) {
            const int32_t slot = active[static_cast<size_t>(i)];
            const uint64_t id = s->slot_ticket[static_cast<size_t>(slot)];
            Ticket& t = s->tickets[id];
            s->stats.flip_evals += s->h_used[i] * t.req.N;
            if (!s->h_done[i]) continue;
            const double secs = std::chrono::duration<double>(now - t.t_submit).count();
            fill_host_result(s->h_out[i], t.req.N, t.req.instance, secs, &t.res);
            t.state = t.cancel_requested ? kCanceled : kDone;
            if (t.cancel_requested) s->stats.canceled++;
            else s->stats.completed++;
            s->slot_ticket[static_cast<size_t>(slot)] = 0;
            s->free_slots.push_back(slot);
            s->resident_bytes -= footprint(t.req);
            s->stats.running--;
        }
    }
}

}  // namespace

extern "C" {

labs_server* labs_serve_create(const labs_serve_opts* o) {
    if (o == nullptr) {
        fail(LABS_EINVAL, "opts is NULL");
        return nullptr;
    }
    if (o->max_slots < 1 || o->max_slots > (1 << 20)) {
        fail(LABS_EINVAL, "max_slots outside 1..2^20");
        return nullptr;
    }
    if (check_N(o->max_N) != LABS_OK) return nullptr;
    if (o->max_K < 1 || o->max_K > LABS_MAX_K) {
        fail(LABS_EINVAL, "max_K outside 1..%d", LABS_MAX_K);
        return nullptr;
    }
    if (o->warps_per_block != 1 && o->warps_per_block != 2 && o->warps_per_block != 4 &&
        o->warps_per_block != 8) {
        fail(LABS_EINVAL, "warps_per_block must be 1, 2, 4 or 8");
        return nullptr;
    }
    if (lgpu::mts_smem_per_warp(o->max_N, o->max_K) * o->warps_per_block > 227u * 1024u) {
        fail(LABS_EINVAL, "max_N/max_K populations of one block exceed shared memory");
        return nullptr;
    }
    if (o->quantum_steps < 1 || o->queue_capacity < 0 || o->hbm_budget_bytes < 0 ||
        o->quantum_timeout_ms < 0 || o->quantum_us < 0 || o->quantum_us > (int64_t{1} << 40)) {
        fail(LABS_EINVAL, "quantum_steps >= 1, queue_capacity/hbm_budget/timeout/quantum_us >= 0");
        return nullptr;
    }
    labs_server* s = new (std::nothrow) labs_server();
    if (s == nullptr) {
        fail(LABS_ENOMEM, "server object");
        return nullptr;
    }
    s->opts = *o;
    cudaGetDevice(&s->device);
    const int nw = 2 * ((o->max_N + 63) / 64);
    s->nwmax = nw;
    s->pop_stride_words = static_cast<size_t>(o->max_K) * nw + static_cast<size_t>(o->max_K);
    const size_t S = static_cast<size_t>(o->max_slots);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev1);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_cfg), sizeof(labs_instance) * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_state), sizeof(lgpu::ServeState) * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_pop), sizeof(uint32_t) * s->pop_stride_words * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_active), sizeof(int32_t) * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_out), sizeof(labs_device_result) * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_done), sizeof(int32_t) * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_used), sizeof(int64_t) * S);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s->h_cfg), sizeof(labs_instance) * S);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s->h_state), sizeof(lgpu::ServeState) * S);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s->h_active), sizeof(int32_t) * S);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s->h_out), sizeof(labs_device_result) * S);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s->h_done), sizeof(int32_t) * S);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s->h_used), sizeof(int64_t) * S);
    if (e != cudaSuccess) {
        cuda_fail(e, "labs_serve_create");
        free_server(s);
        return nullptr;
    }
    s->slot_ticket.assign(S, 0);
    s->free_slots.reserve(S);
    for (size_t i = S; i-- > 0;) s->free_slots.push_back(static_cast<int32_t>(i));
    try {
        s->th = std::thread(scheduler, s);
    } catch (...) {
        fail(LABS_ENOMEM, "scheduler thread");
        free_server(s);
        return nullptr;
    }
    ok();
    return s;
}

int32_t labs_serve_submit(labs_server* s, const labs_request* req, uint64_t* ticket) {
    if (s == nullptr || req == nullptr || ticket == nullptr) return fail(LABS_EINVAL, "NULL argument");
    LABS_TRY(check_run(req->N, req->K, req->replace_policy, req->target_E, req->max_generations,
                       req->max_steps, req->max_iter, req->instance, 1, "request"));
    LABS_TRY(check_variant(req->variant, req->N, false, "request"));
    if (req->N > s->opts.max_N || req->K > s->opts.max_K)
        return fail(LABS_EINVAL, "request N=%d K=%d beyond the server's max_N=%d max_K=%d", req->N, req->K,
                    s->opts.max_N, s->opts.max_K);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed != LABS_OK) return fail(s->failed, "server failed: %s", s->fail_msg.c_str());
    if (static_cast<int64_t>(s->pending.size()) >= s->opts.queue_capacity)
        return fail(LABS_EBUSY, "request queue full (%lld pending)", static_cast<long long>(s->pending.size()));
    const uint64_t id = s->next_ticket++;
    Ticket& t = s->tickets[id];
    t.req = *req;
    t.t_submit = Clock::now();
    s->pending.push_back(id);
    s->stats.submitted++;
    s->stats.pending++;
    *ticket = id;
    s->cv.notify_all();
    return ok();
}

int32_t labs_serve_poll(labs_server* s, uint64_t ticket, labs_result* out) {
    if (s == nullptr) return fail(LABS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(LABS_ENOTFOUND, "unknown ticket %llu", static_cast<unsigned long long>(ticket));
    Ticket& t = it->second;
    if (t.state == kDone) {
        if (out) *out = t.res;
        s->tickets.erase(it);
        return ok();
    }
    if (t.state == kCanceled) {
        s->tickets.erase(it);
        return fail(LABS_ECANCELED, "ticket %llu was cancelled", static_cast<unsigned long long>(ticket));
    }
    if (s->failed != LABS_OK) return fail(s->failed, "server failed: %s", s->fail_msg.c_str());
    return fail(LABS_ENOTREADY, "ticket %llu not finished", static_cast<unsigned long long>(ticket));
}

int32_t labs_serve_cancel(labs_server* s, uint64_t ticket) {
    if (s == nullptr) return fail(LABS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(LABS_ENOTFOUND, "unknown ticket %llu", static_cast<unsigned long long>(ticket));
    Ticket& t = it->second;
    if (t.state == kPending) {
        s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), ticket), s->pending.end());
        t.state = kCanceled;
        s->stats.pending--;
        s->stats.canceled++;
    } else if (t.state == kRunning) {
        t.cancel_requested = true;  // leaves the GPU at the next quantum boundary
    }
    return ok();
}

int32_t labs_serve_stats_get(labs_server* s, labs_serve_stats* out) {
    if (s == nullptr || out == nullptr) return fail(LABS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return ok();
}

int32_t labs_serve_destroy(labs_server* s) {
    if (s == nullptr) return ok();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    free_server(s);
    return ok();
}

}  // extern "C"
