// capi_serve.cu -- host side of the solve service (labs_serve_* in labs.h).
//
// One scheduler thread per server runs the loop
//   admit pending requests (FIFO) while a slot is free, the request's word
//   class still fits in one resident wave of the GPU (shared memory and
//   registers, from the occupancy API) and the HBM arena has a free extent
//   of the request's footprint -> upload the new slots' records and the
//   active list -> launch one quantum: one kernel per word-count class, each
//   on its own stream and with its class's shared memory per warp -> wait
//   for it (bounded) -> harvest finished slots, free their slots and
//   extents.
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
#include <map>
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
// admission rules that held a request back (each counted once per request)
enum HeldBy { kHeldSlots = 1, kHeldHbm = 2, kHeldSmem = 4 };

constexpr int kClasses = 6;
constexpr int kClassNw[kClasses] = {2, 3, 4, 5, 6, 8};

int class_of(int N) {
    const int nw = lgpu::serve_class_nw(N);
    for (int c = 0; c < kClasses; ++c)
        if (kClassNw[c] == nw) return c;
    return kClasses - 1;
}

struct Ticket {
    labs_request req{};
    int state = kPending;
    int32_t slot = -1;
    int cls = -1;
    int held = 0;
    int64_t off = -1;  // bytes into the arena
    bool cancel_requested = false;
    labs_result res{};
    Clock::time_point t_submit;
};

// Arena bytes of a request: its population (K x nw words) and energies (K),
// nw the word count its kernel uses, padded to 16.
int64_t footprint(const labs_request& r) {
    const int64_t nw = lgpu::serve_class_nw(r.N);
    return (static_cast<int64_t>(r.K) * (nw + 1) * 4 + 15) & ~int64_t{15};
}

// First-fit allocator of extents of the device arena (byte offsets, 16-aligned).
struct Arena {
    std::map<int64_t, int64_t> free_ext;  // offset -> length
    int64_t size = 0, used = 0;
    void init(int64_t n) {
        free_ext.clear();
        free_ext[0] = n;
        size = n;
        used = 0;
    }
    int64_t alloc(int64_t n) {
        for (auto it = free_ext.begin(); it != free_ext.end(); ++it) {
            if (it->second < n) continue;
            const int64_t off = it->first, len = it->second;
            free_ext.erase(it);
            if (len > n) free_ext[off + n] = len - n;
            used += n;
            return off;
        }
        return -1;
    }
    void release(int64_t off, int64_t n) {
        used -= n;
        auto it = free_ext.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_ext.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_ext.erase(nx);
        }
        if (it != free_ext.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_ext.erase(it);
            }
        }
    }
};

}  // namespace

struct labs_server {
    labs_serve_opts opts{};
    int device = 0;
    // per word-count class: shared memory per warp, warps resident in one wave
    // (one warp per slot; two warps per slot, 0 where pairs do not apply), active slots
    size_t cls_smem[kClasses] = {};
    int64_t cls_cap[kClasses] = {};
    int64_t cls_cap2[kClasses] = {};
    int64_t cls_active[kClasses] = {};
    int pair_wpb = 2;  // CTA size of the two-warps-per-slot launches
    Arena arena;

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
    labs_serve_stats stats{};
    std::thread th;

    cudaStream_t stream = nullptr;
    cudaStream_t cls_stream[kClasses] = {};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_fork = nullptr;
    cudaEvent_t ev_join[kClasses] = {};
    labs_instance* d_cfg = nullptr;
    int64_t* d_off = nullptr;
    lgpu::ServeState* d_state = nullptr;
    uint32_t* d_pop = nullptr;
    int32_t* d_active = nullptr;
    labs_device_result* d_out = nullptr;
    int32_t* d_done = nullptr;
    int64_t* d_used = nullptr;
    // pinned staging
    labs_instance* h_cfg = nullptr;
    int64_t* h_off = nullptr;
    lgpu::ServeState* h_state = nullptr;
    int32_t* h_active = nullptr;
    labs_device_result* h_out = nullptr;
    int32_t* h_done = nullptr;
    int64_t* h_used = nullptr;
};

namespace {

// Fraction of one resident wave the active slots take, with `extra` more of class c.
double wave_fraction(const labs_server* s, int c, int64_t extra) {
    double f = 0.0;
    for (int k = 0; k < kClasses; ++k) {
        const int64_t n = s->cls_active[k] + (k == c ? extra : 0);
        if (n > 0) f += static_cast<double>(n) / static_cast<double>(s->cls_cap[k]);
    }
    return f;
}

// True if every active slot of an even word class fits one resident wave on two warps
// (and the others on one): the quantum then runs those slots on warp pairs.
bool use_pairs(const labs_server* s) {
    if (s->opts.warps_per_request != 2) return false;
    double f = 0.0;
    for (int k = 0; k < kClasses; ++k) {
        const int64_t n = s->cls_active[k];
        if (n == 0) continue;
        f += s->cls_cap2[k] > 0 ? 2.0 * static_cast<double>(n) / static_cast<double>(s->cls_cap2[k])
                                : static_cast<double>(n) / static_cast<double>(s->cls_cap[k]);
    }
    return f <= 1.0 + 1e-9;
}

void hold(labs_server* s, Ticket& t, int rule) {
    if (t.held & rule) return;
    t.held |= rule;
    if (rule == kHeldSlots) s->stats.deferred_slots++;
    if (rule == kHeldHbm) s->stats.deferred_hbm++;
    if (rule == kHeldSmem) s->stats.deferred_smem++;
}

// A running request leaves: its slot, arena extent and class share are freed.
void release_slot(labs_server* s, Ticket& t) {
    s->slot_ticket[static_cast<size_t>(t.slot)] = 0;
    s->free_slots.push_back(t.slot);
    s->arena.release(t.off, footprint(t.req));
    s->cls_active[t.cls]--;
    s->stats.running--;
    s->stats.arena_used_bytes = s->arena.used;
}

void free_server(labs_server* s) {
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (int c = 0; c < kClasses; ++c)
        if (s->cls_stream[c]) cudaStreamSynchronize(s->cls_stream[c]);
    cudaFree(s->d_cfg);
    cudaFree(s->d_off);
    cudaFreeHost(s->h_off);
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
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    for (int c = 0; c < kClasses; ++c) {
        if (s->ev_join[c]) cudaEventDestroy(s->ev_join[c]);
        if (s->cls_stream[c]) cudaStreamDestroy(s->cls_stream[c]);
    }
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
    std::vector<int32_t> by_class[kClasses];
    bool pairs = false;
    for (;;) {
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
                    release_slot(s, t);
                    s->stats.canceled++;
                }
            }
            // admission, FIFO: a free slot, room in one resident wave for the
            // request's class (always, if nothing runs), a free arena extent
            fresh.clear();
            while (!s->pending.empty()) {
                const uint64_t id = s->pending.front();
                Ticket& t = s->tickets[id];
                if (s->free_slots.empty()) {
                    hold(s, t, kHeldSlots);
                    break;
                }
                const int c = class_of(t.req.N);
                if (s->stats.running > 0 && wave_fraction(s, c, 1) > 1.0 + 1e-9) {
                    hold(s, t, kHeldSmem);
                    break;
                }
                const int64_t off = s->arena.alloc(footprint(t.req));
                if (off < 0) {
                    hold(s, t, kHeldHbm);
                    break;
                }
                s->pending.pop_front();
                const int32_t slot = s->free_slots.back();
                s->free_slots.pop_back();
                s->slot_ticket[static_cast<size_t>(slot)] = id;
                t.state = kRunning;
                t.slot = slot;
                t.cls = c;
                t.off = off;
                s->cls_active[c]++;
                s->stats.running++;
                s->stats.pending--;
                s->stats.arena_used_bytes = s->arena.used;
                s->h_cfg[slot] = t.req;
                s->h_cfg[slot].p_mut_u32 = default_p_mut(t.req.N, t.req.p_mut_u32, t.req.variant);
                s->h_off[slot] = off / 4;
                fresh.push_back(slot);
            }
            // the active slots, grouped by class (one launch per class)
            for (auto& v : by_class) v.clear();
            for (size_t slot = 0; slot < s->slot_ticket.size(); ++slot)
                if (s->slot_ticket[slot] != 0)
                    by_class[s->tickets[s->slot_ticket[slot]].cls].push_back(static_cast<int32_t>(slot));
            pairs = use_pairs(s);
            if (pairs) s->stats.pair_quanta++;
        }
        active.clear();
        int seg_off[kClasses], seg_len[kClasses];
        for (int c = 0; c < kClasses; ++c) {
            seg_off[c] = static_cast<int>(active.size());
            seg_len[c] = static_cast<int>(by_class[c].size());
            active.insert(active.end(), by_class[c].begin(), by_class[c].end());
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
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->d_off + slot, s->h_off + slot, sizeof(int64_t), cudaMemcpyHostToDevice,
                                    s->stream);
            if (e != cudaSuccess) break;
        }
        const int n = static_cast<int>(active.size());
        std::copy(active.begin(), active.end(), s->h_active);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->d_active, s->h_active, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev0, s->stream);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_fork, s->stream);
        // one launch per class, each on its own stream, joined back into the main one
        for (int c = 0; c < kClasses && e == cudaSuccess; ++c) {
            if (seg_len[c] == 0) continue;
            lgpu::ServeArgs a;
            a.cfg = s->d_cfg;
            a.state = s->d_state;
            a.pop = s->d_pop;
            a.pop_off = s->d_off;
            a.active = s->d_active + seg_off[c];
            a.n_active = seg_len[c];
            a.quantum_steps = s->opts.quantum_steps;
            a.quantum_ns = static_cast<uint64_t>(s->opts.quantum_us) * 1000u;
            a.out = s->d_out + seg_off[c];
            a.done = s->d_done + seg_off[c];
            a.quantum_used = s->d_used + seg_off[c];
            a.smem_per_warp = s->cls_smem[c];
            const bool pair = pairs && s->cls_cap2[c] > 0;
            e = cudaStreamWaitEvent(s->cls_stream[c], s->ev_fork, 0);
            if (e == cudaSuccess)
                e = lgpu::launch_serve_quantum(a, kClassNw[c], pair ? 2 : 1,
                                               pair ? s->pair_wpb : s->opts.warps_per_block, s->cls_stream[c]);
            if (e == cudaSuccess) e = cudaEventRecord(s->ev_join[c], s->cls_stream[c]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_join[c], 0);
        }
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
            release_slot(s, t);
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
    const int top = class_of(o->max_N);
    if (lgpu::serve_smem_per_warp(kClassNw[top], o->max_K) * o->warps_per_block > 227u * 1024u) {
        fail(LABS_EINVAL, "max_N/max_K populations of one block exceed shared memory");
        return nullptr;
    }
    if (o->warps_per_request < 0 || o->warps_per_request > 2) {
        fail(LABS_EINVAL, "warps_per_request must be 0, 1 or 2");
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
    s->pair_wpb = std::max(2, o->warps_per_block);
    cudaGetDevice(&s->device);
    // the arena: hbm_budget_bytes, or room for max_slots requests of (max_N, max_K)
    labs_request biggest{};
    biggest.N = o->max_N;
    biggest.K = o->max_K;
    const int64_t fp_max = footprint(biggest);
    const int64_t arena_bytes = o->hbm_budget_bytes > 0 ? (o->hbm_budget_bytes & ~int64_t{15})
                                                        : fp_max * static_cast<int64_t>(o->max_slots);
    if (arena_bytes < fp_max) {
        fail(LABS_EINVAL, "hbm_budget_bytes=%lld holds no request of max_N=%d, max_K=%d (%lld bytes)",
             static_cast<long long>(o->hbm_budget_bytes), o->max_N, o->max_K, static_cast<long long>(fp_max));
        delete s;
        return nullptr;
    }
    s->arena.init(arena_bytes);
    s->stats.arena_bytes = arena_bytes;
    const size_t S = static_cast<size_t>(o->max_slots);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    // one wave per class: warps of its kernel resident at once with its shared memory
    for (int c = 0; c <= top && e == cudaSuccess; ++c) {
        s->cls_smem[c] = lgpu::serve_smem_per_warp(kClassNw[c], o->max_K);
        int blocks = 0;
        e = lgpu::serve_blocks_per_sm(kClassNw[c], 1, o->warps_per_block, s->cls_smem[c], &blocks);
        if (e == cudaSuccess && blocks < 1) {
            fail(LABS_EINVAL, "the quantum kernel for %d-word sequences does not fit on an SM", kClassNw[c]);
            free_server(s);
            return nullptr;
        }
        s->cls_cap[c] = static_cast<int64_t>(blocks) * o->warps_per_block * sm_count();
        if (e == cudaSuccess && o->warps_per_request == 2 && lgpu::serve_pairs_supported(kClassNw[c])) {
            int b2 = 0;
            e = lgpu::serve_blocks_per_sm(kClassNw[c], 2, s->pair_wpb, s->cls_smem[c], &b2);
            s->cls_cap2[c] = static_cast<int64_t>(b2) * s->pair_wpb * sm_count();
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cls_stream[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_off), sizeof(int64_t) * S);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s->h_off), sizeof(int64_t) * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_cfg), sizeof(labs_instance) * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_state), sizeof(lgpu::ServeState) * S);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->d_pop), static_cast<size_t>(arena_bytes));
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
