// kernels.h -- launch interface between the C ABI (capi.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "labs.h"

namespace lgpu {

constexpr int kWarpsPerBlock = 4;

struct MtsArgs {
    int32_t N, K;
    uint32_t p_comb_u32, p_mut_u32;
    int32_t replace_policy, target_E;
    int64_t max_generations, max_steps;
    int32_t max_iter, variant;
    uint64_t seed, first_instance;
    int64_t replicas;
    labs_device_result* d_out;
    uint32_t* d_glf;  // nullptr: no global termination flag
    int4* d_trace;    // nullptr: no trace
    int64_t trace_cap;
    size_t smem_per_warp;
};

// Resumable state of one replica (labs_mts_resume): this header, then K * NW
// population words and K energies, the record padded to 16 bytes.  The run
// it belongs to (N, K, variant, seed, instance) is stored and checked.
struct ResumeHeader {
    uint32_t best[2 * LABS_MAX_W];
    int32_t E_best, status;
    int64_t g, steps;
    int32_t N, K, variant;
    uint32_t instance;
    uint64_t seed;
};
static_assert(sizeof(ResumeHeader) == 80, "resume header layout");

inline size_t resume_state_bytes(int N, int K) {
    const size_t nw = 2 * static_cast<size_t>((N + 63) / 64);
    const size_t body = static_cast<size_t>(K) * nw * 4 + static_cast<size_t>(K) * 4;
    return sizeof(ResumeHeader) + ((body + 15) & ~static_cast<size_t>(15));
}

struct ResumeArgs {
    MtsArgs m;
    unsigned char* d_state;  // replicas records of state_bytes each
    size_t state_bytes;
    int32_t resume;          // 0: start from the initial population
};

struct TabuArgs {
    const uint64_t* d_start;
    int32_t N;
    int64_t B;
    uint64_t seed, first_instance;
    uint32_t generation;
    int32_t max_iter, variant;
    uint64_t* d_best;
    int32_t* d_bestE;
    int64_t* d_steps;
    int4* d_trace;
    int64_t trace_cap;
};

struct BatchArgs {
    const labs_instance* inst;     // queue order
    const int32_t* order;          // queue position -> original index
    int64_t n;
    labs_device_result* out;       // original order
    unsigned long long* queue;     // next queue position
    size_t smem_per_warp;
};

// Device record of one serving slot, between quanta.
constexpr int32_t kSlotFresh = 0;      // admitted, population not built yet
constexpr int32_t kSlotSuspended = 1;  // between two generations
constexpr int32_t kSlotDone = 2;
struct ServeState {
    uint32_t best[2 * LABS_MAX_W];
    int32_t E_best, status;
    int64_t g, steps;
    int32_t phase, pad[3];
};

struct ServeArgs {
    const labs_instance* cfg;    // per slot
    ServeState* state;           // per slot
    uint32_t* pop;               // arena: a slot's extent holds K*NW words then K energies
    const int64_t* pop_off;      // per slot: word offset of its extent in the arena
    const int32_t* active;       // slot of each active index
    int32_t n_active;
    int64_t quantum_steps;       // a slot stops at the first generation boundary past this
    uint64_t quantum_ns;         // > 0: ... or past this much device time (%globaltimer)
    labs_device_result* out;     // per active index (finished slots only)
    int32_t* done;               // per active index
    int64_t* quantum_used;       // steps each active slot took in this quantum
    size_t smem_per_warp;
};

size_t mts_smem_per_warp(int N, int K);
cudaError_t launch_skew(const uint64_t* d_seqs, int N, int64_t B, int32_t* d_out, cudaStream_t stream);
// Word count the service's kernels use for N, and one warp's shared memory for (nw, K).
int serve_class_nw(int N);
size_t serve_smem_per_warp(int nw, int K);
// Resident CTAs per SM of the class-nw quantum kernel with wps warps per slot
// (occupancy API); pairs exist for even nw only (serve_pairs_supported).
int serve_pairs_supported(int nw);
cudaError_t serve_blocks_per_sm(int nw, int wps, int warps_per_block, size_t smem_per_warp, int* blocks);
// One quantum of the slots of one word-count class, wps warps per slot (an
// even warps_per_block for wps = 2).
cudaError_t launch_serve_quantum(const ServeArgs& a, int nw, int wps, int warps_per_block, cudaStream_t stream);
// wps: warps per replica (1, or 2 with an even warps_per_block).
cudaError_t batch_prepare(int nwmax, int wps, int warps_per_block, size_t smem_per_warp, int* max_blocks_per_sm);
cudaError_t launch_batch(const BatchArgs& a, int nwmax, int wps, int blocks, int warps_per_block,
                         cudaStream_t stream);
cudaError_t launch_mts(const MtsArgs& a, cudaStream_t stream);
cudaError_t launch_tabu(const TabuArgs& a, cudaStream_t stream);
cudaError_t launch_mts_skew(const MtsArgs& a, cudaStream_t stream);   // mts_skew.cu
cudaError_t launch_mts_resume(const ResumeArgs& a, cudaStream_t stream);  // mts_resume.cu
cudaError_t launch_tabu_skew(const TabuArgs& a, cudaStream_t stream);
cudaError_t launch_energy(const uint64_t* d_seqs, int N, int64_t B, int32_t* d_E, int32_t* d_C,
                          cudaStream_t stream);

}  // namespace lgpu
