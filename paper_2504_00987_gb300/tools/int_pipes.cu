// int_pipes.cu -- measures, on the current GPU, the throughput (lane
// operations per clock per SM, many warps, independent chains) and the
// dependent-chain latency (cycles, one warp) of the integer instruction
// classes the tabu step is made of.  These rates bound the neighbour
// scoring, which runs on the integer ALU pipes, not on tensor cores or DRAM.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

template <int OP>
__global__ void throughput(uint32_t* out, int iters, uint32_t seed) {
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 7u + i + seed;
    const uint32_t b = seed * 3u + 1u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == 0) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
            if (OP == 1) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[i]) : "r"(b), "r"(it));
            if (OP == 2) asm volatile("popc.b32 %0, %0;" : "+r"(a[i]));
            if (OP == 3) a[i] = __funnelshift_r(a[i], b, it);
            if (OP == 4) a[i] = a[i] * 0x9E3779B9u + b;
            if (OP == 5) a[i] = __shfl_xor_sync(0xFFFFFFFFu, a[i], 1);
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
__global__ void latency(uint32_t* out, long long* cyc, uint32_t seed) {
    uint32_t a = threadIdx.x + seed;
    const uint32_t b = seed * 7u + 3u;
    const long long t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < 256; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == 0) asm volatile("add.u32 %0, %0, %1;" : "+r"(a) : "r"(b));
            if (OP == 1) asm volatile("lop3.b32 %0, %0, %1, %1, 0x96;" : "+r"(a) : "r"(b));
            if (OP == 2) asm volatile("popc.b32 %0, %0;" : "+r"(a));
            if (OP == 3) a = __funnelshift_r(a, b, a);
            if (OP == 4) asm volatile("mad.lo.u32 %0, %0, %1, %1;" : "+r"(a) : "r"(b));
            if (OP == 5) a = __shfl_xor_sync(0xFFFFFFFFu, a, 1);
            if (OP == 6) a = __ballot_sync(0xFFFFFFFFu, a & 1u);
            if (OP == 7) a = __reduce_min_sync(0xFFFFFFFFu, a);
        }
    }
    const long long t1 = clock64();
    out[threadIdx.x] = a;
    if (threadIdx.x == 0) *cyc = t1 - t0;
}

template <int OP>
static void run_tp(const char* name, uint32_t* out, int sms, int clk_khz) {
    const int blocks = sms * 8, threads = 256, iters = 4096;
    throughput<OP><<<blocks, threads>>>(out, 16, 1);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    throughput<OP><<<blocks, threads>>>(out, iters, 1);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double ops = static_cast<double>(blocks) * threads * iters * 8;
    printf("throughput %-6s %7.1f lane-ops/clk/SM\n", name, ops / (ms * 1e-3) / (sms * clk_khz * 1e3));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

template <int OP>
static void run_lat(const char* name, uint32_t* out, long long* cyc) {
    latency<OP><<<1, 32>>>(out, cyc, 1);
    latency<OP><<<1, 32>>>(out, cyc, 1);
    long long h = 0;
    cudaMemcpy(&h, cyc, sizeof h, cudaMemcpyDeviceToHost);
    printf("latency    %-6s %7.2f cycles\n", name, h / 2048.0);
}

int main() {
    int dev = 0, sms = 0, clk = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    uint32_t* out = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&out, static_cast<size_t>(sms) * 8 * 256 * 4) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(long long)) != cudaSuccess) {
        printf("allocation failed\n");
        return 1;
    }
    printf("SMs %d, max SM clock %.0f MHz\n", sms, clk / 1e3);
    run_tp<0>("IADD", out, sms, clk);
    run_tp<1>("LOP3", out, sms, clk);
    run_tp<2>("POPC", out, sms, clk);
    run_tp<3>("SHF", out, sms, clk);
    run_tp<4>("IMAD", out, sms, clk);
    run_tp<5>("SHFL", out, sms, clk);
    run_lat<0>("IADD", out, cyc);
    run_lat<1>("LOP3", out, cyc);
    run_lat<2>("POPC", out, cyc);
    run_lat<3>("SHF", out, cyc);
    run_lat<4>("IMAD", out, cyc);
    run_lat<5>("SHFL", out, cyc);
    run_lat<6>("VOTE", out, cyc);
    run_lat<7>("REDUX", out, cyc);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaFree(out);
    cudaFree(cyc);
    return e == cudaSuccess ? 0 : 1;
}
