// skew.cu -- labs_skew_deviation_batch: the deviation from skew-symmetry
// d(S) of Appendix A (Eqs. 5-9) for a batch of sequences.
//
// For a sequence T of odd length L = 2n - 1 (bits t_0 .. t_{L-1}, centre
// c = n - 1), Eq. 5 counts the i in 1..n-1 with s_{n+i} != (-1)^i s_{n-i};
// in bits that is t_{c+i} xor t_{c-i} xor [i odd], so
//   n_non-skew(T) = popc((R ^ Lr ^ ALT) & bits[1, n-1]),
// with R bit i = t_{c+i}, Lr bit i = t_{c-i} and ALT the odd positions.
// d(S) is the minimum of n_non-skew over the rotations Rot(S; r) (Eq. 6) for
// odd N, and over the rotations followed by one deletion Del(.; i) (Eq. 8)
// for even N (the reading that reproduces the d column of Table II).
//
// With D = S.S (the sequence twice, 2N bits) and DR its reversal, rotation r
// makes u_m = D[r + m]; deleting u_d shifts the positions at and after d by
// one, so R and Lr are bitwise selections between two windows of D (resp.
// DR) on either side of the deleted position.  One warp handles one
// sequence: the windows of rotation r are the same for every lane, the
// lanes split the deletion positions, and the warp takes the minimum.
#include <cuda_runtime.h>

#include <climits>

#include "capi_util.h"
#include "kernels.h"
#include "labs_device.cuh"

namespace lgpu {

constexpr int kSkewWarps = 4;
constexpr int kSkewWords = 2 * LABS_MAX_N / 32 + 2;  // D (2N bits) plus zero padding
constexpr int kSkewWin = LABS_MAX_N / 64 + 2;        // window words: n - 1 <= N/2 bits

// Window word w of the bit string V (shared words) starting at bit `start`.
__device__ __forceinline__ uint32_t window_word(const uint32_t* V, int start, int w) {
    const int o = (start >> 5) + w, b = start & 31;
    return __funnelshift_r(V[o], V[o + 1], b);
}

// Bits [lo, hi) of word w (empty if hi <= lo).
__device__ __forceinline__ uint32_t range_mask(int w, int lo, int hi) {
    return word_lowmask(w, hi) & ~word_lowmask(w, lo);
}

__global__ void __launch_bounds__(kSkewWarps * 32) skew_kernel(const uint64_t* __restrict__ seqs, int N,
                                                               int64_t B, int32_t* __restrict__ out) {
    __shared__ uint32_t Dsh[kSkewWarps][kSkewWords];
    __shared__ uint32_t DRsh[kSkewWarps][kSkewWords];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = static_cast<int64_t>(blockIdx.x) * kSkewWarps + warp;
    if (b >= B) return;
    const int W32 = (N + 31) / 32;
    const uint32_t* S = reinterpret_cast<const uint32_t*>(seqs + b * ((N + 63) / 64));
    uint32_t* D = Dsh[warp];
    uint32_t* DR = DRsh[warp];
    // D[x] = s_{x mod N}, DR[x] = D[2N-1-x], x < 2N; zero beyond.
    for (int k = 0; k < kSkewWords; ++k) {
        const int x = 32 * k + lane;
        int bd = 0, br = 0;
        if (x < 2 * N) {
            const int i = x % N, ir = (2 * N - 1 - x) % N;
            bd = (__ldg(S + i / 32) >> (i & 31)) & 1;
            br = (__ldg(S + ir / 32) >> (ir & 31)) & 1;
        }
        const uint32_t wd = __ballot_sync(kFull, bd), wr = __ballot_sync(kFull, br);
        if (lane == 0) {
            D[k] = wd;
            DR[k] = wr;
        }
    }
    (void)W32;
    __syncwarp();
    const bool odd = (N & 1) != 0;
    const int L = odd ? N : N - 1;  // length of the candidates
    const int c = (L - 1) / 2;      // centre index
    const int n = c + 1;            // L = 2n - 1
    const int nw = (n + 31) / 32;   // window words covering bits 0 .. n-1
    int best = INT_MAX;
    for (int r = 0; r < N; ++r) {
        uint32_t W1[kSkewWin], W2[kSkewWin], W3[kSkewWin], W4[kSkewWin];
#pragma unroll
        for (int w = 0; w < kSkewWin; ++w) {
            if (w < nw) {
                W1[w] = window_word(D, r + c, w);               // u_{c+i}
                W2[w] = window_word(D, r + c + 1, w);           // u_{c+i+1}
                W3[w] = window_word(DR, 2 * N - 1 - r - c, w);  // u_{c-i}
                W4[w] = window_word(DR, 2 * N - 2 - r - c, w);  // u_{c-i+1}
            } else {
                W1[w] = W2[w] = W3[w] = W4[w] = 0u;
            }
        }
        if (odd) {  // rotations only
            if (lane == 0) {
                int cnt = 0;
#pragma unroll
                for (int w = 0; w < kSkewWin; ++w)
                    if (w < nw) cnt += __popc((W1[w] ^ W3[w] ^ 0xAAAAAAAAu) & range_mask(w, 1, n));
                best = min(best, cnt);
            }
            continue;
        }
        for (int d = lane; d < N; d += 32) {  // delete u_d
            int cnt = 0;
#pragma unroll
            for (int w = 0; w < kSkewWin; ++w) {
                if (w < nw) {
                    // R bit i: u_{c+i} if c+i < d else u_{c+i+1};  Lr bit i: u_{c-i} if c-i < d else u_{c-i+1}
                    const uint32_t m1 = range_mask(w, 0, d - c);          // i < d - c
                    const uint32_t m2 = range_mask(w, 0, c - d + 1);      // i <= c - d
                    const uint32_t R = (W1[w] & m1) | (W2[w] & ~m1);
                    const uint32_t Lr = (W3[w] & ~m2) | (W4[w] & m2);
                    cnt += __popc((R ^ Lr ^ 0xAAAAAAAAu) & range_mask(w, 1, n));
                }
            }
            best = min(best, cnt);
        }
    }
    best = __reduce_min_sync(kFull, best);
    if (lane == 0) out[b] = best;
}

cudaError_t launch_skew(const uint64_t* d_seqs, int N, int64_t B, int32_t* d_out, cudaStream_t stream) {
    const int64_t blocks = (B + kSkewWarps - 1) / kSkewWarps;
    skew_kernel<<<static_cast<unsigned>(blocks), kSkewWarps * 32, 0, stream>>>(d_seqs, N, B, d_out);
    return cudaGetLastError();
}

}  // namespace lgpu

extern "C" int32_t labs_skew_deviation_batch(const uint64_t* d_seqs, int32_t N, int64_t B, int32_t* d_d,
                                             labs_stream_t stream) {
    using namespace lcapi;
    if (N < 3 || N > LABS_MAX_N) return fail(LABS_EINVAL, "N=%d outside 3..%d", N, LABS_MAX_N);
    if ((N & 1) == 0 && N < 4) return fail(LABS_EINVAL, "even N must be >= 4");
    if (B < 0) return fail(LABS_EINVAL, "B < 0");
    if (B == 0) return ok();
    if (B > (int64_t{1} << 33)) return fail(LABS_EINVAL, "B too large");
    LABS_TRY(check_dev(d_seqs, 8, "d_seqs", false));
    LABS_TRY(check_dev(d_d, 4, "d_d", false));
    const cudaError_t e = lgpu::launch_skew(d_seqs, N, B, d_d, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "skew kernel launch");
    return ok();
}
