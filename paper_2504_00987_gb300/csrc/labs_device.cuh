// labs_device.cuh -- device primitives of the LABS solver (sm_103a).
//
// Sequences live in registers as NW 32-bit words (2W for W 64-bit words, or
// 3 for 64 < N <= 96), bit i of the vector
// (word i / 32, bit i % 32) holding spin s_{i+1} (1 <-> +1).  A warp owns one
// sequence; every lane keeps an identical copy of the words ("warp-uniform")
// and lane l owns the indices l + 32q, q = 0 .. NW-1, of the per-index
// arrays (correlations C_k, tabu expiry of bit j).
#pragma once

#include <cstdint>

#include "labs.h"

namespace lgpu {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Philox counter word 3 (purpose) of the RNG contract in labs.h.
constexpr uint32_t kPurposeInit = 1u;
constexpr uint32_t kPurposeGen = 2u;
constexpr uint32_t kPurposeMut = 3u;
constexpr uint32_t kPurposeStep = 4u;
constexpr uint32_t kPurposeCross = 5u;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications by fixed odd constants with a Weyl-sequence key
// schedule; round r uses key + r * (golden-ratio, sqrt(3)-1) constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * x.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, x.x);
        const uint32_t lo1 = 0xCD9E8D57u * x.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, x.z);
        x = make_uint4(hi1 ^ x.y ^ k.x, lo1, hi0 ^ x.w ^ k.y, lo0);
    }
    return x;
}

__device__ __forceinline__ uint2 philox_key(uint64_t seed) {
    return make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

__device__ __forceinline__ uint4 draw4(uint2 key, uint32_t instance, uint32_t a, uint32_t b,
                                       uint32_t purpose) {
    return philox4x32_10(make_uint4(instance, a, b, purpose), key);
}

// randInt(lo, hi) inclusive: lo + floor(u * (hi - lo + 1) / 2^32).
__device__ __forceinline__ int32_t rand_int(int32_t lo, int32_t hi, uint32_t u) {
    const uint64_t span = static_cast<uint64_t>(static_cast<int64_t>(hi) - lo + 1);
    return lo + static_cast<int32_t>((static_cast<uint64_t>(u) * span) >> 32);
}

// Bits [0, n) of 32-bit word v (n may lie outside the word).
__device__ __forceinline__ uint32_t word_lowmask(int v, int n) {
    const int hi = n - 32 * v;
    return hi >= 32 ? kFull : (hi <= 0 ? 0u : ((1u << hi) - 1u));
}

// Position of the (n+1)-th set bit of x (n < popc(x)), by halving.
__device__ __forceinline__ int nth_set_bit(uint32_t x, int n) {
    int pos = 0;
#pragma unroll
    for (int width = 16; width >= 1; width >>= 1) {
        const uint32_t lowbits = x & ((1u << width) - 1u);
        const int c = __popc(lowbits);
        if (n >= c) {
            n -= c;
            x >>= width;
            pos += width;
        } else {
            x = lowbits;
        }
    }
    return pos;
}

// out = in >> s for an NW-word vector and a warp-uniform runtime shift
// 0 <= s < 32*NW: word moves by a log-depth select network, then one funnel
// shift per word.  No dynamic register indexing.
template <int NW>
__device__ __forceinline__ void shr_uniform(const uint32_t (&in)[NW], int s, uint32_t (&out)[NW]) {
    uint32_t a[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) a[w] = in[w];
    const int ws = s >> 5;
#pragma unroll
    for (int step = 1; step < NW; step <<= 1) {
        const bool take = (ws & step) != 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) a[w] = take ? (w + step < NW ? a[w + step] : 0u) : a[w];
    }
    const int bs = s & 31;
#pragma unroll
    for (int w = 0; w < NW; ++w) out[w] = __funnelshift_r(a[w], w + 1 < NW ? a[w + 1] : 0u, bs);
}

// oa = a >> s and ob = b >> s for two NW-word vectors and one warp-uniform
// shift 0 <= s < 32*NW: one select network and one set of funnel shifts
// shared by both.
template <int NW>
__device__ __forceinline__ void shr_uniform2(const uint32_t (&a)[NW], const uint32_t (&b)[NW], int s,
                                             uint32_t (&oa)[NW], uint32_t (&ob)[NW]) {
    uint32_t x[NW], y[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        x[w] = a[w];
        y[w] = b[w];
    }
    const int ws = s >> 5;
#pragma unroll
    for (int step = 1; step < NW; step <<= 1) {
        const bool take = (ws & step) != 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            x[w] = take ? (w + step < NW ? x[w + step] : 0u) : x[w];
            y[w] = take ? (w + step < NW ? y[w + step] : 0u) : y[w];
        }
    }
    const int bs = s & 31;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        oa[w] = __funnelshift_r(x[w], w + 1 < NW ? x[w + 1] : 0u, bs);
        ob[w] = __funnelshift_r(y[w], w + 1 < NW ? y[w + 1] : 0u, bs);
    }
}

// Two-word vectors: one 64-bit shift each (7.6 % less time per 1,024 x 10^5
// launch at N = 64 on GB300 than the select network, 4 % fewer instructions).
template <>
__device__ __forceinline__ void shr_uniform2<2>(const uint32_t (&a)[2], const uint32_t (&b)[2], int s,
                                                uint32_t (&oa)[2], uint32_t (&ob)[2]) {
    const uint64_t ra = ((static_cast<uint64_t>(a[1]) << 32) | a[0]) >> s;
    const uint64_t rb = ((static_cast<uint64_t>(b[1]) << 32) | b[0]) >> s;
    oa[0] = static_cast<uint32_t>(ra);
    oa[1] = static_cast<uint32_t>(ra >> 32);
    ob[0] = static_cast<uint32_t>(rb);
    ob[1] = static_cast<uint32_t>(rb >> 32);
}

// Flip bit i (warp-uniform) of an NW-word vector.
template <int NW>
__device__ __forceinline__ void flip_bit(uint32_t (&v)[NW], int i) {
    if constexpr (NW == 2) {  // one 64-bit one-hot mask
        const uint64_t m = 1ull << i;
        v[0] ^= static_cast<uint32_t>(m);
        v[1] ^= static_cast<uint32_t>(m >> 32);
    } else {
        const int wi = i >> 5;
        const uint32_t m = 1u << (i & 31);
#pragma unroll
        for (int w = 0; w < NW; ++w) v[w] ^= (w == wi) ? m : 0u;
    }
}

// Full-width reversal: bit (32*NW - 1 - i) of out = bit i of in.
template <int NW>
__device__ __forceinline__ void reverse_bits(const uint32_t (&in)[NW], uint32_t (&out)[NW]) {
#pragma unroll
    for (int w = 0; w < NW; ++w) out[w] = __brev(in[NW - 1 - w]);
}

// Bit i of an NW-word vector (0 <= i < 32*NW; i may differ between lanes).
template <int NW>
__device__ __forceinline__ uint32_t get_bit(const uint32_t (&v)[NW], int i) {
    const int wi = i >> 5;
    uint32_t x = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) x = (w == wi) ? v[w] : x;
    return (x >> (i & 31)) & 1u;
}

// Skew-symmetric completion of an odd-length sequence (Sec. II.C): with
// centre c = (N-1)/2, s_{c+i} = (-1)^i s_{c-i} for i = 1..c, i.e.
// b_{c+i} = b_{c-i} xor (i odd).  Bits [0, c] are kept, bits >= N cleared.
template <int NW>
__device__ __forceinline__ void skew_complete(uint32_t (&B)[NW], int N) {
    constexpr int NB = 32 * NW;
    const int c = (N - 1) >> 1;
    uint32_t RL[NW], RN[NW];
    reverse_bits<NW>(B, RL);
    shr_uniform<NW>(RL, NB - N, RN);                            // bit m of RN = b_{N-1-m}
    const uint32_t alt = (c & 1) ? 0x55555555u : 0xAAAAAAAAu;  // bit m set iff m - c odd
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t keep = word_lowmask(w, c + 1);
        B[w] = (B[w] & keep) | ((RN[w] ^ alt) & word_lowmask(w, N) & ~keep);
    }
}

}  // namespace lgpu
