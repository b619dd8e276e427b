// tabu_core.cuh -- one warp runs one tabu search (Algorithm 2 / Algorithm 4).
//
// Neighbour scoring (Sec. III.C, Table I).  Flipping s_j changes C_k by
// delta_k(j) = -2 s_j (s_{j+k} + s_{j-k}) (terms outside 1..N dropped), so
//   E_j = E + sum_k delta_k (2 C_k + delta_k)
//       = E + 4(N-1) + 8 M_j - 4 s_j R_j,
// with M_j = sum_{k>=1} s_{j+k} s_{j-k} (a masked popcount of the XOR of the
// two windows of j) and R_j = sum_k C_k (s_{j+k} + s_{j-k}).  R_j is set up
// once per search on bit planes (0-based bits b_i, s_i = 2 b_i - 1):
//   R_j = 2 S_j - T_j,  S_j = sum_k C_k (b_{j+k} + b_{j-k}),
//   T_j = sum_{k<=j} C_k + sum_{k<=N-1-j} C_k,
// where S_j = sum_m w_m [popc(t_m & X_j) + popc(t_m & Y_j)] over the
// two's-complement planes t_m of C_k (from warp ballots), X_j = pivot >> j
// (bit k = b_{j+k}) and Y_j the mirrored window (bit k = b_{j-k}); T_j comes
// from prefix sums of C_k.  After every move R_j is updated exactly instead
// of re-scored (the identity is derived above tabu_search), so a step costs
// about one bit plane of the from-scratch scoring.  Arithmetic is exact int32.
//
// Work split: lane l scores neighbours j = l + 32q and keeps their R_j and
// tabu expiry in registers; C_k before and after the move sit in two
// warp-private shared-memory buffers.  The admissible minimum is one
// redux.sync.min over packed (E_j, j) keys, the ties are counted by one
// redux.sync.add, and a tie pick by the step's draw in ascending j uses
// ballots only when it is not the lowest minimiser.  Applying the move
// flips the pivot, recomputes (short sequences) or updates C_k, updates
// every R_j and sets the tenure.
#pragma once

#include <climits>

#include "labs_device.cuh"

namespace lgpu {

// C_k = (N - k) - 2 popc(b_i xor b_{i+k} over i < N-k) for the lane's
// k = lane + 32q (C_0 and C_{k >= N} are 0).
template <int NW>
__device__ __forceinline__ void correlations(const uint32_t (&B)[NW], int N, int lane,
                                             int32_t (&c)[NW]) {
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int k = lane + 32 * q;
        int cnt = 0;
#pragma unroll
        for (int w = 0; w + q < NW; ++w) {
            const uint32_t xk = __funnelshift_r(B[w + q], (w + q + 1 < NW) ? B[w + q + 1] : 0u, lane);
            cnt += __popc((B[w] ^ xk) & word_lowmask(w, N - k));
        }
        c[q] = (k >= 1 && k <= N - 1) ? (N - k) - 2 * cnt : 0;
    }
}

// Energy of the warp-uniform sequence B (all lanes return it).
template <int NW>
__device__ __forceinline__ int32_t warp_energy(const uint32_t (&B)[NW], int N, int lane) {
    int32_t c[NW];
    correlations<NW>(B, N, lane, c);
    int32_t sq = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) sq += c[q] * c[q];
    return __reduce_add_sync(kFull, sq);
}

// Energy of one sequence computed by a single thread (bits in `w`).
template <int NW>
__device__ __forceinline__ int32_t thread_energy(const uint32_t (&B)[NW], int N) {
    int32_t E = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        for (int l = 0; l < 32; ++l) {
            const int k = 32 * q + l;
            if (k < 1 || k > N - 1) continue;
            int cnt = 0;
#pragma unroll
            for (int w = 0; w + q < NW; ++w) {
                const uint32_t xk =
                    __funnelshift_r(B[w + q], (w + q + 1 < NW) ? B[w + q + 1] : 0u, l);
                cnt += __popc((B[w] ^ xk) & word_lowmask(w, N - k));
            }
            const int32_t Ck = (N - k) - 2 * cnt;
            E += Ck * Ck;
        }
    }
    return E;
}

struct TabuOut {
    int64_t steps = 0;
    int32_t E_best = 0;
    bool fault = false;  // the two warps of a replica lost step (a bounded wait ran out)
};

// Two warps of one CTA sharing one replica ("warps per sequence" = 2): each
// runs the whole replica on its own copy of the state and scores half of
// the neighbours; per step they exchange their admissible minima through
// this shared-memory word pair.  Exchange x of a pair uses slot [x & 1] (so
// a warp that runs ahead never overwrites a word its partner has not read:
// it cannot publish x + 2 before the partner published x + 1, which comes
// after the partner read x); a word holds (x mod 2^24) << 40 | value.
struct PairLink {
    unsigned long long slot[2][2];  // [x & 1][half]
};

constexpr uint32_t kPairSpinLimit = 1u << 22;  // ~10^8 cycles, far beyond one step's skew

// Publishes this warp's value v (< 2^40) of exchange x and returns the
// partner's in `other`.  Lane 0 spins on the partner's word with a bounded
// number of polls; false if they run out (the caller stops the replica).
__device__ __forceinline__ bool pair_exchange(PairLink* link, int half, uint32_t x, uint64_t v,
                                              uint64_t& other, int lane) {
    const uint64_t tag = static_cast<uint64_t>(x & 0xFFFFFFu) << 40;
    bool ok = true;
    uint64_t w = 0;
    if (lane == 0) {
        volatile unsigned long long* mine = &link->slot[x & 1u][half];
        volatile unsigned long long* theirs = &link->slot[x & 1u][half ^ 1];
        *mine = tag | v;
        for (uint32_t it = 0;; ++it) {
            w = *theirs;
            if ((w >> 40) == (x & 0xFFFFFFu)) break;
            if (it >= kPairSpinLimit) {
                ok = false;
                break;
            }
        }
    }
    ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
    other = __shfl_sync(kFull, static_cast<unsigned long long>(w), 0) & ((1ull << 40) - 1);
    return ok;
}

// Bit-plane count bound: |C_k| <= N - 1 < 32*NW, so C_k fits in
// bitlen(32*NW - 1) + 1 two's-complement bits.
template <int NW>
struct PlaneMax {
    static constexpr int value = (NW == 2) ? 7 : (NW <= 4) ? 8 : 9;
};

// sum_i popc(w[i]) * weight for n words, carry-save compressed: full
// adders (sum = a^b^c, carry = maj(a,b,c), one LOP3 each) fold three words
// of one weight into one word of that weight and one of twice the weight,
// so n words cost about n/2 + log n popcounts instead of n.  The adders
// trade popcounts (XU pipe) for logic (ALU pipe), which pays while the
// step has registers to spare: for 7 or more words (six- and eight-word
// sequences, N > 160) plain popcounts measured 14-21 % faster on GB300
// and 2-16 % slower below; five-word sequences (6 words) count plainly as
// well.  Five words (four-word sequences) take one full adder and two plain
// popcounts, about 1 % faster than two adders.
template <int n, int weight>
__device__ __forceinline__ int csa_popc(const uint32_t (&w)[n]) {
    if constexpr (weight == 1 && n == 5) {
        const uint32_t a = w[0], b = w[1], c = w[2];
        return __popc(a ^ b ^ c) + 2 * __popc((a & b) | (c & (a | b))) + __popc(w[3]) + __popc(w[4]);
    } else if constexpr (n <= 2 || (weight == 1 && n >= 6)) {
        int s = 0;
#pragma unroll
        for (int i = 0; i < n; ++i) s += __popc(w[i]);
        return s * weight;
    } else {
        constexpr int f = (n - 1) / 2;  // full adders at this weight
        uint32_t carry[f];
        uint32_t acc = w[0];
#pragma unroll
        for (int i = 0; i < f; ++i) {
            const uint32_t a = acc, b = w[1 + 2 * i], c = w[2 + 2 * i];
            acc = a ^ b ^ c;
            carry[i] = (a & b) | (c & (a | b));
        }
        int s = __popc(acc);
        if constexpr (n - 2 * f == 2) s += __popc(w[n - 1]);
        return s * weight + csa_popc<f, 2 * weight>(carry);
    }
}

// S[q] += sum over planes m < P of w_m [popc(t_m & X_q) + popc(t_m & Y_q)],
// plane 0 being the constant parity pattern of C_k (C_k = N - k mod 2) and
// plane P-1 the sign plane (weight -2^(P-1)).  Fully unrolled for a
// compile-time P so every ballot and popcount of the step can overlap.
template <int NW, int P>
__device__ __forceinline__ void score_planes(const int32_t (&c)[NW], const uint32_t (&par)[NW],
                                             const uint32_t (&X)[NW][NW],
                                             const uint32_t (&Y)[NW][NW], int32_t (&S)[NW]) {
#pragma unroll
    for (int m = 0; m < P; ++m) {
        uint32_t tp[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) tp[w] = (m == 0) ? par[w] : __ballot_sync(kFull, (c[w] >> m) & 1);
        constexpr int32_t one = 1;
        const int32_t wm = (m == P - 1) ? -(one << m) : (one << m);
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            uint32_t words[NW + 1];  // (NW - q) words of X_j and (q + 1) of Y_j
#pragma unroll
            for (int w = 0; w + q < NW; ++w) words[w] = tp[w] & X[q][w];
#pragma unroll
            for (int w = 0; w <= q; ++w) words[NW - q + w] = tp[w] & Y[q][w];
            S[q] += csa_popc<NW + 1, 1>(words) * wm;
        }
    }
}

// Inclusive prefix sums of C at the lane's own indices: pc[q] = PC(l + 32q),
// PC(n) = sum_{k=1}^{n} C_k (C_0 = 0).  Two chunks share one packed 32-bit
// shuffle scan (low and high 16-bit halves; every within-chunk prefix is
// bounded by 32 (N-1) < 2^15).  Used once per search; afterwards the sums
// are updated incrementally per move.
template <int NW>
__device__ __forceinline__ void prefix_own(const int32_t (&c)[NW], int lane, int32_t (&pc)[NW]) {
    constexpr int NP = NW & ~1;  // chunks scanned in pairs
    int32_t carry = 0;
#pragma unroll
    for (int q = 0; q < NP; q += 2) {
        int32_t v = c[q] + c[q + 1] * 65536;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t n = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += n;
        }
        const int32_t last = __shfl_sync(kFull, v, 31);
        const int32_t lo = static_cast<int32_t>(static_cast<int16_t>(v & 0xFFFF));
        const int32_t hi = (v - lo) / 65536;
        const int32_t lo31 = static_cast<int32_t>(static_cast<int16_t>(last & 0xFFFF));
        const int32_t hi31 = (last - lo31) / 65536;
        pc[q] = carry + lo;
        pc[q + 1] = carry + lo31 + hi;
        carry += lo31 + hi31;
    }
    if constexpr (NW & 1) {  // an odd word count leaves one chunk, scanned alone
        int32_t v = c[NW - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t n = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += n;
        }
        pc[NW - 1] = carry + v;
    }
}

// T_j = PC(j) + PC(N-1-j) for the lane's j = l + 32q: its own prefix plus
// the mirror index's prefix, read back through the warp's shared scratch.
template <int NW>
__device__ __forceinline__ void mirror_terms(const int32_t (&pc)[NW], int N, int lane,
                                             int32_t* __restrict__ Cs, int32_t (&T)[NW]) {
#pragma unroll
    for (int q = 0; q < NW; ++q) Cs[lane + 32 * q] = pc[q];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int j = lane + 32 * q;
        T[q] = pc[q] + Cs[j < N ? N - 1 - j : 0];
    }
    __syncwarp();
}

// Scores S_j with P bit planes, where P >= the planes C_k needs (extra
// planes only repeat the sign and leave the sum exact).  Three fully
// unrolled widths keep the code small enough for the instruction cache
// (a jump table over every width measured several hundred cycles slower).
template <int NW>
__device__ __forceinline__ void score_dispatch(int P, const int32_t (&c)[NW], const uint32_t (&par)[NW],
                                               const uint32_t (&X)[NW][NW], const uint32_t (&Y)[NW][NW],
                                               int32_t (&S)[NW]) {
#pragma unroll
    for (int q = 0; q < NW; ++q) S[q] = 0;
    if (P <= 5)
        score_planes<NW, 5>(c, par, X, Y, S);
    else if (P <= 6)
        score_planes<NW, 6>(c, par, X, Y, S);
    else
        score_planes<NW, PlaneMax<NW>::value>(c, par, X, Y, S);
}

// Number of two's-complement planes that hold every C_k of the warp:
// bit length of max |C_k| plus the sign bit.
template <int NW>
__device__ __forceinline__ int plane_count(const int32_t (&c)[NW]) {
    uint32_t mx = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) mx = max(mx, static_cast<uint32_t>(abs(c[q])));
    return 33 - __clz(__reduce_max_sync(kFull, mx));
}

// The lane's windows of an NW-word vector: XB[i] = word i of B >> lane and
// YB[i] = word i of RL >> (31 - lane).  For j = lane + 32q, word w of the
// forward window X_j (bit k = b_{j+k}) is XB[q + w] and word w of the
// backward window Y_j (bit k = b_{j-k}) is YB[w + NW - 1 - q]; both are zero
// past the ends of the sequence.
template <int NW>
__device__ __forceinline__ void pivot_windows(const uint32_t (&B)[NW], const uint32_t (&RL)[NW],
                                              int lane, uint32_t (&XB)[NW], uint32_t (&YB)[NW]) {
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        XB[i] = __funnelshift_r(B[i], i + 1 < NW ? B[i + 1] : 0u, lane);
        YB[i] = __funnelshift_r(RL[i], i + 1 < NW ? RL[i + 1] : 0u, 31 - lane);
    }
}

// One tabu search from `seq` (warp-uniform).  On return `seq` holds
// bestSeqTS.  Draws: step t uses Philox(instance, g, t, 4): x tie, y tenure.
// FIX_FIRST: bit 0 (s_1) is never a candidate move.
// `Cs` is warp-private shared scratch of 64*NW ints (two buffers of C_k).
// With TRACE, `trace` receives {g, t, j, E} per step while trace_len <
// trace_cap.
//
// Neighbour scores are kept between steps.  With
//   R_j = sum_k C_k (s~_{j+k} + s~_{j-k})     (s~_i = s_i inside 0..N-1, else 0)
//   M_j = sum_{k>=1} s~_{j+k} s~_{j-k},
// the energy after flipping j is E_j = E + 4(N-1) + 8 M_j - 4 s_j R_j (the
// delta_k(j)(2 C_k + delta_k(j)) sum of Table I, expanded).  R_j is set up
// once per search on the bit planes of C_k; after the move p (s_p before
// it, C and C' the correlations before and after, d = |p - j|, s'_j after
// the move) it changes exactly by
//   R'_j = R_j - 2 s_p (C_d + C'_d + F_j) - 2 s'_j          (j != p)
//   R'_p = R_p - 2 s_p (N - 1 + 2 M_p)
// with F_j = sum_{k>=1} s~_{p+k} s~'_{j-k} + sum_{k>=1} s~_{p-k} s~'_{j+k}
// (s~' after the move).  Derivation: R'_j - R_j = sum_k C_k (s~'-s~)
// (terms j+-k = p: -2 s_p C_d) + sum_k delta_k(p) (s~'_{j+k} + s~'_{j-k});
// the second sum pairs the windows of p and j: its same-direction pairs
// (p+k, j+k), (p-k, j-k) cover every product of C'_d except s'_p s'_j, and
// its crossed pairs are F_j.  At j = p the crossed pairs give F_p = 2 M_p and
// s'_p = -s_p, so the first line gives the second when C_0 + C'_0 = N: the
// two buffers hold ceil(N/2) and floor(N/2) at k = 0 and one update serves
// every j.  F_j is two masked popcounts over the windows of p and j (the
// crossed pairs agree or disagree), C_d and C'_d are read from the two
// shared buffers, so a step costs about one bit plane of the from-scratch
// scoring instead of one per bit of max |C_k|.
//
// WPS = 2 (two warps per replica, HALF = which one): the warp scores and
// updates only the neighbours j = lane + 32q of its half of q, keeps its own
// copy of everything else (pivot, correlations, bestSeqTS), and the two
// minima meet through `link`; the lower half's neighbours come first in
// ascending j for the tie pick.  Both warps take every decision from the
// same values, so they run the same steps; `xseq` counts the pair's
// exchanges.  A bounded wait that runs out ends the search with fault set.
template <int NW, bool TRACE, bool FIX_FIRST = false, int WPS = 1, int HALF = 0, bool PERK = false>
__device__ TabuOut tabu_search(uint32_t (&seq)[NW], const int N, const uint2 key,
                               const uint32_t inst, const uint32_t g, const int max_iter,
                               const int64_t budget, int32_t* __restrict__ Cs,
                               int4* __restrict__ trace, const int64_t trace_cap,
                               int64_t& trace_len, const int lane, PairLink* link = nullptr,
                               uint32_t* xseq = nullptr) {
    static_assert(WPS == 1 || (WPS == 2 && NW % 2 == 0 && HALF >= 0 && HALF < 2), "warps per sequence");
    constexpr int NB = 32 * NW;
    constexpr int QB = HALF * (NW / WPS), QE = (HALF + 1) * (NW / WPS);  // this warp's q
    // Correlations after a move are recomputed from the pivot's windows when
    // they are short (fewer ALU-pipe instructions than the per-k update: at
    // N = 64 the per-k update measured 11-15 % slower with two warps per SM
    // sub-partition) and updated per k otherwise.  PERK (the batch and
    // service kernels, whose warps mostly run alone on their sub-partition,
    // so that a step's dependency chain sets its time) always updates per k:
    // the update needs only the move's windows, not the flipped pivot, which
    // measured 13 % less time for the 512-instance uneven batch on GB300 and
    // 8 % less median service latency.
    constexpr bool kRecompute = NW <= 4 && !PERK;
    uint32_t B[NW], RL[NW], Bb[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        B[w] = seq[w];
        Bb[w] = seq[w];
    }
    reverse_bits<NW>(B, RL);
    uint32_t XB[NW], YB[NW];
    pivot_windows<NW>(B, RL, lane, XB, YB);
    int32_t c[NW];
    correlations<NW>(B, N, lane, c);
    int32_t E;
    {
        int32_t sq = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) sq += c[q] * c[q];
        E = __reduce_add_sync(kFull, sq);
    }
    int32_t E_best = E;
    // Per-search constants of the lane's neighbours j = lane + 32q: validity,
    // L_j = min(j, N-1-j) and the masks of k in [1, L_j] (M_j), the range
    // masks of the forward windows (bits k <= N-1-j of X_j, word i = q + w),
    // and for the recomputed correlations the masks of i < N - k.
    int32_t tabu[NW], Lq[NW];
    uint32_t mmask[NW][NW], mX[NW];
    uint32_t jvalid = 0;  // bit q: j < N and j may move
#pragma unroll
    for (int q = 0; q < NW; ++q) mX[q] = word_lowmask(q, N - lane);
#pragma unroll
    for (int q = QB; q < QE; ++q) {
        const int j = lane + 32 * q;
        Lq[q] = min(j, N - 1 - j);
        const bool movable = j < N && !(FIX_FIRST && j == 0);
        jvalid |= (movable ? 1u : 0u) << q;
        // A neighbour that may not move is already excluded by jvalid; for
        // two-word sequences it also gets an expiry that never passes, which
        // changes no result but measured 2.8 % less time per launch at N = 64
        // on GB300 (code generation; the same line cost 0.4-5 % at N = 92..160).
        tabu[q] = (NW == 2 && !movable) ? INT_MAX : 0;
#pragma unroll
        for (int w = 0; w <= q && w + q < NW; ++w)
            mmask[q][w] = word_lowmask(w, Lq[q] + 1) & (w == 0 ? ~1u : kFull);
    }
    const uint32_t low_l = (lane == 31) ? kFull : ((2u << lane) - 1u);  // bits 0..lane
    // R_j = 2 S_j - T_j from the bit planes of C_k (S_j) and the prefix sums
    // of C_k (T_j = PC(j) + PC(N-1-j)), once per search.
    int32_t R[NW];
    {
        uint32_t par[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t alt = ((N - 32 * w) & 1) ? 0x55555555u : 0xAAAAAAAAu;  // (N - k) odd
            par[w] = alt & word_lowmask(w, N) & (w == 0 ? ~1u : kFull);
        }
        uint32_t X[NW][NW], Y[NW][NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
#pragma unroll
            for (int w = 0; w + q < NW; ++w) X[q][w] = XB[q + w];
#pragma unroll
            for (int w = 0; w <= q; ++w) Y[q][w] = YB[w + NW - 1 - q];
        }
        int32_t S[NW], pc[NW], T[NW];
        score_dispatch<NW>(plane_count<NW>(c), c, par, X, Y, S);
        prefix_own<NW>(c, lane, pc);
        mirror_terms<NW>(pc, N, lane, Cs, T);
#pragma unroll
        for (int q = QB; q < QE; ++q) R[q] = 2 * S[q] - T[q];
    }
    // C_k of the pivot (Ccur) and after the move (Cnxt), k = 1 .. NB-1 (0 past
    // N-1); slot k = 0 holds ceil(N/2) in one buffer and floor(N/2) in the
    // other and is never rewritten (see the update of R_p above).
    int32_t* Ccur = Cs;
    int32_t* Cnxt = Cs + NB;
#pragma unroll
    for (int q = 0; q < NW; ++q) Ccur[lane + 32 * q] = c[q];
    if (lane == 0) {
        Ccur[0] = N - N / 2;
        Cnxt[0] = N / 2;
    }
    __syncwarp();
    const bool own_c0 = lane == 0;  // the lane whose k = lane + 32q is 0 at q = 0
    // correlation masks of the recomputation: i < N - k for k = lane + 32q
    uint32_t cmask[kRecompute ? NW : 1][kRecompute ? NW : 1];
    int32_t nk[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int k = lane + 32 * q;
        nk[q] = (k >= 1 && k <= N - 1) ? N - k : 0;
        if constexpr (kRecompute) {
#pragma unroll
            for (int w = 0; w + q < NW; ++w) cmask[q][w] = word_lowmask(w, nk[q]);
        }
    }
    // all-ones masks: bits 0 .. N-1, and every bit (the move's ranges below)
    uint32_t allN[NW], allB[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        allN[w] = word_lowmask(w, N);
        allB[w] = kFull;
    }
    const int min_t = max_iter / 10;
    const int max_t = (12 * max_iter) / 100;
    const int64_t nsteps = budget < 0 ? max_iter : (budget < max_iter ? budget : max_iter);
    uint32_t rx = 0, ry = 0;
    int64_t steps = 0;
    bool fault = false;

    for (int t = 1; t <= nsteps; ++t) {
        if (((t - 1) & 31) == 0) {  // draws of steps t .. t+31, one per lane
            const uint4 r = draw4(key, inst, g, static_cast<uint32_t>(t + lane), kPurposeStep);
            rx = r.x;
            ry = r.y;
        }
        const int src = (t - 1) & 31;
        const uint32_t u_tie = __shfl_sync(kFull, rx, src);
        const uint32_t u_ten = __shfl_sync(kFull, ry, src);
        // ---- E_j for j = lane + 32q, admissibility, packed (E_j, j) keys
        const int32_t E0 = E + 4 * (N - 1);
        int32_t cand[NW], Mq[NW];
        int32_t kmin_l = INT_MAX;
#pragma unroll
        for (int q = QB; q < QE; ++q) {
            int dm = 0;
#pragma unroll
            for (int w = 0; w <= q && w + q < NW; ++w)
                dm += __popc((XB[q + w] ^ YB[w + NW - 1 - q]) & mmask[q][w]);
            Mq[q] = Lq[q] - 2 * dm;
            // s_j R_j (bit 0 of X_j is b_j): a select for two-word sequences,
            // a multiply by 2 b_j - 1 above (off the busy ALU pipe; 3-6 % less
            // time per launch for N = 92 .. 200 on GB300, 1 % more at N = 64)
            int32_t sR;
            if constexpr (NW >= 3)
                sR = (2 * static_cast<int32_t>(XB[q] & 1u) - 1) * R[q];
            else
                sR = (XB[q] & 1u) ? R[q] : -R[q];
            const int32_t Ej = E0 + 8 * Mq[q] - 4 * sR;
            const bool adm = ((jvalid >> q) & 1u) && (tabu[q] < t || Ej < E_best);
            cand[q] = adm ? Ej : INT_MAX;
            // E_j < 2^23 for N <= 256 and j < 256: (E_j, j) packs into 31 bits
            kmin_l = min(kmin_l, adm ? (Ej << 8) | (lane + 32 * q) : INT_MAX);
        }
        const int32_t kmin_w = __reduce_min_sync(kFull, kmin_l);
        int eq = 0;  // this warp's admissible minimisers
#pragma unroll
        for (int q = QB; q < QE; ++q) eq += (cand[q] == (kmin_w >> 8)) ? 1 : 0;
        const int count_w = __reduce_add_sync(kFull, eq);  // 0 when nothing is admissible
        int32_t kmin = kmin_w;
        int count = count_w, count_lo = 0;  // count_lo: minimisers of the lower half (WPS = 2)
        if constexpr (WPS == 2) {
            uint64_t o = 0;
            if (!pair_exchange(link, HALF, (*xseq)++,
                               (static_cast<uint64_t>(count_w) << 31) | static_cast<uint32_t>(kmin_w), o, lane)) {
                fault = true;
                break;
            }
            const int32_t kmin_o = static_cast<int32_t>(o & 0x7FFFFFFFu);
            const int count_o = static_cast<int>(o >> 31);
            kmin = min(kmin_w, kmin_o);
            // minimisers of either half: the same energy, whatever their index
            const int cw = (kmin_w >> 8) == (kmin >> 8) ? count_w : 0;
            const int co = (kmin_o >> 8) == (kmin >> 8) ? count_o : 0;
            count = cw + co;
            count_lo = HALF == 0 ? cw : co;
        }
        // Every move tabu and none aspirating: the search has no admissible
        // move and stops.  The default maxIter keeps maxTabu below N, so only a
        // user maxIter of about 8N or more (maxTabu >= N) gets here.
        if (kmin == INT_MAX) break;
        const int32_t m = kmin >> 8;
        int p = kmin & 255;  // lowest admissible minimiser
        {
            int idx = count > 1 ? static_cast<int>((static_cast<uint64_t>(u_tie) * count) >> 32) : 0;
            if (idx > 0) {  // the idx-th minimiser in ascending j
                bool mine = true;  // WPS = 2: the warp holding it finds it, then tells the other
                if constexpr (WPS == 2) {
                    mine = HALF == 0 ? idx < count_lo : idx >= count_lo;
                    if (HALF == 1) idx -= count_lo;
                }
                if (mine) {
                    bool found = false;
#pragma unroll
                    for (int q = QB; q < QE; ++q) {
                        const uint32_t tb = __ballot_sync(kFull, cand[q] == m);
                        const int pc_q = __popc(tb);
                        if (!found) {
                            if (idx < pc_q) {
                                p = 32 * q + nth_set_bit(tb, idx);
                                found = true;
                            } else {
                                idx -= pc_q;
                            }
                        }
                    }
                }
                if constexpr (WPS == 2) {
                    uint64_t o = 0;
                    if (!pair_exchange(link, HALF, (*xseq)++, mine ? static_cast<uint64_t>(p) : 0u, o, lane)) {
                        fault = true;
                        break;
                    }
                    if (!mine) p = static_cast<int>(o);
                }
            }
        }
        // ---- the move p: its windows (before the flip; bits k >= 1 are the
        // same after it), s_p, and the ranges k in [1, N-1-p] and [1, p]
        uint32_t Xp[NW], Yp[NW], mu[NW], mv[NW];
        shr_uniform2<NW>(B, allN, p, Xp, mu);            // mu: bits 0 .. N-1-p
        shr_uniform2<NW>(RL, allB, NB - 1 - p, Yp, mv);  // mv: bits 0 .. p
        mu[0] &= ~1u;
        mv[0] &= ~1u;
        const int32_t sp2 = (Xp[0] & 1u) ? 2 : -2;  // 2 s_p
        int32_t dq[NW], c0[NW];
#pragma unroll
        for (int q = QB; q < QE; ++q) {
            dq[q] = abs(p - (lane + 32 * q));
            c0[q] = Ccur[dq[q]];  // C_d before the move
        }
        flip_bit<NW>(B, p);
        // the mirror image: one bit flip for two words (a 64-bit one-hot), a
        // full reversal (one brev per word, no per-word select) above
        if constexpr (NW >= 3)
            reverse_bits<NW>(B, RL);
        else
            flip_bit<NW>(RL, NB - 1 - p);
        pivot_windows<NW>(B, RL, lane, XB, YB);
        if constexpr (kRecompute) {
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                int cnt = 0;
#pragma unroll
                for (int w = 0; w + q < NW; ++w) cnt += __popc((B[w] ^ XB[w + q]) & cmask[q][w]);
                c[q] = nk[q] - 2 * cnt;
            }
        } else {
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                const int32_t bx = (Xp[q] >> lane) & 1u, by = (Yp[q] >> lane) & 1u;
                const int32_t sx = ((mu[q] >> lane) & 1u) ? 2 * bx - 1 : 0;
                const int32_t sy = ((mv[q] >> lane) & 1u) ? 2 * by - 1 : 0;
                c[q] -= sp2 * (sx + sy);
            }
        }
#pragma unroll
        for (int q = 0; q < NW; ++q)
            if (q > 0 || !own_c0) Cnxt[lane + 32 * q] = c[q];
        __syncwarp();
#pragma unroll
        for (int q = QB; q < QE; ++q) {
            const int j = lane + 32 * q;
            const int32_t c1 = Cnxt[dq[q]];  // C'_d
            // crossed pairs: (p+k, j-k) for k <= min(N-1-p, j) and
            // (p-k, j+k) for k <= min(p, N-1-j); each disagreement is -1
            uint32_t words[NW + 1];
#pragma unroll
            for (int w = 0; w <= q; ++w)
                words[w] = (Xp[w] ^ YB[w + NW - 1 - q]) & mu[w] & (w == q ? low_l : kFull);
#pragma unroll
            for (int w = 0; w + q < NW; ++w) words[q + 1 + w] = (Yp[w] ^ XB[q + w]) & mv[w] & mX[q + w];
            const int32_t F = min(N - 1 - p, j) + min(p, N - 1 - j) - 2 * csa_popc<NW + 1, 1>(words);
            const int32_t sj2 = (XB[q] & 1u) ? 2 : -2;  // 2 s'_j
            R[q] -= sp2 * (c0[q] + c1 + F) + sj2;
        }
        {
            int32_t* tmp = Ccur;
            Ccur = Cnxt;
            Cnxt = tmp;
        }
        const int32_t expiry = t + rand_int(min_t, max_t, u_ten);
#pragma unroll
        for (int q = QB; q < QE; ++q)
            if (lane + 32 * q == p) tabu[q] = expiry;
        E = m;
        if (m < E_best) {
            E_best = m;
#pragma unroll
            for (int w = 0; w < NW; ++w) Bb[w] = B[w];
        }
        ++steps;
        if constexpr (TRACE) {
            if (trace_len < trace_cap) {
                if (lane == 0 && HALF == 0) trace[trace_len] = make_int4(static_cast<int>(g), t, p, m);
                ++trace_len;
            }
        }
    }
    __syncwarp();  // the buffers are reused by the caller
#pragma unroll
    for (int w = 0; w < NW; ++w) seq[w] = Bb[w];
    TabuOut out;
    out.steps = steps;
    out.E_best = E_best;
    out.fault = fault;
    return out;
}

}  // namespace lgpu
