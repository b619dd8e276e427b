// tabu_core.cuh -- one warp runs one tabu search (Algorithm 2 / Algorithm 4).
//
// Neighbour scoring (Sec. III.C).  Flipping s_j changes C_k by
// delta_k(j) = -2 s_j (s_{j+k} + s_{j-k}) (terms outside 1..N dropped), so
//   E_j = E + sum_k delta_k (2 C_k + delta_k)
//       = E + 4(N-1) + 8 M_j - 4 s_j (2 S_j - T_j),
// with (0-based bits b_i, s_i = 2 b_i - 1)
//   M_j = sum_{k=1}^{min(j, N-1-j)} s_{j+k} s_{j-k},
//   S_j = sum_k C_k (b_{j+k} + b_{j-k}),
//   T_j = sum_{k<=j} C_k + sum_{k<=N-1-j} C_k.
// S_j is evaluated on bit planes: with C_k in P-bit two's complement
// (P = bit length of max|C_k| plus a sign bit), S_j = sum_m w_m
// [popc(t_m & X_j) + popc(t_m & Y_j)], where t_m is the bit vector over k of
// bit m of C_k (from a warp ballot), w_m = 2^m (-2^(P-1) for the sign
// plane), X_j = pivot >> j (bit k = b_{j+k}) and Y_j the mirrored window
// (bit k = b_{j-k}).  Every popcount covers 32 pair-terms of one plane, and
// the arithmetic is exact int32 throughout.
//
// Work split: lane l scores neighbours j = l + 32q; lane l keeps C_k and the
// tabu expiry of index l + 32q in registers.  The admissible minimum is a
// warp redux; ties are counted with ballots and broken by the step's tie
// draw in ascending j.  Applying the move updates C_k in O(N) (one delta
// per lane slot), flips the pivot and sets the tenure.
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
    int64_t steps;
    int32_t E_best;
};

// One tabu search from `seq` (warp-uniform).  On return `seq` holds
// bestSeqTS.  Draws: step t uses Philox(instance, g, t, 4): x tie, y tenure.
// `Cs` is warp-private shared scratch of 32*NW ints.  `trace` (nullable)
// receives {g, t, j, E} per step while trace_len < trace_cap.
template <int NW>
__device__ TabuOut tabu_search(uint32_t (&seq)[NW], const int N, const uint2 key,
                               const uint32_t inst, const uint32_t g, const int max_iter,
                               const int64_t budget, int32_t* __restrict__ Cs,
                               int4* __restrict__ trace, const int64_t trace_cap,
                               int64_t& trace_len, const int lane) {
    constexpr int NB = 32 * NW;
    uint32_t B[NW], RL[NW], Bb[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        B[w] = seq[w];
        Bb[w] = seq[w];
    }
    reverse_bits<NW>(B, RL);  // bit (NB-1-i) of RL = b_i
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
    int32_t tabu[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) tabu[q] = 0;
    const int min_t = max_iter / 10;
    const int max_t = (12 * max_iter) / 100;
    const int64_t nsteps = budget < 0 ? max_iter : (budget < max_iter ? budget : max_iter);
    uint32_t rx = 0, ry = 0;
    int64_t steps = 0;

    for (int t = 1; t <= nsteps; ++t) {
        if (((t - 1) & 31) == 0) {  // draws of steps t .. t+31, one per lane
            const uint4 r = draw4(key, inst, g, static_cast<uint32_t>(t + lane), kPurposeStep);
            rx = r.x;
            ry = r.y;
        }
        // ---- windows X_j = B >> j and Y_j (bit k = b_{j-k}) for j = lane + 32q
        uint32_t X[NW][NW], Y[NW][NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
#pragma unroll
            for (int w = 0; w + q < NW; ++w)
                X[q][w] = __funnelshift_r(B[w + q], (w + q + 1 < NW) ? B[w + q + 1] : 0u, lane);
#pragma unroll
            for (int w = 0; w <= q; ++w)
                Y[q][w] = __funnelshift_r(RL[w + NW - 1 - q], (w + NW - q < NW) ? RL[w + NW - q] : 0u,
                                          31 - lane);
        }
        // ---- S_j on the bit planes of C_k
        uint32_t mx = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) mx = max(mx, static_cast<uint32_t>(abs(c[q])));
        mx = __reduce_max_sync(kFull, mx);
        const int P = 33 - __clz(mx);
        int32_t S[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) S[q] = 0;
        for (int m = 0; m < P; ++m) {
            uint32_t tp[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) tp[w] = __ballot_sync(kFull, (c[w] >> m) & 1);
            const int32_t wm = (m == P - 1) ? -(1 << m) : (1 << m);
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                int s = 0;
#pragma unroll
                for (int w = 0; w + q < NW; ++w) s += __popc(tp[w] & X[q][w]);
#pragma unroll
                for (int w = 0; w <= q; ++w) s += __popc(tp[w] & Y[q][w]);
                S[q] += s * wm;
            }
        }
        // ---- T_j = Total + sum_{i=1}^{j} (C_i - C_{N-i})
#pragma unroll
        for (int q = 0; q < NW; ++q) Cs[lane + 32 * q] = c[q];
        __syncwarp();
        int32_t tot = 0;
        int32_t D[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int i = lane + 32 * q;
            const bool in = i >= 1 && i <= N - 1;
            D[q] = in ? c[q] - Cs[in ? N - i : 0] : 0;
            tot += c[q];
        }
        __syncwarp();
        int32_t carry = __reduce_add_sync(kFull, tot);
        int32_t T[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            int32_t v = D[q];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t n = __shfl_up_sync(kFull, v, o);
                if (lane >= o) v += n;
            }
            T[q] = carry + v;
            carry += __shfl_sync(kFull, v, 31);
        }
        // ---- E_j, admissibility (tabu expired or aspiration), candidates
        const int32_t E0 = E + 4 * (N - 1);
        int32_t cand[NW];
        int32_t lmin = INT_MAX;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int j = lane + 32 * q;
            const int L = min(j, N - 1 - j);
            int dm = 0;
#pragma unroll
            for (int w = 0; w <= q && w + q < NW; ++w) {
                const uint32_t mm = word_lowmask(w, L + 1) & (w == 0 ? ~1u : kFull);
                dm += __popc((X[q][w] ^ Y[q][w]) & mm);
            }
            const int32_t M = L - 2 * dm;
            const int32_t sj = ((B[q] >> lane) & 1u) ? 1 : -1;
            const int32_t Ej = E0 + 8 * M - 4 * sj * (2 * S[q] - T[q]);
            const bool adm = j < N && (tabu[q] < t || Ej < E_best);
            cand[q] = adm ? Ej : INT_MAX;
            lmin = min(lmin, cand[q]);
        }
        const int32_t m = __reduce_min_sync(kFull, lmin);
        if (m == INT_MAX) break;  // unreachable: maxTabu < N leaves a bit free
        uint32_t tb[NW];
        int count = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            tb[q] = __ballot_sync(kFull, cand[q] == m);
            count += __popc(tb[q]);
        }
        const int src = (t - 1) & 31;
        const uint32_t u_tie = __shfl_sync(kFull, rx, src);
        const uint32_t u_ten = __shfl_sync(kFull, ry, src);
        int idx = count > 1 ? static_cast<int>((static_cast<uint64_t>(u_tie) * count) >> 32) : 0;
        int p = 0;
        bool found = false;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int pc = __popc(tb[q]);
            if (!found) {
                if (idx < pc) {
                    p = 32 * q + nth_set_bit(tb[q], idx);
                    found = true;
                } else {
                    idx -= pc;
                }
            }
        }
        // ---- apply: C_k += delta_k(p), flip, tenure, bestSeqTS
        uint32_t Xp[NW], Yp[NW];
        shr_uniform<NW>(B, p, Xp);            // bit k = b_{p+k}
        shr_uniform<NW>(RL, NB - 1 - p, Yp);  // bit k = b_{p-k}
        const int32_t sp = (Xp[0] & 1u) ? 1 : -1;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int k = lane + 32 * q;
            const int32_t bx = (Xp[q] >> lane) & 1u, by = (Yp[q] >> lane) & 1u;
            const int32_t sx = (k >= 1 && k <= N - 1 - p) ? 2 * bx - 1 : 0;
            const int32_t sy = (k >= 1 && k <= p) ? 2 * by - 1 : 0;
            c[q] -= 2 * sp * (sx + sy);
        }
        flip_bit<NW>(B, p);
        flip_bit<NW>(RL, NB - 1 - p);
        const int32_t expiry = t + rand_int(min_t, max_t, u_ten);
#pragma unroll
        for (int q = 0; q < NW; ++q)
            if (lane + 32 * q == p) tabu[q] = expiry;
        E = m;
        if (m < E_best) {
            E_best = m;
#pragma unroll
            for (int w = 0; w < NW; ++w) Bb[w] = B[w];
        }
        ++steps;
        if (trace != nullptr && trace_len < trace_cap) {
            if (lane == 0) trace[trace_len] = make_int4(static_cast<int>(g), t, p, m);
            ++trace_len;
        }
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) seq[w] = Bb[w];
    TabuOut out;
    out.steps = steps;
    out.E_best = E_best;
    return out;
}

}  // namespace lgpu
