// tabu_skew.cuh -- the tabu search restricted to skew-symmetric sequences
// (Sec. II.C), one warp per search.
//
// For odd N with centre c = (N-1)/2, move i (0 <= i <= c) flips b_i and, for
// i < c, its partner b_j, j = N-1-i, so a skew-symmetric pivot stays
// skew-symmetric.  The energy of move i < c comes from the single-flip
// energies E_i, E_j that tabu_core.cuh scores for every bit:
//   E_{ij} = E_i + E_j - E + 16 s_i s_j C_d + 8 s_i s_j R - 32
//            - 16 (s_j s_{i-d} + s_i s_{j+d})        (last term iff 3i >= N-1)
// with d = j - i and R = sum_m s_m s_{N-1-m}.  Derivation: flipping {i, j}
// changes C_k by delta_k(i) + delta_k(j), plus 4 s_i s_j at k = d (both
// deltas negate the product s_i s_j, which keeps its sign); in
// sum_k (C_k + delta_k)^2 the cross sum sum_k delta_k(i) delta_k(j) is
// 4 s_i s_j (C_d + R - 2 s_i s_j), because the products s_{i+k} s_{j+k} and
// s_{i-k} s_{j-k} tile C_d without the pair (i, j), and s_{i+k} s_{j-k},
// s_{i-k} s_{j+k} tile R without it; the k = d correction leaves
// 8 s_i s_j (C_d + delta_d(i) + delta_d(j)) + 16.  The identity holds for any
// sequence.  R is unchanged by every move (s_i s_j and s_c^2 keep their
// signs), so it is computed once per search.  Move c is the single flip E_c.
//
// Per step: correlations from the pivot, all N single-flip energies (bit
// planes, prefix sums, as in tabu_core.cuh), partner energies and C_d read
// through the warp's shared scratch, then the admissible minimum over the
// n = c + 1 moves with the same tabu, aspiration, tie and draw rules.
#pragma once

#include "tabu_core.cuh"

namespace lgpu {

template <int NW, bool TRACE, bool FIX_FIRST>
__device__ TabuOut tabu_search_skew(uint32_t (&seq)[NW], const int N, const uint2 key,
                                    const uint32_t inst, const uint32_t g, const int max_iter,
                                    const int64_t budget, int32_t* __restrict__ Cs,
                                    int4* __restrict__ trace, const int64_t trace_cap,
                                    int64_t& trace_len, const int lane) {
    constexpr int NB = 32 * NW;
    const int c = (N - 1) >> 1;
    uint32_t B[NW], RL[NW], Bb[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        B[w] = seq[w];
        Bb[w] = seq[w];
    }
    reverse_bits<NW>(B, RL);
    int32_t cc[NW];
    correlations<NW>(B, N, lane, cc);
    int32_t E;
    {
        int32_t sq = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) sq += cc[q] * cc[q];
        E = __reduce_add_sync(kFull, sq);
    }
    int32_t E_best = E;
    int32_t R;  // sum_m s_m s_{N-1-m} = N - 2 #{m : b_m != b_{N-1-m}}
    {
        uint32_t RN[NW];
        shr_uniform<NW>(RL, NB - N, RN);
        int diff = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) diff += __popc((B[w] ^ RN[w]) & word_lowmask(w, N));
        R = N - 2 * diff;
    }
    // Per-search constants of the single-flip scoring (see tabu_search) and
    // of the moves i = lane + 32q.
    uint32_t par[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t alt = ((N - 32 * w) & 1) ? 0x55555555u : 0xAAAAAAAAu;
        par[w] = alt & word_lowmask(w, N) & (w == 0 ? ~1u : kFull);
    }
    int32_t tabu[NW], Lq[NW], mir[NW], dq[NW];
    uint32_t mmask[NW][NW];
    uint32_t ivalid = 0;  // bit q: move i = lane + 32q exists and may be taken
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        tabu[q] = 0;
        const int j = lane + 32 * q;
        Lq[q] = min(j, N - 1 - j);
        mir[q] = j < N ? N - 1 - j : 0;
        dq[q] = j <= c ? N - 1 - 2 * j : 0;
        ivalid |= (j <= c && !(FIX_FIRST && j == 0) ? 1u : 0u) << q;
#pragma unroll
        for (int w = 0; w <= q && w + q < NW; ++w)
            mmask[q][w] = word_lowmask(w, Lq[q] + 1) & (w == 0 ? ~1u : kFull);
    }
    const int min_t = max_iter / 10;
    const int max_t = (12 * max_iter) / 100;
    const int64_t nsteps = budget < 0 ? max_iter : (budget < max_iter ? budget : max_iter);
    uint32_t rx = 0, ry = 0;
    int64_t steps = 0;

    for (int t = 1; t <= nsteps; ++t) {
        if (((t - 1) & 31) == 0) {
            const uint4 r = draw4(key, inst, g, static_cast<uint32_t>(t + lane), kPurposeStep);
            rx = r.x;
            ry = r.y;
        }
        const int src = (t - 1) & 31;
        const uint32_t u_tie = __shfl_sync(kFull, rx, src);
        const uint32_t u_ten = __shfl_sync(kFull, ry, src);
        // ---- single-flip energies E_x, x = lane + 32q
        int32_t pc[NW], T[NW], S[NW], Ex[NW];
        prefix_own<NW>(cc, lane, pc);
        mirror_terms<NW>(pc, N, lane, Cs, T);
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
        score_dispatch<NW>(plane_count<NW>(cc), cc, par, X, Y, S);
        const int32_t E0 = E + 4 * (N - 1);
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            int dm = 0;
#pragma unroll
            for (int w = 0; w <= q && w + q < NW; ++w) dm += __popc((X[q][w] ^ Y[q][w]) & mmask[q][w]);
            const int32_t V = 2 * S[q] - T[q];
            Ex[q] = E0 + 8 * (Lq[q] - 2 * dm) - 4 * ((X[q][0] & 1u) ? V : -V);
        }
        // ---- partner energy E_j and C_d of each move, through shared scratch
        int32_t Ej[NW], Cd[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) Cs[lane + 32 * q] = Ex[q];
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NW; ++q) Ej[q] = Cs[mir[q]];
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NW; ++q) Cs[lane + 32 * q] = cc[q];  // C_0 = 0 at k = 0
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NW; ++q) Cd[q] = Cs[dq[q]];
        __syncwarp();
        // ---- move energies, admissibility, candidates
        int32_t cand[NW];
        int32_t lmin = INT_MAX;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int i = lane + 32 * q;
            int32_t Ei = Ex[q];
            if (i < c) {
                const int32_t si = (X[q][0] & 1u) ? 1 : -1;
                const int32_t sj = get_bit<NW>(B, N - 1 - i) ? 1 : -1;
                const int32_t sig = si * sj;
                Ei += Ej[q] - E + 16 * sig * Cd[q] + 8 * sig * R - 32;
                if (3 * i >= N - 1) {
                    const int32_t sa = get_bit<NW>(B, 3 * i - (N - 1)) ? 1 : -1;      // s_{i-d}
                    const int32_t sb = get_bit<NW>(B, 2 * (N - 1) - 3 * i) ? 1 : -1;  // s_{j+d}
                    Ei -= 16 * (sj * sa + si * sb);
                }
            }
            const bool adm = ((ivalid >> q) & 1u) && (tabu[q] < t || Ei < E_best);
            cand[q] = adm ? Ei : INT_MAX;
            lmin = min(lmin, cand[q]);
        }
        const int32_t m = __reduce_min_sync(kFull, lmin);
        if (m == INT_MAX) break;  // unreachable while maxTabu < n - 1
        uint32_t tb[NW];
        int count = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            tb[q] = __ballot_sync(kFull, cand[q] == m);
            count += __popc(tb[q]);
        }
        int idx = static_cast<int>((static_cast<uint64_t>(u_tie) * count) >> 32);
        int p = 0;
        bool found = false;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int pc_q = __popc(tb[q]);
            if (!found) {
                if (idx < pc_q) {
                    p = 32 * q + nth_set_bit(tb[q], idx);
                    found = true;
                } else {
                    idx -= pc_q;
                }
            }
        }
        // ---- apply: flip b_p and its partner, correlations, tenure, bestSeqTS
        flip_bit<NW>(B, p);
        flip_bit<NW>(RL, NB - 1 - p);
        if (p < c) {
            flip_bit<NW>(B, N - 1 - p);
            flip_bit<NW>(RL, NB - N + p);
        }
        correlations<NW>(B, N, lane, cc);
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
        if constexpr (TRACE) {
            if (trace_len < trace_cap) {
                if (lane == 0) trace[trace_len] = make_int4(static_cast<int>(g), t, p, m);
                ++trace_len;
            }
        }
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) seq[w] = Bb[w];
    TabuOut out;
    out.steps = steps;
    out.E_best = E_best;
    out.fault = false;  // one warp per search: nothing to lose step with
    return out;
}

}  // namespace lgpu
