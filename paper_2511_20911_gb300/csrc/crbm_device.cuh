// Device helpers shared by the sweep kernels: the Philox generator, bit
// access on packed words, and the per-sweep measurement / correlation steps.
#pragma once

#include "crbm_internal.h"

namespace crbm {
namespace dev {

struct U4 {
    uint32_t x, y, z, w;
};

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies by the round multipliers, the high halves XORed with
// the other two counter words and the round key; the key advances by the two
// Weyl increments between rounds.
__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c0;
        const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c2;
        const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
        c1 = static_cast<uint32_t>(p1);
        c3 = static_cast<uint32_t>(p0);
        c0 = n0;
        c2 = n2;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return {c0, c1, c2, c3};
}

// Rounds 3..9 from the state after round 2, with precomputed round keys
// rk[2r] = k0 + r W0, rk[2r+1] = k1 + r W1 (kernel parameters, so each key is
// a constant-bank operand of its XOR).
__device__ __forceinline__ U4 philox_rounds3to9(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                const uint32_t (&rk)[20]) {
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c0;
        const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c2;
        const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ rk[2 * r];
        const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ rk[2 * r + 1];
        c1 = static_cast<uint32_t>(p1);
        c3 = static_cast<uint32_t>(p0);
        c0 = n0;
        c2 = n2;
    }
    return {c0, c1, c2, c3};
}

// Round 1 of the sweep-keyed counters, split by what varies.  After round 0
// the state is (X, Y, c2, c3) with X, Y fixed for a lane in a sweep and
// (c2, c3) = (hi(M0 cell) ^ key1 ^ tag, lo(M0 cell)).  Round 1 multiplies X
// (once per sweep: Round1Sweep) and c2 (per call); its second output word
// hi(M0 X) ^ c3 ^ rk3 is shared by all calls of a cell.
struct Round1Sweep {
    uint32_t lo;   // lo(M0 X): word 3 after round 1
    uint32_t hik;  // hi(M0 X) ^ rk[3]
};
__device__ __forceinline__ Round1Sweep round1_sweep(uint32_t X, const uint32_t (&rk)[20]) {
    const uint64_t p = static_cast<uint64_t>(kPhiloxM0) * X;
    return {static_cast<uint32_t>(p), static_cast<uint32_t>(p >> 32) ^ rk[3]};
}
// Round 2 multiplies word 2 after round 1, which is the cell's n2 for every
// call of the cell: its product is formed once per cell.
struct Round2Cell {
    uint32_t hi, lo;  // M1 n2
};
__device__ __forceinline__ Round2Cell round2_cell(uint32_t n2) {
    const uint64_t p = static_cast<uint64_t>(kPhiloxM1) * n2;
    return {static_cast<uint32_t>(p >> 32), static_cast<uint32_t>(p)};
}
// The full Philox-4x32-10 output for round-0 state (X, Y, c2, c3) of a call,
// given r1 = round1_sweep(X) and r2 = round2_cell(r1.hik ^ c3).
__device__ __forceinline__ U4 philox_from_round2(uint32_t Y, const Round1Sweep& r1, const Round2Cell& r2,
                                                 uint32_t c2, const uint32_t (&rk)[20]) {
    const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c2;             // round 1
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ Y ^ rk[2];
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * n0;             // round 2
    return philox_rounds3to9(r2.hi ^ static_cast<uint32_t>(p1) ^ rk[4], r2.lo,
                             static_cast<uint32_t>(p0 >> 32) ^ r1.lo ^ rk[5], static_cast<uint32_t>(p0), rk);
}

// Round 1's product M1 c2 of a call: c2 = hi(M0 cell) ^ key1 ^ tag is the
// same for every lane, so its product can be formed once per (cell, tag),
// on the host for the record-driven sweeps.  Stored XORed with the round keys
// it meets: (hi ^ rk2, lo ^ rk4).
struct Round1Call {
    uint32_t h, l;
};
__device__ __forceinline__ Round1Call round1_call(uint32_t c2, const uint32_t (&rk)[20]) {
    const uint64_t p = static_cast<uint64_t>(kPhiloxM1) * c2;
    return {static_cast<uint32_t>(p >> 32) ^ rk[2], static_cast<uint32_t>(p) ^ rk[4]};
}
// The full Philox-4x32-10 output of a call from r1 = round1_sweep(X), the
// cell's r2 = round2_cell(r1.hik ^ c3) and the call's q = round1_call(c2).
__device__ __forceinline__ U4 philox_from_call(uint32_t Y, const Round1Sweep& r1, const Round2Cell& r2,
                                               const Round1Call& q, const uint32_t (&rk)[20]) {
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * (q.h ^ Y);     // round 2
    return philox_rounds3to9(r2.hi ^ q.l, r2.lo, static_cast<uint32_t>(p0 >> 32) ^ r1.lo ^ rk[5],
                             static_cast<uint32_t>(p0), rk);
}

// Round 0 of counter (cell, sweep, chain, tag) needs no per-call multiply:
// M1 * chain is a per-lane constant, M0 * cell is warp-uniform.  The state
// after round 0 is (hi(M1 chain) ^ sweep ^ rk0, lo(M1 chain),
// hi(M0 cell) ^ tag ^ rk1, lo(M0 cell)).
struct Round0Lane {
    uint32_t hi, lo;
};
struct Round0Cell {
    uint32_t a, b;  // hi(M0 cell) ^ rk1, lo(M0 cell)
};
__device__ __forceinline__ Round0Lane round0_lane(uint32_t chain) {
    const uint64_t p = static_cast<uint64_t>(kPhiloxM1) * chain;
    return {static_cast<uint32_t>(p >> 32), static_cast<uint32_t>(p)};
}
__device__ __forceinline__ Round0Cell round0_cell(uint32_t cell, uint32_t rk1) {
    const uint64_t p = static_cast<uint64_t>(kPhiloxM0) * cell;
    return {static_cast<uint32_t>(p >> 32) ^ rk1, static_cast<uint32_t>(p)};
}

__device__ __forceinline__ uint32_t pick(const U4& q, int w) {
    return w == 0 ? q.x : (w == 1 ? q.y : (w == 2 ? q.z : q.w));
}

__device__ __forceinline__ uint32_t bit_of(uint32_t word, int lane) { return (word >> lane) & 1u; }

__device__ __forceinline__ uint32_t rotr(uint32_t x, uint32_t s) { return __funnelshift_r(x, x, s); }

// Release store of a progress counter in global memory.
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Persistent scheduling of (word, chunk of sweeps) items: state[w] = 2 (chunks
// of w done) + (1 while a CTA holds w), as k_sweep_canon_persistent keeps it
// (which has the same loop inline: its sweep compiles faster that way).
// Called by one whole warp: claims,
// with a compare-and-swap on state, the free word with the fewest chunks done
// (all states scanned with 16-byte loads; ties go to the first word in the
// scan order that starts at `start`).  Every lane returns the word (-1 when
// every unfinished word is held by a running CTA, which claims again after
// its chunk, so no work is left behind and nothing waits) and its chunk.
__device__ __forceinline__ void claim_word(int* state, int nw, int n_chunks, unsigned int start, int lane,
                                           int& word, int& chunk) {
    const int nq = (nw + 3) / 4;
    word = -1;
    chunk = 0;
    for (int tries = 0; tries < (1 << 20) && word < 0; ++tries) {
        int best = 0x7fffffff, bk = 0x7fffffff, bw = -1;  // (chunks done, scan rank, word)
        for (int q = lane; q < nq; q += 32) {
            const int4 v = __ldcg(reinterpret_cast<const int4*>(state) + q);
            const int sv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int w = 4 * q + j;
                const int dw = sv[j] >> 1;
                const int rank =
                    static_cast<int>((static_cast<unsigned int>(w) + nw - start) % static_cast<unsigned int>(nw));
                if (w < nw && (sv[j] & 1) == 0 && dw < n_chunks && (dw < best || (dw == best && rank < bk))) {
                    best = dw;
                    bk = rank;
                    bw = w;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
            const int ow = __shfl_xor_sync(0xffffffffu, bw, o);
            if (ob < best || (ob == best && ok < bk)) {
                best = ob;
                bk = ok;
                bw = ow;
            }
        }
        if (bw < 0) break;
        if (lane == 0 && atomicCAS(state + bw, 2 * best, 2 * best + 1) == 2 * best) {
            __threadfence();  // acquire: the previous chunk's stores precede its release
            word = bw;
            chunk = best;
        }
        word = __shfl_sync(0xffffffffu, word, 0);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
    }
}

// Countdown to the sweeps t with (t + 1) % k == 0 (the sweeps after which a
// measurement, a swap round or a correlation sample is taken), started at
// sweep t0, so that the sweep loop needs no integer division per sweep.
// k <= 0: never.  step() answers for the current sweep and moves on to the
// next; every thread calls it once per sweep.
struct EveryCounter {
    int left, k;  // sweeps after the current one before the next hit (k <= 0: negative, never 0)
    __device__ __forceinline__ EveryCounter(uint32_t t0, int k_)
        : left(k_ > 0 ? static_cast<int>(static_cast<uint32_t>(k_) - 1u - t0 % static_cast<uint32_t>(k_)) : -1),
          k(k_) {}
    __device__ __forceinline__ bool step() {
        const bool hit = left == 0;
        left = hit ? k - 1 : left - 1;
        return hit;
    }
};

__device__ __forceinline__ int warp_sum(int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Time to solution: the first measured sweep at or below the chain's target
// energy (kept out of line: it runs only at measurements and only when
// targets are set, and should not add to the sweep loop's registers).
static __device__ __noinline__ void record_first_hit(int64_t* hit, const int32_t* hit_q, uint32_t row, int64_t nJ,
                                              int64_t nP, int64_t M, uint32_t t) {
    int64_t* ht = hit + 2 * static_cast<size_t>(row);
    const int32_t* q = hit_q + 4 * static_cast<size_t>(row);
    const int64_t E = static_cast<int64_t>(q[0]) * nJ + static_cast<int64_t>(q[1]) * nP - static_cast<int64_t>(q[2]) * M;
    if (ht[1] < 0 && E <= ht[0]) ht[1] = static_cast<int64_t>(t) + 1;
}

// Post-sweep step of the SMEM kernels, run by one warp (the one that keeps
// the running sums) after every warp has added its per-lane counts to s_cnt ([0..31] anti-aligned J filters, [32..63]
// anti-aligned J' filters, [64..95] +1 spins; lane = replica slot).  Lane k
// then stands for temperature rung k, held by slot s_sob[k] (the identity
// without tempering):
//  - measurement: rung k's (NJ, NJ', M) go to series row 32 word + k and are
//    added to the running sums s_acc[x][k] (shared memory, so that they hold
//    no registers through the sweep loop);
//  - replica exchange (round m): pairs (k, k+1) with k = m (mod 2) swap rungs
//    when E_k <= E_{k+1}, else when a Philox word (k, m, word, swap tag) is
//    below the host-built threshold of nearbyint(2^32 exp((b_k - b_{k+1}) dE / 16)).
__device__ __forceinline__ void post_sweep_warp(const SweepArgs& a, int* s_cnt, int* s_sob,
                                                 int* s_bos, int lane, int word, uint32_t t,
                                                 bool do_meas, bool do_swap, int64_t meas,
                                                 int64_t* s_acc) {
    const Geometry& g = a.g;
    const int nJr = g.n_real_bonds[0] - 2 * s_cnt[lane];
    const int nPr = g.n_real_bonds[1] - 2 * s_cnt[32 + lane];
    const int Mr = 2 * s_cnt[64 + lane] - g.N;
    s_cnt[lane] = 0;
    s_cnt[32 + lane] = 0;
    s_cnt[64 + lane] = 0;
    const int k = lane;
    const int slot = s_sob[k];
    const int64_t nJ = __shfl_sync(0xffffffffu, nJr, slot);
    const int64_t nP = __shfl_sync(0xffffffffu, nPr, slot);
    const int64_t M = __shfl_sync(0xffffffffu, Mr, slot);
    if (do_meas) {
        const uint32_t row = static_cast<uint32_t>(word) * 32u + k;
        if (meas < a.series_len) {
            int32_t* e = a.series + (static_cast<size_t>(meas) * a.n_chains_padded + row) * 3;
            e[0] = static_cast<int32_t>(nJ);
            e[1] = static_cast<int32_t>(nP);
            e[2] = static_cast<int32_t>(M);
        }
        int64_t* acc = s_acc + k;
        acc[0 * 32] += 1;
        acc[1 * 32] += nJ;
        acc[2 * 32] += nP;
        acc[3 * 32] += M;
        acc[4 * 32] += M < 0 ? -M : M;
        acc[5 * 32] += nJ * nJ;
        acc[6 * 32] += nP * nP;
        acc[7 * 32] += M * M;
        acc[8 * 32] += nJ * nP;
        acc[9 * 32] += nJ * M;
        acc[10 * 32] += nP * M;
        if (a.hit) record_first_hit(a.hit, a.hit_q, row, nJ, nP, M, t);
    }
    if (do_swap) {
        const int32_t* q = a.wq + 3 * word;
        const long long E = static_cast<long long>(q[0]) * nJ + static_cast<long long>(q[1]) * nP -
                            static_cast<long long>(q[2]) * M;
        const long long E1 = __shfl_down_sync(0xffffffffu, E, 1);
        const uint32_t m = (t + 1u) / static_cast<uint32_t>(a.swap_every) - 1u;
        bool accept = false;
        if (k < 31 && (static_cast<uint32_t>(k) & 1u) == (m & 1u)) {
            const long long D = E - E1;
            if (D <= 0) {
                accept = true;
            } else {
                const int idx = word * 32 + k;
                if (D < a.swap_len[idx]) {
                    const U4 u = philox(static_cast<uint32_t>(k), m, static_cast<uint32_t>(word), kTagSwap,
                                        a.key0, a.key1);
                    accept = u.x < a.swap_tab[a.swap_off[idx] + D];
                }
            }
        }
        const uint32_t am = __ballot_sync(0xffffffffu, accept);
        const int up = __shfl_down_sync(0xffffffffu, slot, 1);
        const int dn = __shfl_up_sync(0xffffffffu, slot, 1);
        int ns = slot;
        if ((am >> k) & 1u)
            ns = up;
        else if (k > 0 && ((am >> (k - 1)) & 1u))
            ns = dn;
        s_sob[k] = ns;
        s_bos[ns] = k;
    }
}

// Spin correlations of Sec. IV.B for the chains of each parameter-point
// segment of this word:  C_p(d) += n_p N - 2 sum_r popc((v_r ^ v_{r+d}) & mask_p).
// C_p(d) = C_p(-d), so only row offsets dR <= L/2 are counted and each count
// with 0 < dR < L - dR is added at -d as well.  Work items are (dR, slice of
// rows R); in an item, lane j holds the column offsets dC = j + 32 k and
// walks the row pairs (R, R + dR): the word at (R, C) is a broadcast, the one
// at (R + dR, C + dC) a conflict-free gather, and each XOR word is counted
// for two segments at once.
static __device__ __forceinline__ void accumulate_correlations_word(const SweepArgs& a, const uint32_t* s_v,
                                                                    const int* s_seg, const uint32_t* s_segmask,
                                                                    int warp, int nwarp, int lane) {
    const int L = a.g.L, N = a.g.N, nseg = s_seg[0];
    const int n_dr = L / 2 + 1;
    const int slices = max(1, min(L, (3 * nwarp + n_dr - 1) / n_dr));  // about three items per warp
    const int n_items = n_dr * slices;
    constexpr int kMaxK = 3;  // column offsets per lane: L <= 96 in the SMEM layout
    if (L <= 32) {  // one column offset per lane; lanes >= L count a valid column and drop it
        for (int item = warp; item < n_items; item += nwarp) {
            const int dR = item / slices, sl = item - (item / slices) * slices;
            const int R_begin = sl * L / slices, R_end = (sl + 1) * L / slices;
            const bool mirror = dR > 0 && 2 * dR != L;
            for (int s0 = 0; s0 < nseg; s0 += 2) {
                const uint32_t m0 = s_segmask[s0], m1 = s0 + 1 < nseg ? s_segmask[s0 + 1] : 0u;
                int c0 = 0, c1 = 0;
                for (int R = R_begin; R < R_end; ++R) {
                    const int R2 = R + dR >= L ? R + dR - L : R + dR;
                    const uint32_t* row = s_v + R * L;
                    const uint32_t* row2 = s_v + R2 * L;
                    int C2 = lane < L ? lane : 0;
#pragma unroll 3
                    for (int C = 0; C < L; ++C) {
                        const uint32_t x = row[C] ^ row2[C2];
                        c0 += __popc(x & m0);
                        c1 += __popc(x & m1);
                        C2 = C2 + 1 == L ? 0 : C2 + 1;
                    }
                }
                if (lane < L) {
                    const long long sites = static_cast<long long>(R_end - R_begin) * L;
                    for (int j = 0; j < 2 && s0 + j < nseg; ++j) {
                        const uint32_t mask = j ? m1 : m0;
                        const int p = s_seg[1 + s0 + j] >> 8;
                        const unsigned long long val =
                            static_cast<unsigned long long>(__popc(mask) * sites - 2LL * (j ? c1 : c0));
                        unsigned long long* cp =
                            reinterpret_cast<unsigned long long*>(a.corr + static_cast<size_t>(p) * N);
                        atomicAdd(cp + dR * L + lane, val);
                        if (mirror) atomicAdd(cp + (L - dR) * L + (lane == 0 ? 0 : L - lane), val);
                    }
                }
            }
        }
        return;
    }
    for (int item = warp; item < n_items; item += nwarp) {
        const int dR = item / slices, sl = item - (item / slices) * slices;
        const int R_begin = sl * L / slices, R_end = (sl + 1) * L / slices;
        const bool mirror = dR > 0 && 2 * dR != L;
        for (int s0 = 0; s0 < nseg; s0 += 2) {
            const uint32_t m0 = s_segmask[s0], m1 = s0 + 1 < nseg ? s_segmask[s0 + 1] : 0u;
            int c0[kMaxK], c1[kMaxK];
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) c0[k] = c1[k] = 0;
            for (int R = R_begin; R < R_end; ++R) {
                const int R2 = R + dR >= L ? R + dR - L : R + dR;
                const uint32_t* row = s_v + R * L;
                const uint32_t* row2 = s_v + R2 * L;
                for (int C = 0; C < L; ++C) {
                    const uint32_t x0 = row[C];
#pragma unroll
                    for (int k = 0; k < kMaxK; ++k) {
                        const int dC = lane + 32 * k;
                        if (k * 32 < L && dC < L) {
                            const int C2 = C + dC >= L ? C + dC - L : C + dC;
                            const uint32_t x = x0 ^ row2[C2];
                            c0[k] += __popc(x & m0);
                            c1[k] += __popc(x & m1);
                        }
                    }
                }
            }
            const long long sites = static_cast<long long>(R_end - R_begin) * L;
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) {
                const int dC = lane + 32 * k;
                if (k * 32 >= L || dC >= L) continue;
                for (int j = 0; j < 2 && s0 + j < nseg; ++j) {
                    const uint32_t mask = j ? m1 : m0;
                    const int p = s_seg[1 + s0 + j] >> 8;
                    const unsigned long long val = static_cast<unsigned long long>(
                        __popc(mask) * sites - 2LL * (j ? c1[k] : c0[k]));
                    unsigned long long* cp = reinterpret_cast<unsigned long long*>(a.corr + static_cast<size_t>(p) * N);
                    atomicAdd(cp + dR * L + dC, val);
                    if (mirror) atomicAdd(cp + (L - dR) * L + (dC == 0 ? 0 : L - dC), val);
                }
            }
        }
    }
}

// The same correlations for a square lattice of even side kL <= 32, in
// bit-transposed form: the lattice is first transposed so that lane l holds,
// for every row R, the kL spins of chain l as a kL-bit mask (rows in
// `scratch`, [kL][32] words of the caller's dead shared memory).  Work items
// are (dR, slice of rows R); in an item lane l counts, for every column offset
// dC, the sites at which row R of chain l and row R + dR rotated by dC differ
// (the rotation is one funnel shift of the row written twice side by side),
// and the counts of a parameter point's chains are summed by one warp
// reduction over the point's lane mask.  Every thread of the CTA calls it.
template <int kL>
static __device__ __forceinline__ void accumulate_correlations_bits(const SweepArgs& a, const uint32_t* s_v,
                                                             uint32_t* scratch, const int* s_seg,
                                                             const uint32_t* s_segmask, int warp, int nwarp,
                                                             int lane) {
    static_assert(kL % 2 == 0 && kL >= 4 && kL <= 32, "even side up to 32");
    constexpr int N = kL * kL, n_dr = kL / 2 + 1;
    constexpr uint32_t kFull = kL == 32 ? 0xffffffffu : (1u << (kL % 32)) - 1u;
    for (int R = warp; R < kL; R += nwarp) {
        const uint32_t* row = s_v + R * kL;
        uint32_t m = 0u;
#pragma unroll
        for (int C = 0; C < kL; ++C) m |= ((row[C] >> lane) & 1u) << C;
        scratch[R * 32 + lane] = m;
    }
    // this lane's parameter point: its lane mask, index and whether it reports
    const int nseg = s_seg[0];
    uint32_t smask = 1u << lane;
    int p = -1;
    for (int s = 0; s < nseg; ++s)
        if ((s_segmask[s] >> lane) & 1u) {
            smask = s_segmask[s];
            p = s_seg[1 + s] >> 8;
        }
    const bool leader = p >= 0 && (smask & ((1u << lane) - 1u)) == 0u;  // the point's lowest lane
    const long long n_pt = __popc(smask);
    unsigned long long* cp = reinterpret_cast<unsigned long long*>(a.corr) + static_cast<size_t>(p < 0 ? 0 : p) * N;
    __syncthreads();
    const int slices = max(1, min(kL, (nwarp + n_dr - 1) / n_dr));
    const int n_items = n_dr * slices;
    for (int item = warp; item < n_items; item += nwarp) {
        const int dR = item / slices, sl = item - (item / slices) * slices;
        const int R_begin = sl * kL / slices, R_end = (sl + 1) * kL / slices;
        const bool mirror = dR > 0 && 2 * dR != kL;
        uint32_t cnt[kL];
#pragma unroll
        for (int d = 0; d < kL; ++d) cnt[d] = 0u;
        for (int R = R_begin; R < R_end; ++R) {
            const int R2 = R + dR >= kL ? R + dR - kL : R + dR;
            const uint32_t x = scratch[R * 32 + lane], y = scratch[R2 * 32 + lane];
            const uint32_t lo = kL == 32 ? y : (y | (y << (kL % 32))), hi = kL == 32 ? y : (y >> ((32 - kL) % 32));
#pragma unroll
            for (int d = 0; d < kL; ++d) cnt[d] += __popc((x ^ __funnelshift_r(lo, hi, d)) & kFull);
        }
        const long long sites = static_cast<long long>(R_end - R_begin) * kL;
#pragma unroll
        for (int d = 0; d < kL; ++d) {
            const uint32_t diff = __reduce_add_sync(smask, cnt[d]);
            if (leader) {
                const unsigned long long val = static_cast<unsigned long long>(n_pt * sites - 2LL * diff);
                atomicAdd(cp + dR * kL + d, val);
                if (mirror) atomicAdd(cp + (kL - dR) * kL + (d == 0 ? 0 : kL - d), val);
            }
        }
    }
}

// Correlations of one word: the bit-transposed form for even square sides up
// to 32 when the caller has scratch space, else the word-parallel one (one
// call site in the sweep kernels, out of line: it runs every sq_every sweeps).
static __device__ __noinline__ void accumulate_correlations_any(const SweepArgs& a, const uint32_t* s_v,
                                                                   uint32_t* scratch, const int* s_seg,
                                                                   const uint32_t* s_segmask, int warp, int nwarp,
                                                                   int lane) {
    switch (scratch ? a.g.L : 0) {
#define CRBM_CORR_BITS(k) \
    case k: accumulate_correlations_bits<k>(a, s_v, scratch, s_seg, s_segmask, warp, nwarp, lane); return;
        CRBM_CORR_BITS(4) CRBM_CORR_BITS(6) CRBM_CORR_BITS(8) CRBM_CORR_BITS(10) CRBM_CORR_BITS(12)
        CRBM_CORR_BITS(14) CRBM_CORR_BITS(16) CRBM_CORR_BITS(18) CRBM_CORR_BITS(20) CRBM_CORR_BITS(22)
        CRBM_CORR_BITS(24) CRBM_CORR_BITS(26) CRBM_CORR_BITS(28) CRBM_CORR_BITS(30) CRBM_CORR_BITS(32)
#undef CRBM_CORR_BITS
        default: accumulate_correlations_word(a, s_v, s_seg, s_segmask, warp, nwarp, lane);
    }
}

}  // namespace dev
}  // namespace crbm
