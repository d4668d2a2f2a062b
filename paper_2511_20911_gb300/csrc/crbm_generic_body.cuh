// Body of the generic SMEM-resident sweep (any filter list <= 16 filters, odd
// L, open boundaries; one CTA = one 32-chain word), shared by the
// single-context kernel (crbm_kernels.cu) and the batched kernel
// (crbm_batch.cu).
#pragma once

#include "crbm_device.cuh"

namespace crbm {
namespace generic {

using namespace dev;

// Byte-addressed shared-memory access (records hold byte offsets from the
// start of dynamic shared memory).
__device__ __forceinline__ uint32_t lds32(const char* sm, uint32_t off) {
    return *reinterpret_cast<const uint32_t*>(sm + off);
}
__device__ __forceinline__ uint32_t lds16(const char* sm, uint32_t off) {
    return *reinterpret_cast<const uint16_t*>(sm + off);
}

// w | bit when q < t: a compare and a predicated OR.
__device__ __forceinline__ uint32_t or_if_less(uint32_t w, uint32_t q, uint32_t t, uint32_t bit) {
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
        : "+r"(w)
        : "r"(q), "r"(t), "r"(bit));
    return w;
}

// Generic hidden half-step of one cell (Eq. 9): filter k of the cell reads
// its two endpoint words (the zero word for a zero-padded endpoint, whose
// pad pattern selects table rows that give it no weight), moves the lane's
// bits to address bits 7 and 8 of its table rows [cls][pad][e1 + 2 e2]
// (coefficient sign folded in by the host) and compares the threshold with
// its Philox word.  The lane's decisions go to a 16-bit word, bit k =
// filter k, in row `cell` of the hidden words.
// Draws: Philox-4x32-10 of counter (cell, sweep, chain, tag) from the split
// rounds (crbm_device.cuh): rs = round1_sweep of the lane's sweep word, Y the
// lane's chain word, rk the round keys.  kPaper (CRBM_PRECISION_PAPER, at most
// ten filters): filter k < 8 takes half k & 1 of word k >> 1 of tag 0, filters
// 8 and 9 the halves of word 0 of tag 1, each compared as the upper half of a
// 32-bit word against the 16-bit threshold in the table entry's upper half.
template <bool kPaper>
__device__ __forceinline__ void hidden_cell_generic(const Geometry& g, char* sm, const uint4* __restrict__ rh,
                                                    uint32_t hw_byte, int cell, const Round1Sweep& rs, uint32_t Y,
                                                    const uint32_t (&rk)[20], uint32_t lm, uint32_t rot0,
                                                    uint32_t rot1, uint32_t lb, int lane) {
    const Round0Cell rc = round0_cell(static_cast<uint32_t>(cell), rk[1]);
    const Round2Cell r2 = round2_cell(rs.hik ^ rc.b);
    const uint4* r = rh + static_cast<size_t>(cell) * g.nb;
    uint32_t h = 0u;
    if (kPaper) {
        const U4 q0 = philox_from_round2(Y, rs, r2, rc.a, rk);
        const U4 q1 = g.nb > 8 ? philox_from_round2(Y, rs, r2, rc.a ^ 1u, rk) : U4{0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            if (k < g.nb) {
                const uint32_t word = k < 8 ? pick(q0, k >> 1) : q1.x;
                const uint4 e = __ldg(r + k);
                const uint32_t a = rotr(lds32(sm, e.x) & lm, rot0), b = rotr(lds32(sm, e.y) & lm, rot1);
                h = or_if_less(h, (k & 1) ? word : word << 16, lds32(sm, e.z + (a | b | lb)), 1u << k);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {  // call c draws for filters 4c .. 4c + 3
        if (!kPaper && c < g.n_calls) {
            const U4 q = philox_from_round2(Y, rs, r2, rc.a ^ static_cast<uint32_t>(c), rk);
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int k = 4 * c + x;
                if (k < g.nb) {
                    const uint4 e = __ldg(r + k);
                    const uint32_t a = rotr(lds32(sm, e.x) & lm, rot0), b = rotr(lds32(sm, e.y) & lm, rot1);
                    h = or_if_less(h, pick(q, x), lds32(sm, e.z + (a | b | lb)), 1u << k);
                }
            }
        }
    }
    *reinterpret_cast<uint16_t*>(sm + hw_byte + 64u * static_cast<uint32_t>(cell) + 2u * lane) =
        static_cast<uint16_t>(h);
}

// Generic visible half-step of one cell (Eq. 10): the cell's spins take
// their filters from the hidden rows of at most four cells (own, above,
// left, above-left).  Each row's 16-bit word h is expanded to
// h | (h ^ f) << 16 (f: the filters whose class coefficient is -1 for this
// lane), so that bit k is the term of filter k at its first endpoint and bit
// 16 + k at its second; a spin's n_J, n_J' are then 2 popc(masked) - degree,
// and its table row is the record's row of n = -degree plus
// 2 (2 DJp + 1) popc_J + 2 popc_J'.  kPaper: the spin at window offset x =
// 2r + c takes half x & 1 of word 1 + (x >> 1) of tag 1.
template <bool kPaper>
__device__ __forceinline__ void visible_cell_generic(char* sm, const uint4* __restrict__ rv, int cell,
                                                     const Round1Sweep& rs, uint32_t Y, const uint32_t (&rk)[20],
                                                     uint32_t sflip, uint32_t stepJ, uint32_t lb, int lane) {
    const uint4* r = rv + static_cast<size_t>(cell) * kGenVisRec;
    const Round0Cell rc = round0_cell(static_cast<uint32_t>(cell), rk[1]);
    const U4 q = philox_from_round2(Y, rs, round2_cell(rs.hik ^ rc.b), rc.a ^ (kPaper ? 1u : kTagVis), rk);
    const uint4 src = __ldg(r);
    const uint32_t l2 = 2u * static_cast<uint32_t>(lane);
    uint32_t w[4];
    w[0] = lds16(sm, src.x + l2);
    w[1] = lds16(sm, src.y + l2);
    w[2] = lds16(sm, src.z + l2);
    w[3] = lds16(sm, src.w + l2);
#pragma unroll
    for (int s = 0; s < 4; ++s) w[s] |= (w[s] ^ sflip) << 16;
    const uint4 tb = __ldg(r + 9), so = __ldg(r + 10);
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const uint4 mj = __ldg(r + 1 + 2 * x), mp = __ldg(r + 2 + 2 * x);
        const uint32_t cj = __popc(w[0] & mj.x) + __popc(w[1] & mj.y) + __popc(w[2] & mj.z) + __popc(w[3] & mj.w);
        const uint32_t cp = __popc(w[0] & mp.x) + __popc(w[1] & mp.y) + __popc(w[2] & mp.z) + __popc(w[3] & mp.w);
        const uint32_t row = (x == 0 ? tb.x : x == 1 ? tb.y : x == 2 ? tb.z : tb.w) + cj * stepJ + (cp << 8);
        const uint32_t u = kPaper ? ((x & 1) ? pick(q, 1 + (x >> 1)) : pick(q, 1 + (x >> 1)) << 16) : pick(q, x);
        const uint32_t vw = __ballot_sync(0xffffffffu, u < lds32(sm, row + lb));
        *reinterpret_cast<uint32_t*>(sm + (x == 0 ? so.x : x == 1 ? so.y : x == 2 ? so.z : so.w)) = vw;
    }
}

// Per-lane counts of one cell for the energy/magnetisation measurement:
// anti[cls] = number of anti-aligned real bonds of the cell's filters.
__device__ __forceinline__ void count_cell(const Geometry& g, const uint32_t* s_v,
                                           const uint32_t* __restrict__ ep, int cell, int lane, int& anti0,
                                           int& anti1) {
    const uint32_t* e = ep + static_cast<size_t>(cell) * g.nb;
#pragma unroll
    for (int k = 0; k < kMaxBonds; ++k) {
        if (k < g.nb) {
            const uint32_t ek = __ldg(e + k);
            if ((ek & 0x80008000u) == 0x80008000u) {
                const int x = static_cast<int>(bit_of(s_v[ek & 0x7FFFu] ^ s_v[(ek >> 16) & 0x7FFFu], lane));
                if (g.cls[k]) anti1 += x; else anti0 += x;
            }
        }
    }
}

// Generic SMEM-resident sweep: one CTA per packed word (32 chains), the whole
// lattice, hidden layer and threshold columns in shared memory, all n_sweeps
// sweeps on device.  Warps split the cells of each half-step; __syncthreads
// separates the half-steps (hidden reads v / writes h; visible reads h /
// writes v).  kPaper: CRBM_PRECISION_PAPER draws (see the cores).
template <bool kPaper>
__device__ __forceinline__ void sweep_generic_body(const SweepArgs& a, int word) {
    extern __shared__ __align__(16) uint32_t smem[];
    const Geometry& g = a.g;
    const GenericSmem gs = generic_smem(g);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    char* sm = reinterpret_cast<char*>(smem);
    int64_t* s_acc = reinterpret_cast<int64_t*>(smem);  // [kNSum][32] running sums
    uint32_t* s_tab = smem + gs.tab;
    uint32_t* s_v = smem + gs.v;
    int* s_cnt = reinterpret_cast<int*>(smem + gs.cnt);            // [3][32]
    int* s_seg = reinterpret_cast<int*>(smem + gs.seg);            // [33]
    uint32_t* s_segmask = smem + gs.segmask;                       // [32]
    int* s_sob = reinterpret_cast<int*>(smem + gs.sob);            // [32] slot of each rung
    int* s_bos = s_sob + 32;                                        // [32] rung of each slot
    const int nTg = kGenHid + g.n_vis_tab * g.nTv;
    const uint4* rh = a.crec;                                           // [n_cells][nb] hidden records
    const uint4* rv = a.crec + static_cast<size_t>(g.n_cells) * g.nb;  // [n_cells][kGenVisRec]
    const uint32_t hw_byte = 4u * static_cast<uint32_t>(gs.hw);

    const uint32_t* gtab = a.tab + static_cast<size_t>(word) * nTg * 32;
    for (int x = threadIdx.x; x < nTg * 32; x += blockDim.x) s_tab[x] = gtab[x];
    uint32_t* gv = a.v + static_cast<size_t>(word) * g.N;
    for (int x = threadIdx.x; x < g.N; x += blockDim.x) s_v[x] = gv[x];
    if (threadIdx.x < 2) s_v[g.N + threadIdx.x] = 0u;                  // zero word, scratch word
    if (threadIdx.x < 16) smem[gs.zrow + threadIdx.x] = 0u;            // zero hidden row
    for (int x = threadIdx.x; x < 96; x += blockDim.x) s_cnt[x] = 0;
    if (a.sq_every > 0) {
        for (int x = threadIdx.x; x < 33; x += blockDim.x) s_seg[x] = a.seg[word * 33 + x];
        for (int x = threadIdx.x; x < 32; x += blockDim.x) s_segmask[x] = a.segmask[word * 32 + x];
    }
    const uint32_t sn[2] = {bit_of(a.sneg[2 * word], lane), bit_of(a.sneg[2 * word + 1], lane)};
    uint32_t sflip = 0u;  // filters whose class coefficient is -1 for this lane
    for (int k = 0; k < g.nb; ++k) sflip |= (g.cls[k] ? sn[1] : sn[0]) << k;
    const uint32_t lm = 1u << lane;
    const uint32_t rot0 = static_cast<uint32_t>(lane - 7) & 31u, rot1 = static_cast<uint32_t>(lane - 8) & 31u;
    const uint32_t stepJ = 256u * static_cast<uint32_t>(2 * g.DJp + 1);
    const uint32_t chain = static_cast<uint32_t>(word) * 32u + lane;
    if (warp == 0) {  // replica permutation (identity without tempering)
        const int sob = a.swap_every > 0 ? a.sob[word * 32 + lane] : lane;
        s_sob[lane] = sob;
        s_bos[sob] = lane;
    }
    __syncthreads();
    uint32_t lb = 4u * static_cast<uint32_t>(s_bos[lane]);  // threshold column: the rung this slot holds
    const bool measuring = a.measure_every > 0;
    if (warp == 0 && measuring) {
        for (int x = 0; x < kNSum; ++x) s_acc[x * 32 + lane] = a.sums[static_cast<size_t>(chain) * kNSum + x];
    }
    // sweep and measurement counters: kernel arguments, or the batch's device clock
    const uint32_t t0 = a.clock ? static_cast<uint32_t>(a.clock[0]) : a.t0;
    int64_t meas = a.clock ? a.clock[1] : a.meas0;

    const Round0Lane r0l = round0_lane(chain);
    EveryCounter every_meas(t0, a.measure_every), every_swap(t0, a.swap_every), every_sq(t0, a.sq_every);
    for (int it = 0; it < a.n_sweeps; ++it) {
        const uint32_t t = t0 + static_cast<uint32_t>(it);
        const Round1Sweep rs = round1_sweep(r0l.hi ^ t ^ a.rk[0], a.rk);
        for (int cell = warp; cell < g.n_cells; cell += nwarp)
            hidden_cell_generic<kPaper>(g, sm, rh, hw_byte, cell, rs, r0l.lo, a.rk, lm, rot0, rot1, lb, lane);
        __syncthreads();
        for (int cell = warp; cell < g.n_cells; cell += nwarp)
            visible_cell_generic<kPaper>(sm, rv, cell, rs, r0l.lo, a.rk, sflip, stepJ, lb, lane);
        __syncthreads();
        const bool do_meas = every_meas.step();
        const bool do_swap = every_swap.step();
        if (do_meas || do_swap) {
            int anti0 = 0, anti1 = 0, pos = 0;
            for (int cell = warp; cell < g.n_cells; cell += nwarp) count_cell(g, s_v, a.gep, cell, lane, anti0, anti1);
            for (int x = warp; x < g.N; x += nwarp) pos += static_cast<int>(bit_of(s_v[x], lane));
            atomicAdd(&s_cnt[lane], anti0);
            atomicAdd(&s_cnt[32 + lane], anti1);
            atomicAdd(&s_cnt[64 + lane], pos);
            __syncthreads();
            if (warp == 0) post_sweep_warp(a, s_cnt, s_sob, s_bos, lane, word, t, do_meas, do_swap, meas, s_acc);
            if (do_meas) ++meas;
            __syncthreads();
            if (do_swap) lb = 4u * static_cast<uint32_t>(s_bos[lane]);
        }
        if (every_sq.step()) {
            accumulate_correlations_any(a, s_v, nullptr, s_seg, s_segmask, warp, nwarp, lane);
            __syncthreads();
        }
    }
    for (int x = threadIdx.x; x < g.N; x += blockDim.x) gv[x] = s_v[x];
    if (warp == 0 && a.swap_every > 0) a.sob[word * 32 + lane] = s_sob[lane];
    if (warp == 0 && measuring) {
        for (int x = 0; x < kNSum; ++x) a.sums[static_cast<size_t>(chain) * kNSum + x] = s_acc[x * 32 + lane];
    }
}

}  // namespace generic
}  // namespace crbm
