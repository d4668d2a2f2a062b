// Body of the generic SMEM-resident sweep (any filter list <= 16 filters, odd
// L, open boundaries; one CTA = one 32-chain word), shared by the
// single-context kernel (crbm_kernels.cu) and the batched kernel
// (crbm_batch.cu).
#pragma once

#include "crbm_device.cuh"

namespace crbm {
namespace generic {

using namespace dev;

// Endpoint word of filter k of a cell (built on the host): bits 0..14 the
// site of the first endpoint, bit 15 set when it is a real site (clear for a
// zero-padded one, whose site bits are 0), bits 16..31 the same for the
// second endpoint.
__device__ __forceinline__ int endpoint_term(const uint32_t* s_v, uint32_t half, int lane, uint32_t flip) {
    const int b = static_cast<int>(bit_of(s_v[half & 0x7FFFu], lane) ^ flip);
    return (half & 0x8000u) ? 2 * b - 1 : 0;
}

// Generic hidden half-step: any filter list (<= 16 filters), odd L, open
// boundaries.  m = c1 v1 + c2 v2 with a zero-padded endpoint contributing 0;
// the threshold row is cls * 5 + (m + 2).
// Draws: Philox-4x32-10 of counter (cell, sweep, chain, tag) from the split
// rounds (crbm_device.cuh): rs = round1_sweep of the lane's sweep word, Y the
// lane's chain word, rk the round keys.
__device__ __forceinline__ void hidden_cell_generic(const Geometry& g, const uint32_t* s_v,
                                                    uint32_t* s_h, const uint32_t* s_tab,
                                                    const uint32_t* __restrict__ ep, int cell,
                                                    const Round1Sweep& rs, uint32_t Y, const uint32_t (&rk)[20],
                                                    int lane, int col, const uint32_t (&sn)[2]) {
    const Round0Cell rc = round0_cell(static_cast<uint32_t>(cell), rk[1]);
    const Round2Cell r2 = round2_cell(rs.hik ^ rc.b);
    U4 q[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (c < g.n_calls) q[c] = philox_from_round2(Y, rs, r2, rc.a ^ static_cast<uint32_t>(c), rk);
    const uint32_t* e = ep + static_cast<size_t>(cell) * g.nb;
#pragma unroll
    for (int k = 0; k < kMaxBonds; ++k) {
        if (k < g.nb) {
            const uint32_t ek = __ldg(e + k);
            const int cls = g.cls[k];
            const int m = 2 + endpoint_term(s_v, ek, lane, 0u) + endpoint_term(s_v, ek >> 16, lane, sn[cls]);
            const uint32_t thr = s_tab[(cls * 5 + m) * 32 + col];
            const uint32_t hw = __ballot_sync(0xffffffffu, pick(q[k >> 2], k & 3) < thr);
            if (lane == 0) s_h[cell * g.nb + k] = hw;
        }
    }
}

// Generic visible half-step: incidences of each spin from a CSR list.  Entry
// bits 0..27 = hidden index (cell * nb + k), bit 30 = class, bit 31 = second
// endpoint (coefficient s).
__device__ __forceinline__ void visible_cell_generic(const Geometry& g, uint32_t* s_v,
                                                     const uint32_t* s_h, const uint32_t* s_tab,
                                                     const uint32_t* __restrict__ inc,
                                                     const int32_t* __restrict__ inc_off,
                                                     int cell, int i, int j, const Round1Sweep& rs, uint32_t Y,
                                                     const uint32_t (&rk)[20], int lane, int col,
                                                     const uint32_t (&sn)[2]) {
    const Round0Cell rc = round0_cell(static_cast<uint32_t>(cell), rk[1]);
    const U4 q = philox_from_round2(Y, rs, round2_cell(rs.hik ^ rc.b), rc.a ^ kTagVis, rk);
    const int nP = 2 * g.DJp + 1;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int R = 2 * i + (w >> 1), C = 2 * j + (w & 1);
        if (R < g.L && C < g.L) {
            const int s = R * g.L + C;
            int n[2] = {0, 0};
            const int e0 = __ldg(inc_off + s), e1 = __ldg(inc_off + s + 1);
            for (int e = e0; e < e1; ++e) {
                const uint32_t ent = __ldg(inc + e);
                const int cls = (ent >> 30) & 1;
                const uint32_t b = bit_of(s_h[ent & 0x0FFFFFFFu], lane) ^ ((ent >> 31) ? sn[cls] : 0u);
                n[cls] += 2 * static_cast<int>(b) - 1;
            }
            const uint32_t thr = s_tab[(10 + (n[0] + g.DJ) * nP + (n[1] + g.DJp)) * 32 + col];
            const uint32_t vw = __ballot_sync(0xffffffffu, pick(q, w) < thr);
            if (lane == 0) s_v[s] = vw;
        }
    }
}

// Per-lane counts of one cell for the energy/magnetisation measurement:
// anti[cls] = number of anti-aligned real bonds, pos = number of +1 spins.
__device__ __forceinline__ void count_cell(const Geometry& g, const uint32_t* s_v,
                                           const uint32_t* __restrict__ ep, int cell, int i, int j,
                                           int lane, int& anti0, int& anti1, int& pos) {
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
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int R = 2 * i + (w >> 1), C = 2 * j + (w & 1);
        if (R < g.L && C < g.L) pos += static_cast<int>(bit_of(s_v[R * g.L + C], lane));
    }
}

// Generic SMEM-resident sweep: one CTA per packed word (32 chains), the whole
// lattice, hidden layer and threshold columns in shared memory, all n_sweeps
// sweeps on device.  Warps split the cells of each half-step; __syncthreads
// separates the half-steps (hidden reads v / writes h; visible reads h /
// writes v).
__device__ __forceinline__ void sweep_generic_body(const SweepArgs& a, int word) {
    extern __shared__ __align__(16) uint32_t smem[];
    const Geometry& g = a.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    int64_t* s_acc = reinterpret_cast<int64_t*>(smem);  // [kNSum][32] running sums
    uint32_t* s_tab = smem + kAccWords;
    uint32_t* s_v = s_tab + g.nTab * 32;
    uint32_t* s_h = s_v + g.N;
    int* s_cnt = reinterpret_cast<int*>(s_h + g.n_cells * g.nb);  // [3][32]
    int* s_seg = s_cnt + 96;                                       // [33]
    uint32_t* s_segmask = reinterpret_cast<uint32_t*>(s_seg + 33); // [32]
    int* s_sob = reinterpret_cast<int*>(s_segmask + 32);          // [32] slot of each rung
    int* s_bos = s_sob + 32;                                        // [32] rung of each slot

    const uint32_t* gtab = a.tab + static_cast<size_t>(word) * g.nTab * 32;
    for (int x = threadIdx.x; x < g.nTab * 32; x += blockDim.x) s_tab[x] = gtab[x];
    uint32_t* gv = a.v + static_cast<size_t>(word) * g.N;
    for (int x = threadIdx.x; x < g.N; x += blockDim.x) s_v[x] = gv[x];
    for (int x = threadIdx.x; x < 96; x += blockDim.x) s_cnt[x] = 0;
    if (a.sq_every > 0) {
        for (int x = threadIdx.x; x < 33; x += blockDim.x) s_seg[x] = a.seg[word * 33 + x];
        for (int x = threadIdx.x; x < 32; x += blockDim.x) s_segmask[x] = a.segmask[word * 32 + x];
    }
    const uint32_t sn[2] = {bit_of(a.sneg[2 * word], lane), bit_of(a.sneg[2 * word + 1], lane)};
    const uint32_t chain = static_cast<uint32_t>(word) * 32u + lane;
    if (warp == 0) {  // replica permutation (identity without tempering)
        const int sob = a.swap_every > 0 ? a.sob[word * 32 + lane] : lane;
        s_sob[lane] = sob;
        s_bos[sob] = lane;
    }
    __syncthreads();
    int col = s_bos[lane];  // threshold column: the rung this slot holds
    const bool measuring = a.measure_every > 0;
    if (warp == 0 && measuring) {
        for (int x = 0; x < kNSum; ++x) s_acc[x * 32 + lane] = a.sums[static_cast<size_t>(chain) * kNSum + x];
    }
    // sweep and measurement counters: kernel arguments, or the batch's device clock
    const uint32_t t0 = a.clock ? static_cast<uint32_t>(a.clock[0]) : a.t0;
    int64_t meas = a.clock ? a.clock[1] : a.meas0;
    const int i_first = warp / g.W, j_first = warp - (warp / g.W) * g.W;
    const int di = nwarp / g.W, dj = nwarp - (nwarp / g.W) * g.W;

    const Round0Lane r0l = round0_lane(chain);
    for (int it = 0; it < a.n_sweeps; ++it) {
        const uint32_t t = t0 + static_cast<uint32_t>(it);
        const Round1Sweep rs = round1_sweep(r0l.hi ^ t ^ a.rk[0], a.rk);
        for (int cell = warp; cell < g.n_cells; cell += nwarp)
            hidden_cell_generic(g, s_v, s_h, s_tab, a.gep, cell, rs, r0l.lo, a.rk, lane, col, sn);
        __syncthreads();
        int i = i_first, j = j_first;
        for (int cell = warp; cell < g.n_cells; cell += nwarp) {
            visible_cell_generic(g, s_v, s_h, s_tab, a.inc, a.inc_off, cell, i, j, rs, r0l.lo, a.rk, lane, col,
                                 sn);
            i += di;
            j += dj;
            if (j >= g.W) {
                j -= g.W;
                ++i;
            }
        }
        __syncthreads();
        const bool do_meas = measuring && (t + 1u) % static_cast<uint32_t>(a.measure_every) == 0u;
        const bool do_swap = a.swap_every > 0 && (t + 1u) % static_cast<uint32_t>(a.swap_every) == 0u;
        if (do_meas || do_swap) {
            int anti0 = 0, anti1 = 0, pos = 0;
            i = i_first;
            j = j_first;
            for (int cell = warp; cell < g.n_cells; cell += nwarp) {
                count_cell(g, s_v, a.gep, cell, i, j, lane, anti0, anti1, pos);
                i += di;
                j += dj;
                if (j >= g.W) {
                    j -= g.W;
                    ++i;
                }
            }
            atomicAdd(&s_cnt[lane], anti0);
            atomicAdd(&s_cnt[32 + lane], anti1);
            atomicAdd(&s_cnt[64 + lane], pos);
            __syncthreads();
            if (warp == 0) post_sweep_warp0(a, s_cnt, s_sob, s_bos, lane, word, t, do_meas, do_swap, meas, s_acc);
            if (do_meas) ++meas;
            __syncthreads();
            if (do_swap) col = s_bos[lane];
        }
        if (a.sq_every > 0 && (t + 1u) % static_cast<uint32_t>(a.sq_every) == 0u) {
            accumulate_correlations(a, s_v, s_seg, s_segmask, warp, nwarp, lane);
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
