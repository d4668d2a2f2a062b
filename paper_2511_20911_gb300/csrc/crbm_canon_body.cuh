// Body of the canonical SMEM-resident sweep (one CTA = one 32-chain word, or
// one band of cell rows of a word in a thread-block cluster), shared by the
// persistent kernel (crbm_canon.cu) and the batched kernel (crbm_batch.cu).
#pragma once

#include <cooperative_groups.h>

#include "crbm_canon_core.cuh"

namespace crbm {
namespace canon {

namespace cg = cooperative_groups;

template <bool kSmem>
__device__ __forceinline__ uint4 ld_rec(const uint4* p) {
    return kSmem ? *p : __ldg(p);
}
// The first word of a cell's record 5 (Q2.lo).
template <bool kSmem>
__device__ __forceinline__ uint32_t ld_rec5(const uint4* r) {
    return kSmem ? reinterpret_cast<const uint32_t*>(r + 5)[0] : __ldg(reinterpret_cast<const uint32_t*>(r + 5));
}

// The two halves of a cluster barrier, so that work no other CTA waits for
// can run between them: arrive (release: this thread's earlier shared-memory
// stores, local and remote) and wait (acquire).  Every thread of the CTA
// executes both, the same number of times on every rank.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// CTA barrier, or cluster barrier (release / acquire over the cluster's
// shared memory) when a word is split over the CTAs of a cluster.
template <bool kCluster>
__device__ __forceinline__ void body_sync() {
    if (kCluster)
        cg::this_cluster().sync();
    else
        __syncthreads();
}

// Whole-run body of the canonical SMEM-resident sweep for packed word `word`:
// load tables, spins and replica permutation into shared memory, run
// n_sweeps sweeps from global sweep t0 (measurement index meas0) with
// measurement / replica exchange / correlations, write the state back.
// State is read with L1-bypassing loads: under the persistent scheduler the
// previous chunk of this word may have been written by another SM.
// kSmemRec: the per-cell records are first copied into shared memory after
// the replica tables (canon_smem_records() decides on the host), else read
// through the read-only cache.
// kCluster: the CTA holds band `band` of the word's a.n_bands bands of cell
// rows; the word's bands are the cluster ranks rank0 .. rank0 + n_bands - 1
// (a cluster may hold several words of one context, or padding ranks of that
// context with band >= n_bands).  Every rank holds the whole lattice;
// it updates its own rows and, as it goes, writes the hidden words of its
// last cell row into the next band (the upper neighbours of that band's first
// row) and the spins of its first spin row into the previous band (the last
// window row of that band's last cell row), wrapping around.  Half-steps end
// with a cluster barrier; measurement counts are summed into the word's
// band 0, which runs the measurement and the replica exchange.  Padding ranks
// (band >= n_bands) only keep the barrier count, which is the same for every
// rank because a cluster never mixes contexts.  Correlations need the whole
// lattice, so a word with sq_every > 0 is never split (n_bands == 1).
// A band does the cells other bands wait for first (its last cell row in
// the hidden half-step, its first in the visible one), arrives at the cluster
// barrier, does the rest and only then waits.  Those boundary cells are the
// only ones that read rows a neighbour writes, and they run after the
// previous barrier completed, so no band overwrites a row its neighbour has
// yet to read.
// kPaper: CRBM_PRECISION_PAPER draws (two Philox calls per cell, the visible
// uniforms passed from the hidden half-step through shared memory).
template <bool kSmemRec, bool kCluster, bool kPaper = false>
__device__ __forceinline__ void sweep_canon_body(const SweepArgs& a, int word, uint32_t t0, int n_sweeps,
                                                 int64_t meas0, int band = 0, int rank0 = 0) {
    extern __shared__ __align__(16) uint32_t smem[];
    const Geometry& g = a.g;
    const int W = g.W, Wc = g.Wc;  // rows and columns of cells
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // The warp that keeps the running sums and finishes each measurement: the
    // last, which has the fewest cells when they do not divide evenly, so that
    // it can finish a measurement while the others start the next sweep.
    const int post_warp = nwarp - 1;
    const int nb = kCluster ? a.n_bands : 1;
    const bool active = band < nb;
    const int row0 = active ? band * W / nb : 0, row1 = active ? (band + 1) * W / nb : 0;
    // (the two forms of the cell range compile to measurably faster code in
    // the exact and the paper-precision sweep respectively; they are equal)
    const int c_begin = (kCluster || kPaper) ? row0 * Wc : 0;
    const int c_end = (kCluster || kPaper) ? row1 * Wc : g.n_cells;
    int64_t* s_acc = reinterpret_cast<int64_t*>(smem);  // [kNSum][32] running sums
    uint32_t* s_th = smem + kAccWords;          // [2][4][32]
    uint32_t* s_tv = s_th + kCanonTh;           // [4][32][32]
    uint32_t* s_v = s_th + kCanonTab;           // [N]
    uint32_t* s_w = s_v + g.N;                  // [n_cells][32] per-lane hidden words
    int* s_cnt = reinterpret_cast<int*>(s_w + g.n_cells * 32);   // [3][32]
    int* s_seg = s_cnt + 96;                                      // [33]
    uint32_t* s_segmask = reinterpret_cast<uint32_t*>(s_seg + 33); // [32]
    int* s_sob = reinterpret_cast<int*>(s_segmask + 32);          // [32] slot of each rung
    int* s_bos = s_sob + 32;                                        // [32] rung of each slot
    char* sm = reinterpret_cast<char*>(smem);
    // cluster neighbours (unused without a split)
    char* sm_next = sm;
    char* sm_prev = sm;
    int* cnt0 = s_cnt;
    const int* bos0 = s_bos;
    if (kCluster && active) {
        cg::cluster_group cl = cg::this_cluster();
        if (nb > 1) {
            sm_next = cl.map_shared_rank(sm, static_cast<unsigned int>(rank0 + (band + 1) % nb));
            sm_prev = cl.map_shared_rank(sm, static_cast<unsigned int>(rank0 + (band + nb - 1) % nb));
        }
        cnt0 = cl.map_shared_rank(s_cnt, static_cast<unsigned int>(rank0));
        bos0 = cl.map_shared_rank(s_bos, static_cast<unsigned int>(rank0));
    }

    const uint4* recs = a.crec;
    const uint32_t chain = static_cast<uint32_t>(word) * 32u + lane;
    LaneConst lc = lane_const(lane, lane);
    const Round0Lane r0l = round0_lane(chain);
    const bool measuring = a.measure_every > 0;
    if (active) {
        if (kSmemRec) {  // [n_cells][kCellRec] records, 16-byte aligned
            uint4* s_rec = reinterpret_cast<uint4*>(smem + canon_smem_rec_offset(g));
            for (int x = threadIdx.x; x < g.n_cells * kCellRec; x += blockDim.x) s_rec[x] = __ldg(a.crec + x);
            recs = s_rec;
        }
        const uint4* gt = reinterpret_cast<const uint4*>(a.ctab + static_cast<size_t>(word) * kCanonTab);
        for (int x = threadIdx.x; x < kCanonTab / 4; x += blockDim.x) reinterpret_cast<uint4*>(s_th)[x] = gt[x];
        const uint32_t* gv = a.v + static_cast<size_t>(word) * g.N;
        for (int x = threadIdx.x; x < g.N; x += blockDim.x) s_v[x] = __ldcg(gv + x);
        for (int x = threadIdx.x; x < 96; x += blockDim.x) s_cnt[x] = 0;
        if (a.sq_every > 0) {
            for (int x = threadIdx.x; x < 33; x += blockDim.x) s_seg[x] = a.seg[word * 33 + x];
            for (int x = threadIdx.x; x < 32; x += blockDim.x) s_segmask[x] = a.segmask[word * 32 + x];
        }
        if (warp == post_warp) {  // replica permutation (identity without tempering)
            const int sob = a.swap_every > 0 ? __ldcg(a.sob + word * 32 + lane) : lane;
            s_sob[lane] = sob;
            s_bos[sob] = lane;
        }
    }
    __syncthreads();
    lc.lb = 4u * static_cast<uint32_t>(s_bos[lane]);  // lane reads the column of its rung
    if (active && band == 0 && warp == post_warp && measuring) {
        for (int x = 0; x < kNSum; ++x)
            s_acc[x * 32 + lane] = __ldcg(a.sums + static_cast<size_t>(chain) * kNSum + x);
    }
    if (kCluster) body_sync<true>();  // every rank started before any shared memory crosses CTAs

    // sweep and measurement counters: kernel arguments, or the batch's device clock
    int64_t meas = meas0;
    // Cells of this warp: c_begin + warp, + nwarp, ...; each described by its
    // kCellRec records (shared-memory byte offsets and round-0 Philox words).
    const uint32_t lane4 = 4u * static_cast<uint32_t>(lane);
    const uint4* rec0 = recs + static_cast<size_t>(c_begin + warp) * kCellRec;
    const int rstep = nwarp * kCellRec;
    const int last_row = c_end - Wc, first_row_end = c_begin + Wc;

    EveryCounter every_meas(t0, a.measure_every), every_swap(t0, a.swap_every), every_sq(t0, kCluster ? 0 : a.sq_every);
    for (int it = 0; it < n_sweeps; ++it) {
        const uint32_t t = t0 + static_cast<uint32_t>(it);
        const Round1Sweep rs = round1_sweep(r0l.hi ^ t ^ a.rk[0], a.rk);
        const uint4* rec = rec0;
        if (kPaper && !kCluster) {
            for (int cell = c_begin + warp; cell < c_end; cell += nwarp, rec += rstep) {
                const uint4 h0 = ld_rec<kSmemRec>(rec), h1 = ld_rec<kSmemRec>(rec + 1),
                            h2 = ld_rec<kSmemRec>(rec + 2);
                sts_off(sm, h1.y + lane4, hidden_cell_rec_paper(sm, h0, h1, h2, s_th, rs, r0l.lo, a.rk, lc,
                                                                2u * lane4));
            }
            __syncthreads();
            rec = rec0;
            for (int cell = c_begin + warp; cell < c_end; cell += nwarp, rec += rstep)
                visible_cell_rec_paper(sm, ld_rec<kSmemRec>(rec + 3), ld_rec<kSmemRec>(rec + 4), lane4, s_tv, lc);
            __syncthreads();
        } else if (kCluster && nb > 1) {  // a band of a split word, or a padding rank of one
            // the last cell row first (the next band waits for its hidden words), arrive, the rest,
            // then wait: the cluster barrier's latency overlaps the interior rows
            if (active) {
                for (int cell = last_row + warp; cell < c_end; cell += nwarp) {
                    const uint4* r = recs + static_cast<size_t>(cell) * kCellRec;
                    const uint4 h0 = ld_rec<kSmemRec>(r), h1 = ld_rec<kSmemRec>(r + 1), h2 = ld_rec<kSmemRec>(r + 2);
                    const uint32_t w = hidden_cell_rec(sm, h0, h1, h2, ld_rec5<kSmemRec>(r), s_th, rs, r0l.lo, a.rk, lc);
                    sts_off(sm, h1.y + lane4, w);
                    sts_off(sm_next, h1.y + lane4, w);
                }
            }
            cluster_arrive();
            if (active) {
                for (int cell = c_begin + warp; cell < last_row; cell += nwarp) {
                    const uint4* r = recs + static_cast<size_t>(cell) * kCellRec;
                    const uint4 h0 = ld_rec<kSmemRec>(r), h1 = ld_rec<kSmemRec>(r + 1), h2 = ld_rec<kSmemRec>(r + 2);
                    sts_off(sm, h1.y + lane4,
                            hidden_cell_rec(sm, h0, h1, h2, ld_rec5<kSmemRec>(r), s_th, rs, r0l.lo, a.rk, lc));
                }
            }
            __syncthreads();
            cluster_wait();
            // the first cell row first (the previous band waits for its spins)
            if (active) {
                for (int cell = c_begin + warp; cell < first_row_end; cell += nwarp) {
                    const uint4* r = recs + static_cast<size_t>(cell) * kCellRec;
                    const uint4 v0 = ld_rec<kSmemRec>(r + 3);
                    const U4 o = visible_cell_rec(sm, v0, ld_rec<kSmemRec>(r + 4), lane4, s_tv, rs, r0l.lo, a.rk, lc);
                    sts_off(sm_prev, v0.x, o.x);
                    sts_off(sm_prev, v0.x + 4u, o.y);
                }
            }
            cluster_arrive();
            if (active) {
                for (int cell = first_row_end + warp; cell < c_end; cell += nwarp) {
                    const uint4* r = recs + static_cast<size_t>(cell) * kCellRec;
                    visible_cell_rec(sm, ld_rec<kSmemRec>(r + 3), ld_rec<kSmemRec>(r + 4), lane4, s_tv, rs, r0l.lo,
                                     a.rk, lc);
                }
            }
            __syncthreads();
            cluster_wait();
        } else {  // the whole word in one CTA
        for (int cell = c_begin + warp; cell < c_end; cell += nwarp, rec += rstep) {
            const uint4 h0 = ld_rec<kSmemRec>(rec), h1 = ld_rec<kSmemRec>(rec + 1), h2 = ld_rec<kSmemRec>(rec + 2);
            const uint32_t h5 = kSmemRec ? reinterpret_cast<const uint32_t*>(rec + 5)[0]
                                         : __ldg(reinterpret_cast<const uint32_t*>(rec + 5));
            const uint32_t w = hidden_cell_rec(sm, h0, h1, h2, h5, s_th, rs, r0l.lo, a.rk, lc);
            sts_off(sm, h1.y + lane4, w);
            if (kCluster && nb > 1 && cell >= last_row) sts_off(sm_next, h1.y + lane4, w);
        }
        body_sync<kCluster>();
        rec = rec0;
        for (int cell = c_begin + warp; cell < c_end; cell += nwarp, rec += rstep) {
            const uint4 v0 = ld_rec<kSmemRec>(rec + 3), v1 = ld_rec<kSmemRec>(rec + 4);
            const U4 o = visible_cell_rec(sm, v0, v1, lane4, s_tv, rs, r0l.lo, a.rk, lc);
            if (kCluster && nb > 1 && cell < first_row_end) {
                sts_off(sm_prev, v0.x, o.x);
                sts_off(sm_prev, v0.x + 4u, o.y);
            }
        }
        body_sync<kCluster>();
        }
        const bool do_meas = every_meas.step();
        const bool do_swap = every_swap.step();
        if (do_meas || do_swap) {
            if (active) {
                int anti0 = 0, anti1 = 0, pos = 0;
                rec = rec0;
                for (int cell = c_begin + warp; cell < c_end; cell += nwarp, rec += rstep)
                    count_cell_rec(sm, ld_rec<kSmemRec>(rec), ld_rec<kSmemRec>(rec + 1), lane, anti0, anti1, pos);
                atomicAdd(&cnt0[lane], anti0);
                atomicAdd(&cnt0[32 + lane], anti1);
                atomicAdd(&cnt0[64 + lane], pos);
            }
            body_sync<kCluster>();
            if (band == 0 && warp == post_warp)
                post_sweep_warp(a, s_cnt, s_sob, s_bos, lane, word, t, do_meas, do_swap, meas, s_acc);
            if (do_meas) ++meas;
            // A swap round changes the permutation every warp reads next; a
            // measurement alone touches only warp post_warp's sums and the counts, which
            // the next measurement reaches after the next sweep's barriers.
            if (do_swap) {
                body_sync<kCluster>();
                if (active) lc.lb = 4u * static_cast<uint32_t>(bos0[lane]);
            }
        }
        if (every_sq.step()) {
            accumulate_correlations_any(a, s_v, s_w, s_seg, s_segmask, warp, nwarp, lane);  // s_w: dead here
            __syncthreads();
        }
    }
    if (kCluster) body_sync<true>();  // no rank reads another's shared memory after this
    if (!active) return;
    uint32_t* gv = a.v + static_cast<size_t>(word) * g.N;
    const int s_begin = kCluster ? 2 * row0 * g.Lc : 0;  // own spin rows
    const int s_end = kCluster ? min(2 * row1, g.L) * g.Lc : g.N;
    for (int x = s_begin + static_cast<int>(threadIdx.x); x < s_end; x += blockDim.x) gv[x] = s_v[x];
    if (band == 0 && warp == post_warp && a.swap_every > 0) a.sob[word * 32 + lane] = s_sob[lane];
    if (band == 0 && warp == post_warp && measuring) {
        for (int x = 0; x < kNSum; ++x) a.sums[static_cast<size_t>(chain) * kNSum + x] = s_acc[x * 32 + lane];
    }
}


}  // namespace canon
}  // namespace crbm
