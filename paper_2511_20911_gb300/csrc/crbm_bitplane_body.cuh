// The bit-plane SMEM sweep body (CRBM_RNG_BITPLANE, ten SS filters on an
// even periodic lattice) and its shared-memory layout, shared by the
// persistent kernel (crbm_bitplane.cu) and the batched launch
// (crbm_batch.cu).  The comparison scheme is described in crbm_bitplane.cu.
#pragma once

#include "crbm_bitplane_core.cuh"

namespace crbm {
namespace bp {

using namespace dev;

constexpr int kBpNodes = 10;   // hidden filters per cell

// Records of the sweep: [n_cells * 10] hidden endpoint pairs, [N][3] spin
// incidences (layout in crbm_host.cpp), rounded up to whole uint4.
__host__ __device__ inline size_t bp_rec_words(const Geometry& g) {
    return (static_cast<size_t>(g.n_cells) * kBpNodes + 3 * static_cast<size_t>(g.N) + 3) & ~static_cast<size_t>(3);
}

// Shared memory, 32-bit words: running sums, the word's planes and sign masks
// as built (bit l = rung l) and as used (bit l = the rung that slot l holds,
// the identity without replica exchange), counts, the replica permutation
// (rung -> slot, slot -> rung), spins, hidden words (rounded up to whole
// uint4), the straggler counts and list, then the records when staged.
constexpr int kBpSmemV = kAccWords + 2 * kBpTab + 96 + 64;
static_assert(kBpSmemV % 4 == 0, "spins start on a 16-byte boundary");
__host__ __device__ inline size_t bp_hid_words(const Geometry& g) {
    return (static_cast<size_t>(g.n_cells) * kBpNodes + 3) & ~static_cast<size_t>(3);
}
// Straggler list: (node, open chains) pairs, a quarter of the larger half-step
// (at least 32 entries, a multiple of 4); nodes beyond it finish in place.
__host__ __device__ inline int bp_strag_cap(const Geometry& g) {
    const int n = g.n_cells * kBpNodes > g.N ? g.n_cells * kBpNodes : g.N;
    const int q = ((n / 4) + 3) & ~3;
    return q < 32 ? 32 : q;
}
// the list and its two counters (hidden, visible), padded to a whole uint4
__host__ __device__ inline size_t bp_strag_words(const Geometry& g) { return 2 * static_cast<size_t>(bp_strag_cap(g)) + 4; }


// The sweeps of one packed word: its planes, spins and sums in, n sweeps
// from global sweep t0 (measurement index meas0), spins and sums out.  hrec,
// vrec: the node records (hidden endpoint pairs, spin incidences), staged in
// shared memory by the caller or read from global memory.
template <bool kSwap>
__device__ __forceinline__ void sweep_bitplane_body(const SweepArgs& a, const uint32_t* hrec, const uint32_t* vrec,
                                                    int word, uint32_t t0, int n_sweeps, int64_t meas) {
    extern __shared__ __align__(16) uint32_t smem[];
    const Geometry& g = a.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // the warp that keeps the running sums and finishes each measurement: the last, which has the
    // fewest node groups when they do not divide evenly, so that it can finish a measurement while
    // the others start the next sweep
    const int post_warp = nwarp - 1;
    const int N = g.N, nh = g.n_cells * kBpNodes;
    int64_t* s_acc = reinterpret_cast<int64_t*>(smem);          // [kNSum][32] running sums
    uint32_t* s_tab0 = smem + kAccWords;                         // [kBpTab] planes, sign masks by rung
    uint32_t* s_tab = s_tab0 + kBpTab;                           // [kBpTab] the same by slot
    int* s_cnt = reinterpret_cast<int*>(s_tab + kBpTab);         // [3][32] measurement counts
    int* s_sob = s_cnt + 96;                                     // [32] slot of each rung
    int* s_bos = s_sob + 32;                                     // [32] rung of each slot
    uint32_t* s_v = smem + kBpSmemV;                             // [N] spin words
    uint32_t* s_h = s_v + N;                                     // [n_cells * 10] hidden words
    int* s_nst = reinterpret_cast<int*>(s_h + bp_hid_words(g));   // [2] straggler counts (+2 pad)
    uint2* s_list = reinterpret_cast<uint2*>(s_nst + 4);           // [cap] stragglers (node, open chains)
    const int cap = bp_strag_cap(g);
    const uint32_t* gt = a.ctab + static_cast<size_t>(word) * kCanonTab;
    for (int x = threadIdx.x; x < kBpTab; x += blockDim.x) (kSwap ? s_tab0 : s_tab)[x] = gt[x];
    const uint32_t* gv = a.v + static_cast<size_t>(word) * N;
    for (int x = threadIdx.x; x < N; x += blockDim.x) s_v[x] = __ldcg(gv + x);
    for (int x = threadIdx.x; x < 96; x += blockDim.x) s_cnt[x] = 0;
    if (threadIdx.x < 2) s_nst[threadIdx.x] = 0;
    if (warp == post_warp) {  // replica permutation (identity without replica exchange)
        const int sob = kSwap ? __ldcg(a.sob + word * 32 + lane) : lane;
        s_sob[lane] = sob;
        s_bos[sob] = lane;
    }
    // bit l of a plane as used = bit s_bos[l] of the plane as built
    auto permute_planes = [&]() {
        const uint32_t src = static_cast<uint32_t>(s_bos[lane]);
        for (int x = warp; x < kBpTab; x += nwarp) s_tab[x] = __ballot_sync(0xffffffffu, (s_tab0[x] >> src) & 1u);
    };
    if (kSwap) {
        __syncthreads();
        permute_planes();
    }
    const bool measuring = a.measure_every > 0;
    const uint32_t chain = static_cast<uint32_t>(word) * 32u + lane;
    if (measuring && warp == post_warp)
        for (int x = 0; x < kNSum; ++x) s_acc[x * 32 + lane] = __ldcg(a.sums + static_cast<size_t>(chain) * kNSum + x);
    __syncthreads();
    uint32_t fl0 = s_tab[kBpFlip], fl1 = s_tab[kBpFlip + 1];
    // Philox round 0 of the word (counter word 2): shared by every call of the CTA
    const uint64_t pw = static_cast<uint64_t>(kPhiloxM1) * static_cast<uint32_t>(word);
    const uint32_t Yw = static_cast<uint32_t>(pw), hiW = static_cast<uint32_t>(pw >> 32) ^ a.rk[0];

    EveryCounter every_meas(t0, a.measure_every), every_swap(t0, kSwap ? a.swap_every : 0);
    for (int it = 0; it < n_sweeps; ++it) {
        const uint32_t t = t0 + static_cast<uint32_t>(it);
        const Round1Sweep rs = round1_sweep(hiW ^ t, a.rk);  // round 1's sweep-wide product
        if (kSwap) {  // the sign masks follow the rungs
            fl0 = s_tab[kBpFlip];
            fl1 = s_tab[kBpFlip + 1];
        }
        // hidden half-step (Eq. 9): thread = hidden node (cell, k).  Its endpoints select per chain
        // the threshold planes of m = e1 + s e2 (P: m = 2, M: m = -2, Z: m = 0, whose threshold 2^31
        // has only plane 0 set)
        struct Hid {
            uint32_t P, M, Z, c2;
            const uint32_t* tp;
            Round2Cell r2;
        };
        auto hidden_node = [&](int nd) {
            const uint32_t r = hrec[nd];
            const uint32_t cell = static_cast<uint32_t>(nd / kBpNodes);
            const uint32_t k = static_cast<uint32_t>(nd) - cell * kBpNodes;
            const uint32_t cls = k >= 8u ? 1u : 0u;
            const uint32_t e1 = s_v[r & 0xFFFFu];
            const uint32_t e2 = s_v[r >> 16] ^ (cls ? fl1 : fl0);
            const uint64_t pc = static_cast<uint64_t>(kPhiloxM0) * cell;
            return Hid{e1 & e2, ~(e1 | e2), e1 ^ e2,
                       static_cast<uint32_t>(pc >> 32) ^ a.rk[1] ^ (kTagBitplane + 8u * k),
                       s_tab + kBpHidPlanes + cls * 96u, round2_cell(rs.hik ^ static_cast<uint32_t>(pc))};
        };
        for (int base = warp * 32; base < nh; base += nwarp * 32) {
            const int node = base + lane;
            const bool valid = node < nh;
            const Hid hn = hidden_node(valid ? node : 0);
            uint32_t lt = 0u, eq = valid ? 0xffffffffu : 0u;
            auto planes = [&](const U4& q, uint32_t j) {
                bp::hidden_planes(q, hn.tp + 4u * j, hn.P, hn.M, j == 0u ? hn.Z : 0u, lt, eq);
            };
            // calls 0 and 1 together, then the open nodes to the straggler list
            const U4 q0 = philox_from_round2(Yw, rs, hn.r2, hn.c2, a.rk);
            const U4 q1 = philox_from_round2(Yw, rs, hn.r2, hn.c2 ^ 1u, a.rk);
            planes(q0, 0u);
            planes(q1, 1u);
            if (push_straggler(static_cast<uint32_t>(node), eq, s_nst, s_list, cap, lane)) eq = 0u;
#pragma unroll 1
            for (uint32_t j = 2; j < 8u; ++j) {  // only where the list was full
                if (!__any_sync(0xffffffffu, eq != 0u)) break;
                planes(philox_from_round2(Yw, rs, hn.r2, hn.c2 ^ j, a.rk), j);
            }
            if (valid) s_h[node] = lt;  // final, or the decided part of a straggler
        }
        __syncthreads();
        {
            const int n_st = min(s_nst[0], cap);
            for (int base = warp * 32; base < n_st; base += nwarp * 32) {
                const bool valid = base + lane < n_st;
                const uint2 e = valid ? s_list[base + lane] : make_uint2(0u, 0u);
                const int node = static_cast<int>(e.x);
                const Hid hn = hidden_node(node);
                uint32_t lt = s_h[node], eq = e.y;
#pragma unroll 1
                for (uint32_t j = 2; j < 8u; ++j) {
                    if (!__any_sync(0xffffffffu, eq != 0u)) break;
                    bp::hidden_planes(philox_from_round2(Yw, rs, hn.r2, hn.c2 ^ j, a.rk), hn.tp + 4u * j, hn.P, hn.M,
                                      0u, lt, eq);
                }
                if (valid) s_h[node] = lt;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nst[0] = 0;  // every thread has read it (before the barrier above)
        // visible half-step (Eq. 10): thread = spin site; its four J incidences, counted bit-sliced,
        // and its J' incidence select one of the 5 x 2 visible threshold planes per chain
        struct Vis {
            uint32_t hp, c2;
            bp::Count4 n4;
            Round2Cell r2;
        };
        auto visible_node = [&](int sd) {
            const uint32_t r0 = vrec[3 * sd], r1 = vrec[3 * sd + 1], r2w = vrec[3 * sd + 2];
            auto hin = [&](uint32_t x, uint32_t fl) { return s_h[x & 0x7FFFu] ^ ((x & 0x8000u) ? fl : 0u); };
            const uint32_t h0 = hin(r0, fl0), h1 = hin(r0 >> 16, fl0), h2 = hin(r1, fl0), h3 = hin(r1 >> 16, fl0);
            const uint32_t cell = (r2w >> 16) & 0xFFFu, x = r2w >> 28;
            const uint64_t pc = static_cast<uint64_t>(kPhiloxM0) * cell;
            return Vis{hin(r2w, fl1), static_cast<uint32_t>(pc >> 32) ^ a.rk[1] ^ (kTagBitplane + 8u * (10u + x)),
                       bp::count4(h0, h1, h2, h3), round2_cell(rs.hik ^ static_cast<uint32_t>(pc))};
        };
        const uint32_t* tv = s_tab + kBpVisPlanes;  // [count][J' bit][32]
        auto vis_planes = [&](const Vis& vn, const U4& q, uint32_t j, uint32_t& lt, uint32_t& eq) {
            const uint4 T = bp::visible_planes(tv + 4u * j, vn.hp, vn.n4);
            bp::plane_step(q.x, T.x, lt, eq);
            bp::plane_step(q.y, T.y, lt, eq);
            bp::plane_step(q.z, T.z, lt, eq);
            bp::plane_step(q.w, T.w, lt, eq);
        };
        for (int base = warp * 32; base < N; base += nwarp * 32) {
            const int sx = base + lane;
            const bool valid = sx < N;
            const Vis vn = visible_node(valid ? sx : 0);
            uint32_t lt = 0u, eq = valid ? 0xffffffffu : 0u;
            vis_planes(vn, philox_from_round2(Yw, rs, vn.r2, vn.c2, a.rk), 0u, lt, eq);
            vis_planes(vn, philox_from_round2(Yw, rs, vn.r2, vn.c2 ^ 1u, a.rk), 1u, lt, eq);
            if (push_straggler(static_cast<uint32_t>(sx), eq, s_nst + 1, s_list, cap, lane)) eq = 0u;
#pragma unroll 1
            for (uint32_t j = 2; j < 8u; ++j) {  // only where the list was full
                if (!__any_sync(0xffffffffu, eq != 0u)) break;
                vis_planes(vn, philox_from_round2(Yw, rs, vn.r2, vn.c2 ^ j, a.rk), j, lt, eq);
            }
            if (valid) s_v[sx] = lt;  // no spin is read in this half-step
        }
        __syncthreads();
        {
            const int n_st = min(s_nst[1], cap);
            for (int base = warp * 32; base < n_st; base += nwarp * 32) {
                const bool valid = base + lane < n_st;
                const uint2 e = valid ? s_list[base + lane] : make_uint2(0u, 0u);
                const int sx = static_cast<int>(e.x);
                const Vis vn = visible_node(sx);
                uint32_t lt = s_v[sx], eq = e.y;
#pragma unroll 1
                for (uint32_t j = 2; j < 8u; ++j) {
                    if (!__any_sync(0xffffffffu, eq != 0u)) break;
                    vis_planes(vn, philox_from_round2(Yw, rs, vn.r2, vn.c2 ^ j, a.rk), j, lt, eq);
                }
                if (valid) s_v[sx] = lt;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nst[1] = 0;
        const bool do_meas = every_meas.step();
        const bool do_swap = kSwap && every_swap.step();
        if (do_meas || do_swap) {
            // per chain: anti-aligned J and J' filters, +1 spins.  A warp takes 32 nodes (spins) at
            // a time, lane = node, and a bit transpose turns their 32 chain words into one word per
            // chain, lane = chain, whose popcount is that chain's count
            int anti0 = 0, anti1 = 0, pos = 0;
            for (int base = warp * 32; base < nh; base += nwarp * 32) {
                const int node = base + lane;
                uint32_t dJ = 0u, dP = 0u;
                if (node < nh) {
                    const uint32_t r = hrec[node];
                    const uint32_t d = s_v[r & 0xFFFFu] ^ s_v[r >> 16];
                    if (node % kBpNodes < 8) dJ = d;
                    else dP = d;
                }
                anti0 += __popc(transpose32(dJ, lane));
                anti1 += __popc(transpose32(dP, lane));
            }
            for (int base = warp * 32; base < N; base += nwarp * 32)
                pos += __popc(transpose32(base + lane < N ? s_v[base + lane] : 0u, lane));
            atomicAdd(&s_cnt[lane], anti0);
            atomicAdd(&s_cnt[32 + lane], anti1);
            atomicAdd(&s_cnt[64 + lane], pos);
            __syncthreads();
            if (warp == post_warp) post_sweep_warp(a, s_cnt, s_sob, s_bos, lane, word, t, do_meas, do_swap, meas, s_acc);
            if (do_meas) ++meas;
            // a measurement alone touches only warp post_warp's sums and the counts, which the next
            // measurement reaches after the next sweep's barriers; a swap round re-permutes the planes
            if (do_swap) {
                __syncthreads();
                permute_planes();
                __syncthreads();
            }
        }
    }
    if (kSwap && warp == post_warp) a.sob[word * 32 + lane] = s_sob[lane];
    uint32_t* gvo = a.v + static_cast<size_t>(word) * N;
    for (int x = threadIdx.x; x < N; x += blockDim.x) gvo[x] = s_v[x];
    if (measuring && warp == post_warp)
        for (int x = 0; x < kNSum; ++x) a.sums[static_cast<size_t>(chain) * kNSum + x] = s_acc[x * 32 + lane];
}

}  // namespace bp
}  // namespace crbm
