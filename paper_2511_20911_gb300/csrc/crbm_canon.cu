// Canonical fast path of the SMEM-resident sweep: the ten SS filters of
// Fig. 1 on an even, periodic L x L lattice (four J filters and one J' filter
// per spin, Eq. 8).
//
// Same mapping as the generic kernel (warp = 32 chains of one packed word,
// lane = chain), but the per-lane work is reduced to what the integer pipes
// must do per node: each packed word the node depends on is masked to the
// lane's bit and rotated (funnel shift) straight into the address bits of a
// lane-expanded threshold table; OR-ing those bits with the lane's column
// offset gives the table address.  The host builds the tables so that they
// absorb the coefficient signs s and the field sums (Eqs. 9-10), so a node
// costs one address merge, one shared load, one compare and one ballot.
#include "crbm_device.cuh"

#ifndef CRBM_SWEEP_MIN_BLOCKS
#define CRBM_SWEEP_MIN_BLOCKS 2
#endif

namespace crbm {
namespace {

using namespace dev;

// Byte-addressed 32-bit shared-memory load.
__device__ __forceinline__ uint32_t lds_at(const uint32_t* base, uint32_t byte_off) {
    return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(base) + byte_off);
}

struct LaneConst {
    uint32_t lm;      // 1 << lane
    uint32_t lb;      // 4 * lane: the lane's column in a [.][32] table
    uint32_t rot[5];  // rotate-right amounts taking bit `lane` to bit 7 + j
};

// Hidden half-step of one cell (Eq. 9).  Table s_th[cls][e1 + 2 e2][lane]
// (byte offset cls*512 + idx*128 + 4 lane): the e1 bit is rotated to bit 7,
// the e2 bit to bit 8.
__device__ __forceinline__ void hidden_cell(const uint32_t* s_v, uint32_t* s_h, const uint32_t* s_th,
                                            int L, int cell, int i, int j, uint32_t X, uint32_t Y,
                                            const Round0Cell rc, const uint32_t (&rk)[20],
                                            const LaneConst& lc) {
    const int R0 = 2 * i, R1 = R0 + 1, R2 = (R0 + 2 == L) ? 0 : R0 + 2;
    const int C0 = 2 * j, C1 = C0 + 1, C2 = (C0 + 2 == L) ? 0 : C0 + 2;
    const uint32_t m00 = s_v[R0 * L + C0] & lc.lm, m01 = s_v[R0 * L + C1] & lc.lm;
    const uint32_t m02 = s_v[R0 * L + C2] & lc.lm, m10 = s_v[R1 * L + C0] & lc.lm;
    const uint32_t m11 = s_v[R1 * L + C1] & lc.lm, m12 = s_v[R1 * L + C2] & lc.lm;
    const uint32_t m20 = s_v[R2 * L + C0] & lc.lm, m21 = s_v[R2 * L + C1] & lc.lm;
    // first endpoints at bit 7
    const uint32_t a00 = rotr(m00, lc.rot[0]), a01 = rotr(m01, lc.rot[0]);
    const uint32_t a10 = rotr(m10, lc.rot[0]), a11 = rotr(m11, lc.rot[0]);
    const uint32_t a12 = rotr(m12, lc.rot[0]);
    // second endpoints at bit 8
    const uint32_t b01 = rotr(m01, lc.rot[1]), b02 = rotr(m02, lc.rot[1]);
    const uint32_t b10 = rotr(m10, lc.rot[1]), b11 = rotr(m11, lc.rot[1]);
    const uint32_t b12 = rotr(m12, lc.rot[1]), b20 = rotr(m20, lc.rot[1]);
    const uint32_t b21 = rotr(m21, lc.rot[1]);
    const U4 q0 = philox_rounds1to9(X, Y, rc.a, rc.b, rk);
    const U4 q1 = philox_rounds1to9(X, Y, rc.a ^ 1u, rc.b, rk);
    const U4 q2 = philox_rounds1to9(X, Y, rc.a ^ 2u, rc.b, rk);
    const uint32_t* thJ = s_th;
    const uint32_t* thP = s_th + 128;
    uint32_t* h = s_h + cell * 10;
    // filters 0..7 (J) and 8..9 (J'): (first endpoint, second endpoint)
    h[0] = __ballot_sync(0xffffffffu, q0.x < lds_at(thJ, a00 | b01 | lc.lb));
    h[1] = __ballot_sync(0xffffffffu, q0.y < lds_at(thJ, a01 | b02 | lc.lb));
    h[2] = __ballot_sync(0xffffffffu, q0.z < lds_at(thJ, a10 | b11 | lc.lb));
    h[3] = __ballot_sync(0xffffffffu, q0.w < lds_at(thJ, a11 | b12 | lc.lb));
    h[4] = __ballot_sync(0xffffffffu, q1.x < lds_at(thJ, a00 | b10 | lc.lb));
    h[5] = __ballot_sync(0xffffffffu, q1.y < lds_at(thJ, a10 | b20 | lc.lb));
    h[6] = __ballot_sync(0xffffffffu, q1.z < lds_at(thJ, a01 | b11 | lc.lb));
    h[7] = __ballot_sync(0xffffffffu, q1.w < lds_at(thJ, a11 | b21 | lc.lb));
    h[8] = __ballot_sync(0xffffffffu, q2.x < lds_at(thP, a00 | b11 | lc.lb));
    h[9] = __ballot_sync(0xffffffffu, q2.y < lds_at(thP, a12 | b21 | lc.lb));
}

// Visible half-step of one cell (Eq. 10).  Each spin's five filter units sit
// in slots 0..4 (bits 7..11) of a 5-bit index into s_tv[site][idx][lane]
// (byte offset site*4096 + idx*128 + 4 lane).  Slot assignment (own cell /
// cell above "u" / cell to the left "l"), chosen so that a unit shared by two
// spins of the cell sits in the same slot for both:
//   spin (0,0): b0 b4 b8 l.b1 u.b5     spin (0,1): b0 b6 b1 u.b7 u.b9
//   spin (1,0): b2 b4 b5 l.b3 l.b9     spin (1,1): b2 b6 b8 b3 b7
__device__ __forceinline__ void visible_cell(uint32_t* s_v, const uint32_t* s_h, const uint32_t* s_tv,
                                             int L, int W, int cell, int i, int j, uint32_t X,
                                             uint32_t Y, const Round0Cell rc, const uint32_t (&rk)[20],
                                             const LaneConst& lc) {
    const int iu = (i == 0) ? W - 1 : i - 1;
    const int jl = (j == 0) ? W - 1 : j - 1;
    const uint32_t* ho = s_h + cell * 10;
    const uint32_t* hu = s_h + (iu * W + j) * 10;
    const uint32_t* hl = s_h + (i * W + jl) * 10;
    const uint32_t o0 = rotr(ho[0] & lc.lm, lc.rot[0]), o2 = rotr(ho[2] & lc.lm, lc.rot[0]);
    const uint32_t o4 = rotr(ho[4] & lc.lm, lc.rot[1]), o6 = rotr(ho[6] & lc.lm, lc.rot[1]);
    const uint32_t o8 = rotr(ho[8] & lc.lm, lc.rot[2]), o1 = rotr(ho[1] & lc.lm, lc.rot[2]);
    const uint32_t o5 = rotr(ho[5] & lc.lm, lc.rot[2]), o3 = rotr(ho[3] & lc.lm, lc.rot[3]);
    const uint32_t o7 = rotr(ho[7] & lc.lm, lc.rot[4]);
    const uint32_t l1 = rotr(hl[1] & lc.lm, lc.rot[3]), l3 = rotr(hl[3] & lc.lm, lc.rot[3]);
    const uint32_t l9 = rotr(hl[9] & lc.lm, lc.rot[4]);
    const uint32_t u5 = rotr(hu[5] & lc.lm, lc.rot[4]), u7 = rotr(hu[7] & lc.lm, lc.rot[3]);
    const uint32_t u9 = rotr(hu[9] & lc.lm, lc.rot[4]);
    const U4 q = philox_rounds1to9(X, Y, rc.a ^ kTagVis, rc.b, rk);
    const uint32_t t00 = lds_at(s_tv, o0 | o4 | o8 | l1 | u5 | lc.lb);
    const uint32_t t01 = lds_at(s_tv + 1024, o0 | o6 | o1 | u7 | u9 | lc.lb);
    const uint32_t t10 = lds_at(s_tv + 2048, o2 | o4 | o5 | l3 | l9 | lc.lb);
    const uint32_t t11 = lds_at(s_tv + 3072, o2 | o6 | o8 | o3 | o7 | lc.lb);
    const int r0 = 2 * i * L + 2 * j;
    s_v[r0] = __ballot_sync(0xffffffffu, q.x < t00);
    s_v[r0 + 1] = __ballot_sync(0xffffffffu, q.y < t01);
    s_v[r0 + L] = __ballot_sync(0xffffffffu, q.z < t10);
    s_v[r0 + L + 1] = __ballot_sync(0xffffffffu, q.w < t11);
}

// Per-lane counts of one cell for the measurement: anti-aligned J and J'
// filters of the window, and +1 spins of the cell.
__device__ __forceinline__ void count_cell(const uint32_t* s_v, int L, int i, int j, int lane,
                                           int& anti0, int& anti1, int& pos) {
    const int R0 = 2 * i, R1 = R0 + 1, R2 = (R0 + 2 == L) ? 0 : R0 + 2;
    const int C0 = 2 * j, C1 = C0 + 1, C2 = (C0 + 2 == L) ? 0 : C0 + 2;
    const uint32_t w00 = s_v[R0 * L + C0], w01 = s_v[R0 * L + C1], w02 = s_v[R0 * L + C2];
    const uint32_t w10 = s_v[R1 * L + C0], w11 = s_v[R1 * L + C1], w12 = s_v[R1 * L + C2];
    const uint32_t w20 = s_v[R2 * L + C0], w21 = s_v[R2 * L + C1];
    anti0 += bit_of(w00 ^ w01, lane) + bit_of(w01 ^ w02, lane) + bit_of(w10 ^ w11, lane) +
             bit_of(w11 ^ w12, lane) + bit_of(w00 ^ w10, lane) + bit_of(w10 ^ w20, lane) +
             bit_of(w01 ^ w11, lane) + bit_of(w11 ^ w21, lane);
    anti1 += bit_of(w00 ^ w11, lane) + bit_of(w12 ^ w21, lane);
    pos += bit_of(w00, lane) + bit_of(w01, lane) + bit_of(w10, lane) + bit_of(w11, lane);
}

__global__ void __launch_bounds__(512, CRBM_SWEEP_MIN_BLOCKS) k_sweep_canon(const SweepArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const Geometry& g = a.g;
    const int L = g.L, W = g.W;
    const int word = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    uint32_t* s_th = smem;                      // [2][4][32]
    uint32_t* s_tv = smem + kCanonTh;           // [4][32][32]
    uint32_t* s_v = smem + kCanonTab;           // [N]
    uint32_t* s_h = s_v + g.N;                  // [n_cells][10]
    int* s_cnt = reinterpret_cast<int*>(s_h + g.n_cells * 10);   // [3][32]
    int* s_seg = s_cnt + 96;                                      // [33]
    uint32_t* s_segmask = reinterpret_cast<uint32_t*>(s_seg + 33); // [32]

    const uint4* gt = reinterpret_cast<const uint4*>(a.ctab + static_cast<size_t>(word) * kCanonTab);
    for (int x = threadIdx.x; x < kCanonTab / 4; x += blockDim.x) reinterpret_cast<uint4*>(smem)[x] = gt[x];
    uint32_t* gv = a.v + static_cast<size_t>(word) * g.N;
    for (int x = threadIdx.x; x < g.N; x += blockDim.x) s_v[x] = gv[x];
    for (int x = threadIdx.x; x < 96; x += blockDim.x) s_cnt[x] = 0;
    if (a.sq_every > 0) {
        for (int x = threadIdx.x; x < 33; x += blockDim.x) s_seg[x] = a.seg[word * 33 + x];
        for (int x = threadIdx.x; x < 32; x += blockDim.x) s_segmask[x] = a.segmask[word * 32 + x];
    }
    const uint32_t chain = static_cast<uint32_t>(word) * 32u + lane;
    LaneConst lc;
    lc.lm = 1u << lane;
    lc.lb = 4u * lane;
#pragma unroll
    for (int s = 0; s < 5; ++s) lc.rot[s] = static_cast<uint32_t>(lane - 7 - s) & 31u;
    const Round0Lane r0l = round0_lane(chain);
    __syncthreads();

    int64_t acc[kNSum];
    const bool measuring = a.measure_every > 0;
    if (warp == 0 && measuring) {
#pragma unroll
        for (int x = 0; x < kNSum; ++x) acc[x] = a.sums[static_cast<size_t>(chain) * kNSum + x];
    }
    int64_t meas = a.meas0;
    // Cells of this warp: warp, warp + nwarp, ...; (i, j) advanced without division.
    const int i_first = warp / W, j_first = warp - (warp / W) * W;
    const int di = nwarp / W, dj = nwarp - (nwarp / W) * W;

    for (int it = 0; it < a.n_sweeps; ++it) {
        const uint32_t t = a.t0 + static_cast<uint32_t>(it);
        const uint32_t X = r0l.hi ^ t ^ a.rk[0];
        int i = i_first, j = j_first;
        for (int cell = warp; cell < g.n_cells; cell += nwarp) {
            hidden_cell(s_v, s_h, s_th, L, cell, i, j, X, r0l.lo,
                        round0_cell(static_cast<uint32_t>(cell), a.rk[1]), a.rk, lc);
            i += di;
            j += dj;
            if (j >= W) {
                j -= W;
                ++i;
            }
        }
        __syncthreads();
        i = i_first;
        j = j_first;
        for (int cell = warp; cell < g.n_cells; cell += nwarp) {
            visible_cell(s_v, s_h, s_tv, L, W, cell, i, j, X, r0l.lo,
                         round0_cell(static_cast<uint32_t>(cell), a.rk[1]), a.rk, lc);
            i += di;
            j += dj;
            if (j >= W) {
                j -= W;
                ++i;
            }
        }
        __syncthreads();
        if (measuring && (t + 1u) % static_cast<uint32_t>(a.measure_every) == 0u) {
            int anti0 = 0, anti1 = 0, pos = 0;
            i = i_first;
            j = j_first;
            for (int cell = warp; cell < g.n_cells; cell += nwarp) {
                count_cell(s_v, L, i, j, lane, anti0, anti1, pos);
                i += di;
                j += dj;
                if (j >= W) {
                    j -= W;
                    ++i;
                }
            }
            atomicAdd(&s_cnt[lane], anti0);
            atomicAdd(&s_cnt[32 + lane], anti1);
            atomicAdd(&s_cnt[64 + lane], pos);
            __syncthreads();
            if (warp == 0) measure_finalize(a, s_cnt, lane, chain, meas, acc);
            ++meas;
            __syncthreads();
        }
        if (a.sq_every > 0 && (t + 1u) % static_cast<uint32_t>(a.sq_every) == 0u) {
            accumulate_correlations(a, s_v, s_seg, s_segmask, warp, nwarp, lane);
            __syncthreads();
        }
    }
    for (int x = threadIdx.x; x < g.N; x += blockDim.x) gv[x] = s_v[x];
    if (warp == 0 && measuring) {
#pragma unroll
        for (int x = 0; x < kNSum; ++x) a.sums[static_cast<size_t>(chain) * kNSum + x] = acc[x];
    }
}

}  // namespace

size_t smem_bytes_canon(const Geometry& g) {
    return sizeof(uint32_t) * (static_cast<size_t>(kCanonTab) + g.N + static_cast<size_t>(g.n_cells) * 10 +
                               96 + 33 + 32);
}

cudaError_t launch_sweep_canon(const SweepArgs& a, int warps_per_cta, cudaStream_t st) {
    const size_t smem = smem_bytes_canon(a.g);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_sweep_canon, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_sweep_canon<<<a.n_words, warps_per_cta * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace crbm
