// CUDA kernels of the CRBM block-Gibbs sampler (sm_103a).
//
// Work mapping: 32 chains share one packed 32-bit word per site (bit l =
// chain 32w + l); a warp works on one word, lane l owning chain 32w + l.  The
// packed words are warp-uniform, so every shared-memory read of the lattice is
// a broadcast, and each lane only extracts its own bit, draws its own Philox
// words and compares against its own threshold column; __ballot_sync packs
// the 32 decisions back into one word.  Everything is integer arithmetic:
// no tensor cores, no floating point on the path.
#include "crbm_internal.h"

namespace crbm {
namespace {

struct U4 {
    uint32_t x, y, z, w;
};

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies by the round multipliers, the high halves XORed with
// the other two counter words and the round key; the key advances by the two
// Weyl increments between rounds.
__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c0;
        const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c2;
        const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
        c1 = static_cast<uint32_t>(p1);
        c3 = static_cast<uint32_t>(p0);
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ uint32_t pick(const U4& q, int w) {
    return w == 0 ? q.x : (w == 1 ? q.y : (w == 2 ? q.z : q.w));
}

__device__ __forceinline__ uint32_t bit_of(uint32_t word, int lane) { return (word >> lane) & 1u; }

// Site index of window offset (r, c) of cell (i, j), or -1 for a zero-padded
// (open boundary) site.  r, c <= 2 and 2i, 2j <= L - 1, so one wrap suffices.
__device__ __forceinline__ int site_of(const Geometry& g, int i, int j, int r, int c) {
    int R = 2 * i + r, C = 2 * j + c;
    if (R >= g.L) {
        if (!g.periodic) return -1;
        R -= g.L;
    }
    if (C >= g.L) {
        if (!g.periodic) return -1;
        C -= g.L;
    }
    return R * g.L + C;
}

// ----------------------------------------------------------------------------
// Hidden half-step of one cell (Eq. 9), canonical SS filters, even periodic L.
// The nine window words are read once; bond k's second endpoint carries the
// class sign s, applied per lane as an XOR with the lane's sign bit.
__device__ __forceinline__ void hidden_cell_canon(const Geometry& g, const uint32_t* s_v,
                                                  uint32_t* s_h, int cell, int i, int j,
                                                  uint32_t t, uint32_t chain, int lane,
                                                  uint32_t k0, uint32_t k1, uint32_t sn0,
                                                  uint32_t sn1, const uint32_t (&th)[2][3]) {
    const int L = g.L;
    const int R0 = 2 * i, R1 = R0 + 1, R2 = (R0 + 2 == L) ? 0 : R0 + 2;
    const int C0 = 2 * j, C1 = C0 + 1, C2 = (C0 + 2 == L) ? 0 : C0 + 2;
    const uint32_t b00 = bit_of(s_v[R0 * L + C0], lane), b01 = bit_of(s_v[R0 * L + C1], lane);
    const uint32_t b02 = bit_of(s_v[R0 * L + C2], lane), b10 = bit_of(s_v[R1 * L + C0], lane);
    const uint32_t b11 = bit_of(s_v[R1 * L + C1], lane), b12 = bit_of(s_v[R1 * L + C2], lane);
    const uint32_t b20 = bit_of(s_v[R2 * L + C0], lane), b21 = bit_of(s_v[R2 * L + C1], lane);
    const U4 q0 = philox(cell, t, chain, 0u, k0, k1);
    const U4 q1 = philox(cell, t, chain, 1u, k0, k1);
    const U4 q2 = philox(cell, t, chain, 2u, k0, k1);
    // sum = b(first) + (b(second) ^ sign) in {0, 1, 2}  <->  m = 2 sum - 2
    auto decide = [&](uint32_t e1, uint32_t e2, uint32_t sn, int cls, uint32_t u) -> uint32_t {
        const uint32_t sum = e1 + (e2 ^ sn);
        const uint32_t thr = sum == 0u ? th[cls][0] : (sum == 1u ? th[cls][1] : th[cls][2]);
        return __ballot_sync(0xffffffffu, u < thr);
    };
    uint32_t* h = s_h + cell * 10;
    const uint32_t h0 = decide(b00, b01, sn0, 0, q0.x);
    const uint32_t h1 = decide(b01, b02, sn0, 0, q0.y);
    const uint32_t h2 = decide(b10, b11, sn0, 0, q0.z);
    const uint32_t h3 = decide(b11, b12, sn0, 0, q0.w);
    const uint32_t h4 = decide(b00, b10, sn0, 0, q1.x);
    const uint32_t h5 = decide(b10, b20, sn0, 0, q1.y);
    const uint32_t h6 = decide(b01, b11, sn0, 0, q1.z);
    const uint32_t h7 = decide(b11, b21, sn0, 0, q1.w);
    const uint32_t h8 = decide(b00, b11, sn1, 1, q2.x);
    const uint32_t h9 = decide(b12, b21, sn1, 1, q2.y);
    if (lane == 0) {
        h[0] = h0; h[1] = h1; h[2] = h2; h[3] = h3; h[4] = h4;
        h[5] = h5; h[6] = h6; h[7] = h7; h[8] = h8; h[9] = h9;
    }
}

// Visible half-step of one cell (Eq. 10), canonical SS filters.  Each spin
// sees four J filters and one J' filter (own cell, the cell above, the cell
// to the left); n_J = 2c - 4 with c the number of +1 terms, n_J' = 2b - 1,
// so the table row is 10 + (n_J + 4) * 3 + (n_J' + 1) = 10 + 6c + 2b.
__device__ __forceinline__ void visible_cell_canon(const Geometry& g, uint32_t* s_v,
                                                   const uint32_t* s_h, const uint32_t* s_tab,
                                                   int cell, int i, int j, uint32_t t,
                                                   uint32_t chain, int lane, uint32_t k0,
                                                   uint32_t k1, uint32_t sn0, uint32_t sn1) {
    const int W = g.W, L = g.L;
    const int iu = (i == 0) ? W - 1 : i - 1;
    const int jl = (j == 0) ? W - 1 : j - 1;
    const uint32_t* ho = s_h + cell * 10;
    const uint32_t* hu = s_h + (iu * W + j) * 10;
    const uint32_t* hl = s_h + (i * W + jl) * 10;
    const uint32_t o0 = bit_of(ho[0], lane), o1 = bit_of(ho[1], lane), o2 = bit_of(ho[2], lane);
    const uint32_t o3 = bit_of(ho[3], lane), o4 = bit_of(ho[4], lane), o5 = bit_of(ho[5], lane);
    const uint32_t o6 = bit_of(ho[6], lane), o7 = bit_of(ho[7], lane), o8 = bit_of(ho[8], lane);
    const uint32_t u5 = bit_of(hu[5], lane) ^ sn0, u7 = bit_of(hu[7], lane) ^ sn0;
    const uint32_t u9 = bit_of(hu[9], lane) ^ sn1;
    const uint32_t l1 = bit_of(hl[1], lane) ^ sn0, l3 = bit_of(hl[3], lane) ^ sn0;
    const uint32_t l9 = bit_of(hl[9], lane);
    const U4 q = philox(cell, t, chain, kTagVis, k0, k1);
    // (0,0): b0 e1, b1(left) e2, b4 e1, b5(up) e2 | b8 e1
    const uint32_t c00 = o0 + l1 + o4 + u5, p00 = o8;
    // (0,1): b0 e2, b1 e1, b6 e1, b7(up) e2 | b9(up) e2
    const uint32_t c01 = (o0 ^ sn0) + o1 + o6 + u7, p01 = u9;
    // (1,0): b2 e1, b3(left) e2, b4 e2, b5 e1 | b9(left) e1
    const uint32_t c10 = o2 + l3 + (o4 ^ sn0) + o5, p10 = l9;
    // (1,1): b2 e2, b3 e1, b6 e2, b7 e1 | b8 e2
    const uint32_t c11 = (o2 ^ sn0) + o3 + (o6 ^ sn0) + o7, p11 = o8 ^ sn1;
    const uint32_t t00 = s_tab[(10 + 6 * c00 + 2 * p00) * 32 + lane];
    const uint32_t t01 = s_tab[(10 + 6 * c01 + 2 * p01) * 32 + lane];
    const uint32_t t10 = s_tab[(10 + 6 * c10 + 2 * p10) * 32 + lane];
    const uint32_t t11 = s_tab[(10 + 6 * c11 + 2 * p11) * 32 + lane];
    const uint32_t v00 = __ballot_sync(0xffffffffu, q.x < t00);
    const uint32_t v01 = __ballot_sync(0xffffffffu, q.y < t01);
    const uint32_t v10 = __ballot_sync(0xffffffffu, q.z < t10);
    const uint32_t v11 = __ballot_sync(0xffffffffu, q.w < t11);
    if (lane == 0) {
        const int r0 = 2 * i * L + 2 * j;
        s_v[r0] = v00;
        s_v[r0 + 1] = v01;
        s_v[r0 + L] = v10;
        s_v[r0 + L + 1] = v11;
    }
}

// Generic hidden half-step: any filter list (<= 16 filters), odd L, open
// boundaries.  m = c1 v1 + c2 v2 with a zero-padded endpoint contributing 0;
// the threshold row is cls * 5 + (m + 2).
__device__ __forceinline__ void hidden_cell_generic(const Geometry& g, const uint32_t* s_v,
                                                    uint32_t* s_h, const uint32_t* s_tab,
                                                    int cell, int i, int j, uint32_t t,
                                                    uint32_t chain, int lane, uint32_t k0,
                                                    uint32_t k1, const uint32_t (&sn)[2]) {
    U4 q[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (c < g.n_calls) q[c] = philox(cell, t, chain, static_cast<uint32_t>(c), k0, k1);
#pragma unroll
    for (int k = 0; k < kMaxBonds; ++k) {
        if (k < g.nb) {
            const int s1 = site_of(g, i, j, g.r1[k], g.c1[k]);
            const int s2 = site_of(g, i, j, g.r2[k], g.c2[k]);
            const int cls = g.cls[k];
            int m = 2;
            if (s1 >= 0) m += 2 * static_cast<int>(bit_of(s_v[s1], lane)) - 1;
            if (s2 >= 0) m += 2 * static_cast<int>(bit_of(s_v[s2], lane) ^ sn[cls]) - 1;
            const uint32_t thr = s_tab[(cls * 5 + m) * 32 + lane];
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
                                                     int cell, int i, int j, uint32_t t,
                                                     uint32_t chain, int lane, uint32_t k0,
                                                     uint32_t k1, const uint32_t (&sn)[2]) {
    const U4 q = philox(cell, t, chain, kTagVis, k0, k1);
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
            const uint32_t thr = s_tab[(10 + (n[0] + g.DJ) * nP + (n[1] + g.DJp)) * 32 + lane];
            const uint32_t vw = __ballot_sync(0xffffffffu, pick(q, w) < thr);
            if (lane == 0) s_v[s] = vw;
        }
    }
}

// Per-lane counts of one cell for the energy/magnetisation measurement:
// anti[cls] = number of anti-aligned real bonds, pos = number of +1 spins.
__device__ __forceinline__ void count_cell(const Geometry& g, const uint32_t* s_v, int i, int j,
                                           int lane, int& anti0, int& anti1, int& pos) {
#pragma unroll
    for (int k = 0; k < kMaxBonds; ++k) {
        if (k < g.nb) {
            const int s1 = site_of(g, i, j, g.r1[k], g.c1[k]);
            const int s2 = site_of(g, i, j, g.r2[k], g.c2[k]);
            if (s1 >= 0 && s2 >= 0) {
                const int x = static_cast<int>(bit_of(s_v[s1] ^ s_v[s2], lane));
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

__device__ __forceinline__ int warp_sum(int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ----------------------------------------------------------------------------
// SMEM-resident sweep: one CTA per packed word (32 chains), the whole lattice,
// hidden layer and threshold columns in shared memory, all n_sweeps sweeps on
// device.  Warps split the cells of each half-step; __syncthreads separates
// the half-steps (hidden reads v / writes h; visible reads h / writes v).
template <bool kCanon>
__global__ void __launch_bounds__(kCanon ? 1024 : 512) k_sweep_smem(const SweepArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const Geometry& g = a.g;
    const int word = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    uint32_t* s_tab = smem;
    uint32_t* s_v = s_tab + g.nTab * 32;
    uint32_t* s_h = s_v + g.N;
    int* s_cnt = reinterpret_cast<int*>(s_h + g.n_cells * g.nb);  // [3][32]
    int* s_seg = s_cnt + 96;                                       // [33]
    uint32_t* s_segmask = reinterpret_cast<uint32_t*>(s_seg + 33); // [32]

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
    __syncthreads();
    uint32_t th[2][3];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        th[c][0] = s_tab[(c * 5 + 0) * 32 + lane];
        th[c][1] = s_tab[(c * 5 + 2) * 32 + lane];
        th[c][2] = s_tab[(c * 5 + 4) * 32 + lane];
    }
    int64_t acc[kNSum];
    const bool measuring = a.measure_every > 0;
    if (warp == 0 && measuring) {
#pragma unroll
        for (int x = 0; x < kNSum; ++x) acc[x] = a.sums[static_cast<size_t>(chain) * kNSum + x];
    }
    int64_t meas = a.meas0;

    for (int it = 0; it < a.n_sweeps; ++it) {
        const uint32_t t = a.t0 + static_cast<uint32_t>(it);
        for (int cell = warp; cell < g.n_cells; cell += nwarp) {
            const int i = cell / g.W, j = cell - (cell / g.W) * g.W;
            if (kCanon)
                hidden_cell_canon(g, s_v, s_h, cell, i, j, t, chain, lane, a.key0, a.key1, sn[0],
                                  sn[1], th);
            else
                hidden_cell_generic(g, s_v, s_h, s_tab, cell, i, j, t, chain, lane, a.key0,
                                    a.key1, sn);
        }
        __syncthreads();
        for (int cell = warp; cell < g.n_cells; cell += nwarp) {
            const int i = cell / g.W, j = cell - (cell / g.W) * g.W;
            if (kCanon)
                visible_cell_canon(g, s_v, s_h, s_tab, cell, i, j, t, chain, lane, a.key0, a.key1,
                                   sn[0], sn[1]);
            else
                visible_cell_generic(g, s_v, s_h, s_tab, a.inc, a.inc_off, cell, i, j, t, chain,
                                     lane, a.key0, a.key1, sn);
        }
        __syncthreads();
        if (measuring && (t + 1u) % static_cast<uint32_t>(a.measure_every) == 0u) {
            int anti0 = 0, anti1 = 0, pos = 0;
            for (int cell = warp; cell < g.n_cells; cell += nwarp) {
                const int i = cell / g.W, j = cell - (cell / g.W) * g.W;
                count_cell(g, s_v, i, j, lane, anti0, anti1, pos);
            }
            atomicAdd(&s_cnt[lane], anti0);
            atomicAdd(&s_cnt[32 + lane], anti1);
            atomicAdd(&s_cnt[64 + lane], pos);
            __syncthreads();
            if (warp == 0) {
                const int64_t nJ = g.n_real_bonds[0] - 2 * s_cnt[lane];
                const int64_t nP = g.n_real_bonds[1] - 2 * s_cnt[32 + lane];
                const int64_t M = 2 * s_cnt[64 + lane] - g.N;
                s_cnt[lane] = 0;
                s_cnt[32 + lane] = 0;
                s_cnt[64 + lane] = 0;
                if (meas < a.series_len) {
                    int32_t* e = a.series + (static_cast<size_t>(meas) * a.n_chains_padded + chain) * 3;
                    e[0] = static_cast<int32_t>(nJ);
                    e[1] = static_cast<int32_t>(nP);
                    e[2] = static_cast<int32_t>(M);
                }
                acc[0] += 1;
                acc[1] += nJ;
                acc[2] += nP;
                acc[3] += M;
                acc[4] += M < 0 ? -M : M;
                acc[5] += nJ * nJ;
                acc[6] += nP * nP;
                acc[7] += M * M;
                acc[8] += nJ * nP;
                acc[9] += nJ * M;
                acc[10] += nP * M;
            }
            ++meas;
            __syncthreads();
        }
        if (a.sq_every > 0 && (t + 1u) % static_cast<uint32_t>(a.sq_every) == 0u) {
            // C_p(d) += sum over the chains of segment p of sum_r s_r s_{r+d}
            //         = n_p N - 2 sum_r popc((v_r ^ v_{r+d}) & mask_p)
            const int L = g.L, N = g.N, nseg = s_seg[0];
            for (int d = warp; d < N; d += nwarp) {
                const int dR = d / L, dC = d - (d / L) * L;
                for (int sgi = 0; sgi < nseg; ++sgi) {
                    const uint32_t mask = s_segmask[sgi];
                    int cnt = 0;
                    for (int r = lane; r < N; r += 32) {
                        const int R = r / L, C = r - (r / L) * L;
                        int R2 = R + dR, C2 = C + dC;
                        if (R2 >= L) R2 -= L;
                        if (C2 >= L) C2 -= L;
                        cnt += __popc((s_v[r] ^ s_v[R2 * L + C2]) & mask);
                    }
                    cnt = warp_sum(cnt);
                    if (lane == 0) {
                        const int p = s_seg[1 + sgi] >> 8;
                        const long long val = static_cast<long long>(__popc(mask)) * N - 2LL * cnt;
                        atomicAdd(reinterpret_cast<unsigned long long*>(a.corr + static_cast<size_t>(p) * N + d),
                                  static_cast<unsigned long long>(val));
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int x = threadIdx.x; x < g.N; x += blockDim.x) gv[x] = s_v[x];
    if (warp == 0 && measuring) {
#pragma unroll
        for (int x = 0; x < kNSum; ++x) a.sums[static_cast<size_t>(chain) * kNSum + x] = acc[x];
    }
}

// Initial spins: site (R, C) of chain c is +1 iff word 2(R&1)+(C&1) of
// Philox((cell, 0, c, tag 5)) < 2^31.  One warp per (word, site).
__global__ void k_init(const Geometry g, uint32_t* v, int n_words, uint32_t k0, uint32_t k1) {
    const int lane = threadIdx.x & 31;
    const long long nw = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long x = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         x < static_cast<long long>(n_words) * g.N; x += nw) {
        const int word = static_cast<int>(x / g.N), s = static_cast<int>(x - static_cast<long long>(word) * g.N);
        const int R = s / g.L, C = s - (s / g.L) * g.L;
        const uint32_t cell = static_cast<uint32_t>((R >> 1) * g.W + (C >> 1));
        const U4 q = philox(cell, 0u, static_cast<uint32_t>(word) * 32u + lane, kTagInit, k0, k1);
        const uint32_t b = __ballot_sync(0xffffffffu, pick(q, 2 * (R & 1) + (C & 1)) < 0x80000000u);
        if (lane == 0) v[x] = b;
    }
}

__global__ void k_unpack(const Geometry g, const uint32_t* v, int8_t* out, int n_words) {
    const long long total = static_cast<long long>(n_words) * 32 * g.N;
    for (long long x = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long chain = x / g.N;
        const int s = static_cast<int>(x - chain * g.N);
        const uint32_t w = v[(chain >> 5) * g.N + s];
        out[x] = ((w >> (chain & 31)) & 1u) ? 1 : -1;
    }
}

__global__ void k_pack(const Geometry g, const int8_t* in, uint32_t* v, int n_words) {
    const int lane = threadIdx.x & 31;
    const long long nw = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long x = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         x < static_cast<long long>(n_words) * g.N; x += nw) {
        const long long word = x / g.N;
        const int s = static_cast<int>(x - word * g.N);
        const int8_t val = in[(word * 32 + lane) * g.N + s];
        const uint32_t b = __ballot_sync(0xffffffffu, val > 0);
        if (lane == 0) v[x] = b;
    }
}

__global__ void k_philox(const uint32_t* in, uint32_t* out, int n) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t* a = in + 6 * static_cast<size_t>(x);
    const U4 q = philox(a[0], a[1], a[2], a[3], a[4], a[5]);
    uint32_t* o = out + 4 * static_cast<size_t>(x);
    o[0] = q.x;
    o[1] = q.y;
    o[2] = q.z;
    o[3] = q.w;
}

}  // namespace

cudaError_t launch_philox(const uint32_t* in, uint32_t* out, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_philox<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

size_t smem_bytes_smem_layout(const Geometry& g) {
    return sizeof(uint32_t) * (static_cast<size_t>(g.nTab) * 32 + g.N +
                               static_cast<size_t>(g.n_cells) * g.nb + 96 + 33 + 32);
}

cudaError_t launch_init(const Geometry& g, uint32_t* v, int n_words, uint32_t key0, uint32_t key1,
                        cudaStream_t st) {
    const long long work = static_cast<long long>(n_words) * g.N;
    const int blocks = static_cast<int>((work + 7) / 8 < 152 * 64 ? (work + 7) / 8 : 152 * 64);
    k_init<<<blocks, 256, 0, st>>>(g, v, n_words, key0, key1);
    return cudaGetLastError();
}

cudaError_t launch_sweep_smem(const SweepArgs& a, int warps_per_cta, cudaStream_t st) {
    const size_t smem = smem_bytes_smem_layout(a.g);
    if (a.g.canonical) {
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(
                k_sweep_smem<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return e;
        }
        k_sweep_smem<true><<<a.n_words, warps_per_cta * 32, smem, st>>>(a);
    } else {
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(
                k_sweep_smem<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return e;
        }
        k_sweep_smem<false><<<a.n_words, warps_per_cta * 32, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geometry& g, const uint32_t* v, int8_t* out, int n_words,
                          cudaStream_t st) {
    const long long total = static_cast<long long>(n_words) * 32 * g.N;
    const int blocks = static_cast<int>((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    k_unpack<<<blocks, 256, 0, st>>>(g, v, out, n_words);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Geometry& g, const int8_t* in, uint32_t* v, int n_words,
                        cudaStream_t st) {
    const long long work = static_cast<long long>(n_words) * g.N;
    const int blocks = static_cast<int>((work + 7) / 8 < 152 * 64 ? (work + 7) / 8 : 152 * 64);
    k_pack<<<blocks, 256, 0, st>>>(g, in, v, n_words);
    return cudaGetLastError();
}

}  // namespace crbm
