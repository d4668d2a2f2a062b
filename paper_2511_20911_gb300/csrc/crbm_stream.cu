// Streamed sweep for lattices too large for shared memory (canonical SS
// filters, even periodic L x Lc): spins and hidden units live in HBM and one sweep
// is two launches, the hidden half-step (Eq. 9) then the visible half-step
// (Eq. 10).  Spins are stored as 64-chain words, two 32-bit halves per site
// ([group][site][2]); a CTA works on one 32-chain half and one tile of cells,
// staging its tile (plus a one-site / one-cell halo) in shared memory with
// plain coalesced loads, and reuses the per-cell cores of the SMEM path.  In
// paper precision (kPaper) the hidden half-step makes the tag-0 and tag-1
// calls and the visible half-step draws the tag-1 call again for its four
// 16-bit uniforms: three calls per cell instead of four.
#include "crbm_bitplane_core.cuh"
#include "crbm_canon_core.cuh"

namespace crbm {
namespace {

using namespace dev;
using namespace canon;

constexpr int kTI = 16;  // tile rows of cells
constexpr int kTJ = 16;  // tile columns of cells
#ifndef CRBM_STREAM_THREADS
#define CRBM_STREAM_THREADS 256
#endif
#ifndef CRBM_STREAM_VIS_THREADS
#define CRBM_STREAM_VIS_THREADS 256
#endif
constexpr int kStreamThreads = CRBM_STREAM_THREADS;      // hidden and count kernels
constexpr int kStreamVisThreads = CRBM_STREAM_VIS_THREADS;

__device__ __forceinline__ size_t vidx(int w, int N, int s) {
    return (static_cast<size_t>(w >> 1) * N + s) * 2 + (w & 1);
}

// With replica exchange a lane (replica slot) reads the threshold column of
// the rung it holds: s_bos[slot] = rung, from the word's slot-of-rung array.
// Threads of warp 0 write it; the caller's next barrier publishes it.
__device__ __forceinline__ void stage_rungs(const SweepArgs& a, int w, int* s_bos) {
    if (threadIdx.x < 32) {
        const int lane = static_cast<int>(threadIdx.x);
        s_bos[a.swap_every > 0 ? __ldg(a.sob + static_cast<size_t>(w) * 32 + lane) : lane] = lane;
    }
}
#ifndef CRBM_STREAM_MIN_BLOCKS
#define CRBM_STREAM_MIN_BLOCKS 4
#endif
#ifndef CRBM_STREAM_VIS_MIN_BLOCKS
#define CRBM_STREAM_VIS_MIN_BLOCKS 4
#endif

// Stage spin rows 2 i0 .. 2 i0 + 2 TI and columns 2 j0 .. 2 j0 + 2 TJ
// (wrapped) of half-word w into s_v[(2 TI + 1)][(2 TJ + 1)].  Every load of a
// thread is issued before its first shared store.  kOneWrap: L >= 2 TI and
// Lc >= 2 TJ, so 2 i0 + r <= L + 30 (2 j0 + c <= Lc + 30) needs at most one
// subtraction of L (Lc).
// n / d for 1 <= d <= 32 and 0 <= n < 2^16 (the tile-local indices) without a
// division: one high multiply by m = ceil(2^32 / d), exact because
// n (m d - 2^32) < 2^32 keeps the fraction below the next integer (d = 1,
// whose m does not fit 32 bits, passes n through).
struct SmallDiv {
    uint32_t m;
    int d;
    __device__ __forceinline__ explicit SmallDiv(int d_)
        : m(d_ > 1 ? static_cast<uint32_t>((0x100000000ull + static_cast<uint64_t>(d_) - 1u) /
                                           static_cast<uint64_t>(d_))
                   : 0u),
          d(d_) {}
    __device__ __forceinline__ int operator()(int n) const {
        return d > 1 ? static_cast<int>(__umulhi(static_cast<uint32_t>(n), m)) : n;
    }
};

template <bool kOneWrap>
__device__ __forceinline__ void stage_spin_tile(const SweepArgs& a, int w, int i0, int j0, uint32_t* s_v) {
    constexpr int VS = 2 * kTJ + 1, NV = (2 * kTI + 1) * VS;
    constexpr int IT = (NV + kStreamThreads - 1) / kStreamThreads;
    const int L = a.g.L, Lc = a.g.Lc;
    const uint32_t* vw = a.v + vidx(w, a.g.N, 0);  // site s of half-word w at vw[2 s]
    uint32_t val[IT];
#pragma unroll
    for (int k = 0; k < IT; ++k) {
        const int x = threadIdx.x + k * kStreamThreads;
        const int r = x / VS, c = x - (x / VS) * VS;
        int R = 2 * i0 + r, C = 2 * j0 + c;
        if (kOneWrap) {
            R -= R >= L ? L : 0;
            C -= C >= Lc ? Lc : 0;
        } else {
            R %= L;
            C %= Lc;
        }
        val[k] = 0u;
        if (x < NV) val[k] = vw[2 * (R * Lc + C)];
    }
#pragma unroll
    for (int k = 0; k < IT; ++k) {
        const int x = threadIdx.x + k * kStreamThreads;
        if (x < NV) s_v[x] = val[k];
    }
}

__device__ __forceinline__ void stage_spin_tile(const SweepArgs& a, int w, int i0, int j0, uint32_t* s_v) {
    if (a.g.L >= 2 * kTI && a.g.Lc >= 2 * kTJ)
        stage_spin_tile<true>(a, w, i0, j0, s_v);
    else
        stage_spin_tile<false>(a, w, i0, j0, s_v);
}

// Stage the hidden words of cells i0 - 1 .. i0 + TI - 1 x j0 - 1 .. j0 + TJ - 1
// (wrapped) of half-word w into s_h[(TI + 1)][(TJ + 1)][32], 16 bytes per
// load, in batches whose loads are all issued before their stores.
// kOneWrap: W > TI and Wc > TJ, so i0 - 1 + li in [-1, W + TI - 2] (and the
// same for columns) wraps with one add or subtraction of W (Wc).
template <bool kOneWrap>
__device__ __forceinline__ void stage_hidden_halo(const SweepArgs& a, int w, int i0, int j0, uint32_t* s_h) {
    constexpr int HS = kTJ + 1, NQ = (kTI + 1) * HS * 8;  // 8 uint4 per cell
    constexpr int IT = (NQ + kStreamVisThreads - 1) / kStreamVisThreads;
    constexpr int B = 5;  // loads in flight per thread
    const int W = a.g.W, Wc = a.g.Wc;
    const uint4* hw = reinterpret_cast<const uint4*>(a.h + static_cast<size_t>(w) * a.g.n_cells * 32);
#pragma unroll
    for (int k0 = 0; k0 < IT; k0 += B) {
        uint4 val[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int x = threadIdx.x + (k0 + k) * kStreamVisThreads;
            const int lcell = x >> 3, q = x & 7;
            const int li = lcell / HS, lj = lcell - (lcell / HS) * HS;
            int gi = i0 - 1 + li, gj = j0 - 1 + lj;
            if (kOneWrap) {
                gi += gi < 0 ? W : 0;
                gi -= gi >= W ? W : 0;
                gj += gj < 0 ? Wc : 0;
                gj -= gj >= Wc ? Wc : 0;
            } else {
                gi = (gi % W + W) % W;
                gj = (gj % Wc + Wc) % Wc;
            }
            val[k] = make_uint4(0u, 0u, 0u, 0u);
            if (k0 + k < IT && x < NQ) val[k] = hw[(gi * Wc + gj) * 8 + q];
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int x = threadIdx.x + (k0 + k) * kStreamVisThreads;
            if (k0 + k < IT && x < NQ) reinterpret_cast<uint4*>(s_h)[x] = val[k];
        }
    }
}

// Hidden half-step of one tile: v tile rows 2 i0 .. 2 i0 + 2 TI and columns
// 2 j0 .. 2 j0 + 2 TJ (wrapped), the lanes' hidden words out to
// h[word][cell][32].
template <bool kPaper>
__global__ void __launch_bounds__(kStreamThreads, CRBM_STREAM_MIN_BLOCKS) k_stream_hidden(const SweepArgs a, uint32_t t) {
    __shared__ __align__(16) uint32_t s_th[kCanonTh];
    __shared__ uint32_t s_v[(2 * kTI + 1) * (2 * kTJ + 1)];
    __shared__ __align__(16) uint32_t s_h[kTI * kTJ * 32];
    __shared__ uint4 s_q[kTI * kTJ][2];  // per tile cell: hidden_call_words
    __shared__ int s_bos[32];            // rung of each replica slot
    const Geometry& g = a.g;
    const int W = g.W, Wc = g.Wc;
    const int w = blockIdx.y;
    const int tiles_j = (Wc + kTJ - 1) / kTJ;
    const int i0 = (blockIdx.x / tiles_j) * kTI, j0 = (blockIdx.x % tiles_j) * kTJ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const uint32_t* gt = a.ctab + static_cast<size_t>(w) * kCanonTab;
    for (int x = threadIdx.x; x < kCanonTh; x += blockDim.x) s_th[x] = gt[x];
    constexpr int VS = 2 * kTJ + 1;
    stage_spin_tile(a, w, i0, j0, s_v);
    stage_rungs(a, w, s_bos);
    const uint32_t chain = static_cast<uint32_t>(w) * 32u + lane;
    const Round0Lane r0l = round0_lane(chain);
    const Round1Sweep rs = round1_sweep(r0l.hi ^ t ^ a.rk[0], a.rk);
    const int ni = min(kTI, W - i0), nj = min(kTJ, Wc - j0);
    // the warp-uniform Philox words of each cell, once per CTA instead of once per warp-cell
    for (int x = threadIdx.x; x < kTI * kTJ; x += blockDim.x) {
        const int li = x / kTJ, lj = x - li * kTJ;
        if (li < ni && lj < nj)
            hidden_call_words(static_cast<uint32_t>((i0 + li) * Wc + j0 + lj), a.rk, s_q[x][0], s_q[x][1]);
    }
    __syncthreads();
    const LaneConst lc = lane_const(lane, s_bos[lane]);
    // warp = columns lj of the tile, cells walked down the column
    for (int lj = warp; lj < nj; lj += nwarp) {
        const uint32_t* v = s_v + 2 * lj;
        uint32_t* hp = s_h + lj * 32 + lane;
        const uint4* q = s_q[lj];
        for (int li = 0; li < ni; ++li, v += 2 * VS, hp += kTJ * 32, q += 2 * kTJ)
            *hp = kPaper ? hidden_cell_paper(v, VS, s_th, rs, r0l.lo, q[0], q[1], a.rk, lc)
                         : hidden_cell(v, VS, s_th, rs, r0l.lo, q[0], q[1], a.rk, lc);
    }
    __syncthreads();
    // tile rows of hidden words are contiguous runs of nj * 32 words in h
    for (int x = threadIdx.x; x < kTI * kTJ * 8; x += blockDim.x) {
        const int li = x / (kTJ * 8), rest = x - li * (kTJ * 8);
        if (li >= ni || rest >= nj * 8) continue;
        reinterpret_cast<uint4*>(a.h + (static_cast<size_t>(w) * g.n_cells + (i0 + li) * Wc + j0) * 32)[rest] =
            reinterpret_cast<const uint4*>(s_h)[x];
    }
}

// Visible half-step of one tile: hidden words of the tile cells plus the row
// of cells above and the column to the left (wrapped), new spins out.
// Three CTAs per SM (its shared memory) leave room for 85 registers a thread:
// paper precision takes 72 (0.9 % faster than at 64); exact precision is
// 0.4 % faster held to 64.
template <bool kPaper>
__global__ void __launch_bounds__(kStreamVisThreads, kPaper ? 3 : CRBM_STREAM_VIS_MIN_BLOCKS)
    k_stream_visible(const SweepArgs a, uint32_t t) {
    __shared__ __align__(16) uint32_t s_tv[4 * 32 * 32];
    __shared__ __align__(16) uint32_t s_h[(kTI + 1) * (kTJ + 1) * 32];
    __shared__ uint32_t s_o[2 * kTI * 2 * kTJ];
    __shared__ uint4 s_q[kTI * kTJ];  // per tile cell: visible_call_words
    __shared__ int s_bos[32];         // rung of each replica slot
    const Geometry& g = a.g;
    const int L = g.L, Lc = g.Lc, W = g.W, Wc = g.Wc, N = g.N;
    const int w = blockIdx.y;
    const int tiles_j = (Wc + kTJ - 1) / kTJ;
    const int i0 = (blockIdx.x / tiles_j) * kTI, j0 = (blockIdx.x % tiles_j) * kTJ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const uint4* gt = reinterpret_cast<const uint4*>(a.ctab + static_cast<size_t>(w) * kCanonTab + kCanonTh);
    for (int x = threadIdx.x; x < 4 * 32 * 32 / 4; x += blockDim.x) reinterpret_cast<uint4*>(s_tv)[x] = gt[x];
    constexpr int HS = kTJ + 1;
    if (W > kTI && Wc > kTJ)
        stage_hidden_halo<true>(a, w, i0, j0, s_h);
    else
        stage_hidden_halo<false>(a, w, i0, j0, s_h);
    stage_rungs(a, w, s_bos);
    const uint32_t chain = static_cast<uint32_t>(w) * 32u + lane;
    const Round0Lane r0l = round0_lane(chain);
    const Round1Sweep rs = round1_sweep(r0l.hi ^ t ^ a.rk[0], a.rk);
    constexpr int VO = 2 * kTJ;
    const int ni = min(kTI, W - i0), nj = min(kTJ, Wc - j0);
    for (int x = threadIdx.x; x < kTI * kTJ; x += blockDim.x) {
        const int li = x / kTJ, lj = x - li * kTJ;
        if (li < ni && lj < nj) {
            const uint32_t cell = static_cast<uint32_t>((i0 + li) * Wc + j0 + lj);
            s_q[x] = kPaper ? visible_call_words_paper(cell, a.rk) : visible_call_words(cell, a.rk);
        }
    }
    __syncthreads();
    const LaneConst lc = lane_const(lane, s_bos[lane]);
    for (int lj = warp; lj < nj; lj += nwarp) {
        const uint32_t* ho = s_h + (HS + lj + 1) * 32 + lane;
        uint32_t* o = s_o + 2 * lj;
        const uint4* q = s_q + lj;
        for (int li = 0; li < ni; ++li, ho += HS * 32, o += 2 * VO, q += kTJ) {
            if (kPaper)
                visible_cell_paper(o, VO, ho[0], ho[-HS * 32], ho[-32], s_tv, rs, r0l.lo, *q, a.rk, lc);
            else
                visible_cell(o, VO, ho[0], ho[-HS * 32], ho[-32], s_tv, rs, r0l.lo, *q, a.rk, lc);
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < 2 * kTI * VO; x += blockDim.x) {
        const int r = x / VO, c = x - (x / VO) * VO;
        const int R = 2 * i0 + r, C = 2 * j0 + c;
        if (R >= L || C >= Lc) continue;
        a.v[vidx(w, N, R * Lc + C)] = s_o[x];
    }
}

// ---- bit-plane uniforms (CRBM_RNG_BITPLANE) in the streamed layout ----
// The same word-parallel comparison as the SMEM bit-plane sweep
// (crbm_bitplane.cu): a thread takes one node of a tile for the 32 chains of
// the half-word, and the hidden units travel through HBM bit-sliced, one
// word per (cell, filter): h[word][cell][10].

// Hidden half-step of one tile: the spin tile (halo included) in, the tile's
// hidden words out.
__global__ void __launch_bounds__(kStreamThreads) k_stream_bp_hidden(const SweepArgs a, uint32_t t) {
    constexpr int kCap = kTI * kTJ * 10 / 4;  // straggler list: a quarter of the tile's nodes
    __shared__ __align__(16) uint32_t s_tab[kBpTab];
    __shared__ uint32_t s_v[(2 * kTI + 1) * (2 * kTJ + 1)];
    __shared__ uint32_t s_h[kTI * kTJ * 10];
    __shared__ uint2 s_list[kCap];
    __shared__ int s_off[2][10];  // the filters' endpoint offsets in the staged tile
    __shared__ int s_nst;
    const Geometry& g = a.g;
    const int W = g.W, Wc = g.Wc;
    const int w = blockIdx.y;
    const int tiles_j = (Wc + kTJ - 1) / kTJ;
    const int i0 = (blockIdx.x / tiles_j) * kTI, j0 = (blockIdx.x % tiles_j) * kTJ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    constexpr int VS = 2 * kTJ + 1;
    const uint32_t* gt = a.ctab + static_cast<size_t>(w) * kCanonTab;
    for (int x = threadIdx.x; x < kBpTab; x += blockDim.x) s_tab[x] = gt[x];
    if (threadIdx.x < 10) {
        const int k = threadIdx.x;
        s_off[0][k] = g.r1[k] * VS + g.c1[k];
        s_off[1][k] = g.r2[k] * VS + g.c2[k];
    }
    if (threadIdx.x == 0) s_nst = 0;
    stage_spin_tile(a, w, i0, j0, s_v);
    __syncthreads();
    const uint32_t fl0 = s_tab[kBpFlip], fl1 = s_tab[kBpFlip + 1];
    const int ni = min(kTI, W - i0), nj = min(kTJ, Wc - j0), nn = ni * nj * 10;
    const SmallDiv div_nj(nj);
    const uint64_t pw = static_cast<uint64_t>(kPhiloxM1) * static_cast<uint32_t>(w);
    const uint32_t Yw = static_cast<uint32_t>(pw);
    const Round1Sweep rs = round1_sweep(static_cast<uint32_t>(pw >> 32) ^ a.rk[0] ^ t, a.rk);
    // node nd of the tile: its threshold planes (P: m = 2, M: m = -2, Z: m = 0), Philox cell words
    // and the index of its hidden word in s_h
    struct Hid {
        uint32_t P, M, Z, c2;
        const uint32_t* tp;
        Round2Cell r2;
        int out;
    };
    auto hidden_node = [&](int nd) {
        const int lc = nd / 10, k = nd - lc * 10;
        const int li = div_nj(lc), lj = lc - li * nj;
        const uint32_t cls = k >= 8 ? 1u : 0u;
        const uint32_t* v = s_v + 2 * li * VS + 2 * lj;
        const uint32_t e1 = v[s_off[0][k]];
        const uint32_t e2 = v[s_off[1][k]] ^ (cls ? fl1 : fl0);
        const uint32_t cell = static_cast<uint32_t>((i0 + li) * Wc + j0 + lj);
        const uint64_t pc = static_cast<uint64_t>(kPhiloxM0) * cell;
        return Hid{e1 & e2, ~(e1 | e2), e1 ^ e2,
                   static_cast<uint32_t>(pc >> 32) ^ a.rk[1] ^ (kTagBitplane + 8u * static_cast<uint32_t>(k)),
                   s_tab + kBpHidPlanes + cls * 96u, round2_cell(rs.hik ^ static_cast<uint32_t>(pc)),
                   (li * kTJ + lj) * 10 + k};
    };
    for (int base = warp * 32; base < nn; base += nwarp * 32) {
        const int node = base + lane;
        const bool valid = node < nn;
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
        if (bp::push_straggler(static_cast<uint32_t>(node), eq, &s_nst, s_list, kCap, lane)) eq = 0u;
#pragma unroll 1
        for (uint32_t j = 2; j < 8u; ++j) {  // only where the list was full
            if (!__any_sync(0xffffffffu, eq != 0u)) break;
            planes(philox_from_round2(Yw, rs, hn.r2, hn.c2 ^ j, a.rk), j);
        }
        if (valid) s_h[hn.out] = lt;  // final, or the decided part of a straggler
    }
    __syncthreads();
    const int n_st = min(s_nst, kCap);
    for (int base = warp * 32; base < n_st; base += nwarp * 32) {
        const bool valid = base + lane < n_st;
        const uint2 e = valid ? s_list[base + lane] : make_uint2(0u, 0u);
        const Hid hn = hidden_node(static_cast<int>(e.x));
        uint32_t lt = s_h[hn.out], eq = e.y;
#pragma unroll 1
        for (uint32_t j = 2; j < 8u; ++j) {
            if (!__any_sync(0xffffffffu, eq != 0u)) break;
            bp::hidden_planes(philox_from_round2(Yw, rs, hn.r2, hn.c2 ^ j, a.rk), hn.tp + 4u * j, hn.P, hn.M, 0u, lt,
                              eq);
        }
        if (valid) s_h[hn.out] = lt;
    }
    __syncthreads();
    // tile rows of hidden words are runs of 10 nj words in h
    for (int x = threadIdx.x; x < kTI * kTJ * 10; x += blockDim.x) {
        const int li = x / (kTJ * 10), rest = x - li * (kTJ * 10);
        if (li >= ni || rest >= nj * 10) continue;
        a.h[(static_cast<size_t>(w) * g.n_cells + (i0 + li) * Wc + j0) * 10 + rest] = s_h[x];
    }
}

// Visible half-step of one tile: the hidden words of the tile's cells and of
// the row above and the column to the left (wrapped) in, new spins out.
__global__ void __launch_bounds__(kStreamVisThreads, CRBM_STREAM_MIN_BLOCKS) k_stream_bp_visible(const SweepArgs a, uint32_t t) {
    constexpr int HS = kTJ + 1;
    __shared__ __align__(16) uint32_t s_tab[kBpTab];
    __shared__ uint32_t s_h[(kTI + 1) * HS * 10];
    __shared__ uint32_t s_o[2 * kTI * 2 * kTJ];
    constexpr int kCap = 2 * kTI * 2 * kTJ / 4;  // straggler list: a quarter of the tile's spins
    __shared__ uint2 s_list[kCap];
    __shared__ int s_inc[4][5];  // per spin class x: hidden word offset (cell row, column, filter) | flags
    __shared__ int s_nst;
    const Geometry& g = a.g;
    const int L = g.L, Lc = g.Lc, W = g.W, Wc = g.Wc, N = g.N;
    const int w = blockIdx.y;
    const int tiles_j = (Wc + kTJ - 1) / kTJ;
    const int i0 = (blockIdx.x / tiles_j) * kTI, j0 = (blockIdx.x % tiles_j) * kTJ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const uint32_t* gt = a.ctab + static_cast<size_t>(w) * kCanonTab;
    for (int x = threadIdx.x; x < kBpTab; x += blockDim.x) s_tab[x] = gt[x];
    if (threadIdx.x == 0) s_nst = 0;
    if (threadIdx.x < 4) {
        // the five filters touching the spin at window offset (r, c): endpoints
        // at (r, c) of the own cell, (r + 2, c) of the cell above, (r, c + 2) of
        // the cell to the left; J filters first, the J' filter last
        const int x = threadIdx.x, r = x >> 1, c = x & 1;
        int nJ = 0;
        for (int k = 0; k < 10; ++k)
            for (int e = 0; e < 2; ++e) {
                const int er = e ? g.r2[k] : g.r1[k], ec = e ? g.c2[k] : g.c1[k];
                int dr = -1, dc = -1;
                if (er == r && ec == c) dr = 1, dc = 1;
                else if (er == r + 2 && ec == c) dr = 0, dc = 1;
                else if (er == r && ec == c + 2) dr = 1, dc = 0;
                if (dr < 0) continue;
                const int off = (dr * HS + dc) * 10 + k;  // relative to the spin's cell at (li, lj) -> (li + 1, lj + 1)
                const int v = off | (e << 16);
                if (g.cls[k] == 0) s_inc[x][nJ++] = v;
                else s_inc[x][4] = v;
            }
    }
    // hidden halo: cells (i0 - 1 .. i0 + ni - 1) x (j0 - 1 .. j0 + nj - 1), wrapped
    const int ni = min(kTI, W - i0), nj = min(kTJ, Wc - j0);
    const uint32_t* hw = a.h + static_cast<size_t>(w) * g.n_cells * 10;
    for (int x = threadIdx.x; x < (kTI + 1) * HS * 10; x += blockDim.x) {
        const int lc = x / 10, k = x - lc * 10;
        const int li = lc / HS, lj = lc - li * HS;
        if (li > ni || lj > nj) continue;
        // li <= ni <= W - i0 (and lj <= nj <= Wc - j0): i0 - 1 + li lies in [-1, W - 1]
        int gi = i0 - 1 + li, gj = j0 - 1 + lj;
        gi += gi < 0 ? W : 0;
        gj += gj < 0 ? Wc : 0;
        s_h[x] = hw[(gi * Wc + gj) * 10 + k];
    }
    __syncthreads();
    const uint32_t fl0 = s_tab[kBpFlip], fl1 = s_tab[kBpFlip + 1];
    const int nr = 2 * ni, nc = 2 * nj, nn = nr * nc;
    const SmallDiv div_nc(nc);
    constexpr int VO = 2 * kTJ;
    const uint64_t pw = static_cast<uint64_t>(kPhiloxM1) * static_cast<uint32_t>(w);
    const uint32_t Yw = static_cast<uint32_t>(pw);
    const Round1Sweep rs = round1_sweep(static_cast<uint32_t>(pw >> 32) ^ a.rk[0] ^ t, a.rk);
    const uint32_t* tv = s_tab + kBpVisPlanes;
    // spin sx of the tile: its J' bit hp, the bit-sliced count n4 of its four J incidences, Philox
    // cell words and its index in s_o
    struct Vis {
        uint32_t hp, c2;
        bp::Count4 n4;
        Round2Cell r2;
        int out;
    };
    auto visible_node = [&](int sd) {
        const int R = div_nc(sd), C = sd - R * nc;  // tile-local spin row and column
        const int x = 2 * (R & 1) + (C & 1);
        const uint32_t* hc = s_h + (((R >> 1) + 1) * HS + (C >> 1) + 1) * 10;  // own cell's words
        auto hin = [&](int v, uint32_t fl) {
            return hc[(v & 0xFFFF) - (HS + 1) * 10] ^ ((v >> 16) ? fl : 0u);
        };
        const uint32_t h0 = hin(s_inc[x][0], fl0), h1 = hin(s_inc[x][1], fl0), h2 = hin(s_inc[x][2], fl0),
                       h3 = hin(s_inc[x][3], fl0);
        const uint32_t cell = static_cast<uint32_t>((i0 + (R >> 1)) * Wc + j0 + (C >> 1));
        const uint64_t pc = static_cast<uint64_t>(kPhiloxM0) * cell;
        return Vis{hin(s_inc[x][4], fl1),
                   static_cast<uint32_t>(pc >> 32) ^ a.rk[1] ^ (kTagBitplane + 8u * (10u + static_cast<uint32_t>(x))),
                   bp::count4(h0, h1, h2, h3), round2_cell(rs.hik ^ static_cast<uint32_t>(pc)), R * VO + C};
    };
    auto planes = [&](const Vis& vn, const U4& q, uint32_t j, uint32_t& lt, uint32_t& eq) {
        const uint4 T = bp::visible_planes(tv + 4u * j, vn.hp, vn.n4);
        bp::plane_step(q.x, T.x, lt, eq);
        bp::plane_step(q.y, T.y, lt, eq);
        bp::plane_step(q.z, T.z, lt, eq);
        bp::plane_step(q.w, T.w, lt, eq);
    };
    for (int base = warp * 32; base < nn; base += nwarp * 32) {
        const int sx = base + lane;
        const bool valid = sx < nn;
        const Vis vn = visible_node(valid ? sx : 0);
        uint32_t lt = 0u, eq = valid ? 0xffffffffu : 0u;
        // calls 0 and 1 (a loop, so that the threshold planes are not held in registers across
        // tiles), then the open spins to the straggler list
#pragma unroll 1
        for (uint32_t j = 0; j < 2u; ++j) planes(vn, philox_from_round2(Yw, rs, vn.r2, vn.c2 ^ j, a.rk), j, lt, eq);
        if (bp::push_straggler(static_cast<uint32_t>(sx), eq, &s_nst, s_list, kCap, lane)) eq = 0u;
#pragma unroll 1
        for (uint32_t j = 2; j < 8u; ++j) {  // only where the list was full
            if (!__any_sync(0xffffffffu, eq != 0u)) break;
            planes(vn, philox_from_round2(Yw, rs, vn.r2, vn.c2 ^ j, a.rk), j, lt, eq);
        }
        if (valid) s_o[vn.out] = lt;  // final, or the decided part of a straggler
    }
    __syncthreads();
    const int n_st = min(s_nst, kCap);
    for (int base = warp * 32; base < n_st; base += nwarp * 32) {
        const bool valid = base + lane < n_st;
        const uint2 e = valid ? s_list[base + lane] : make_uint2(0u, 0u);
        const Vis vn = visible_node(static_cast<int>(e.x));
        uint32_t lt = s_o[vn.out], eq = e.y;
#pragma unroll 1
        for (uint32_t j = 2; j < 8u; ++j) {
            if (!__any_sync(0xffffffffu, eq != 0u)) break;
            planes(vn, philox_from_round2(Yw, rs, vn.r2, vn.c2 ^ j, a.rk), j, lt, eq);
        }
        if (valid) s_o[vn.out] = lt;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < 2 * kTI * VO; x += blockDim.x) {
        const int r = x / VO, c = x - (x / VO) * VO;
        const int R = 2 * i0 + r, C = 2 * j0 + c;
        if (r >= nr || c >= nc || R >= L || C >= Lc) continue;
        a.v[vidx(w, N, R * Lc + C)] = s_o[x];
    }
}

// Measurement counts of one tile (anti-aligned J / J' filters and +1 spins
// per chain), summed over the CTA in shared memory, then into cnt[chain][3].
__global__ void __launch_bounds__(kStreamThreads, CRBM_STREAM_MIN_BLOCKS) k_stream_count(const SweepArgs a) {
    __shared__ uint32_t s_v[(2 * kTI + 1) * (2 * kTJ + 1)];
    __shared__ int s_cnt[96];
    const Geometry& g = a.g;
    const int W = g.W, Wc = g.Wc;
    const int w = blockIdx.y;
    const int tiles_j = (Wc + kTJ - 1) / kTJ;
    const int i0 = (blockIdx.x / tiles_j) * kTI, j0 = (blockIdx.x % tiles_j) * kTJ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    constexpr int VS = 2 * kTJ + 1;
    stage_spin_tile(a, w, i0, j0, s_v);
    for (int x = threadIdx.x; x < 96; x += blockDim.x) s_cnt[x] = 0;
    __syncthreads();
    int anti0 = 0, anti1 = 0, pos = 0;
    const int ni = min(kTI, W - i0), nj = min(kTJ, Wc - j0);
    for (int lj = warp; lj < nj; lj += nwarp)
        for (int li = 0; li < ni; ++li)
            count_cell(s_v + 2 * li * VS + 2 * lj, 0, VS, 2 * VS, 0, 1, 2, lane, anti0, anti1, pos);
    atomicAdd(&s_cnt[lane], anti0);
    atomicAdd(&s_cnt[32 + lane], anti1);
    atomicAdd(&s_cnt[64 + lane], pos);
    __syncthreads();
    if (threadIdx.x < 96) {
        const int kind = threadIdx.x >> 5, l = threadIdx.x & 31;
        atomicAdd(&a.cnt[(static_cast<size_t>(w) * 32 + l) * 3 + kind], s_cnt[threadIdx.x]);
    }
}

// Turn the per-chain counts into (NJ, NJ', M), append the series entry,
// accumulate the sums and clear the counts.
__global__ void k_stream_finalize(const SweepArgs a, int64_t meas, int64_t sweeps_done) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.n_chains_padded) return;
    const Geometry& g = a.g;
    int* cn = a.cnt + static_cast<size_t>(c) * 3;
    const int64_t nJ = g.n_real_bonds[0] - 2 * static_cast<int64_t>(cn[0]);
    const int64_t nP = g.n_real_bonds[1] - 2 * static_cast<int64_t>(cn[1]);
    const int64_t M = 2 * static_cast<int64_t>(cn[2]) - g.N;
    cn[0] = cn[1] = cn[2] = 0;
    if (meas < a.series_len) {
        int32_t* e = a.series + (static_cast<size_t>(meas) * a.n_chains_padded + c) * 3;
        e[0] = static_cast<int32_t>(nJ);
        e[1] = static_cast<int32_t>(nP);
        e[2] = static_cast<int32_t>(M);
    }
    int64_t* s = a.sums + static_cast<size_t>(c) * kNSum;
    s[0] += 1;
    s[1] += nJ;
    s[2] += nP;
    s[3] += M;
    s[4] += M < 0 ? -M : M;
    s[5] += nJ * nJ;
    s[6] += nP * nP;
    s[7] += M * M;
    s[8] += nJ * nP;
    s[9] += nJ * M;
    s[10] += nP * M;
    if (a.hit) {  // time to solution: first measured sweep at or below the target energy
        int64_t* ht = a.hit + 2 * static_cast<size_t>(c);
        const int32_t* q = a.hit_q + 4 * static_cast<size_t>(c);
        const int64_t E = static_cast<int64_t>(q[0]) * nJ + static_cast<int64_t>(q[1]) * nP -
                          static_cast<int64_t>(q[2]) * M;
        if (ht[1] < 0 && E <= ht[0]) ht[1] = sweeps_done;
    }
}

// Post-sweep step with replica exchange: one warp per 32-chain half-word w
// (a ladder), lane = slot for the counts and rung for the rest, exactly the
// SMEM kernels' step (post_sweep_warp): rung k's measurement from the slot
// that holds it into row 32 w + k of the sums and series, then the
// exchange round, and the new slot-of-rung array back to sob.  Half-words
// past the last ladder (padding of the 64-chain groups) only clear their
// counts.
__global__ void __launch_bounds__(32) k_stream_post_pt(const SweepArgs a, int64_t meas, uint32_t t, int do_meas,
                                                       int do_swap) {
    __shared__ int s_cnt[96], s_sob[32], s_bos[32];
    __shared__ int64_t s_acc[kNSum * 32];
    const int w = blockIdx.x, lane = threadIdx.x;
    int* cn = a.cnt + (static_cast<size_t>(w) * 32 + lane) * 3;
    s_cnt[lane] = cn[0];
    s_cnt[32 + lane] = cn[1];
    s_cnt[64 + lane] = cn[2];
    cn[0] = cn[1] = cn[2] = 0;
    if (w >= a.n_chains / 32) return;
    const size_t row = static_cast<size_t>(w) * 32 + lane;
    const int sob = a.sob[row];
    s_sob[lane] = sob;
    s_bos[sob] = lane;
    if (do_meas)
        for (int x = 0; x < kNSum; ++x) s_acc[x * 32 + lane] = a.sums[row * kNSum + x];
    __syncwarp();
    post_sweep_warp(a, s_cnt, s_sob, s_bos, lane, w, t, do_meas != 0, do_swap != 0, meas, s_acc);
    __syncwarp();
    if (do_meas)
        for (int x = 0; x < kNSum; ++x) a.sums[row * kNSum + x] = s_acc[x * 32 + lane];
    if (do_swap) a.sob[row] = s_sob[lane];
}

}  // namespace

cudaError_t launch_sweep_stream(const SweepArgs& a, cudaStream_t st, int64_t* launches) {
    const int tiles = ((a.g.W + kTI - 1) / kTI) * ((a.g.Wc + kTJ - 1) / kTJ);
    const dim3 grid(tiles, a.n_words);
    int64_t meas = a.meas0;
    for (int it = 0; it < a.n_sweeps; ++it) {
        const uint32_t t = a.t0 + static_cast<uint32_t>(it);
        if (a.g.bitplane) {
            k_stream_bp_hidden<<<grid, kStreamThreads, 0, st>>>(a, t);
            k_stream_bp_visible<<<grid, kStreamVisThreads, 0, st>>>(a, t);
        } else if (a.g.paper) {
            k_stream_hidden<true><<<grid, kStreamThreads, 0, st>>>(a, t);
            k_stream_visible<true><<<grid, kStreamVisThreads, 0, st>>>(a, t);
        } else {
            k_stream_hidden<false><<<grid, kStreamThreads, 0, st>>>(a, t);
            k_stream_visible<false><<<grid, kStreamVisThreads, 0, st>>>(a, t);
        }
        *launches += 2;
        const bool do_meas = a.measure_every > 0 && (t + 1u) % static_cast<uint32_t>(a.measure_every) == 0u;
        const bool do_swap = a.swap_every > 0 && (t + 1u) % static_cast<uint32_t>(a.swap_every) == 0u;
        if (do_meas || do_swap) {
            k_stream_count<<<grid, kStreamThreads, 0, st>>>(a);
            if (a.swap_every > 0)
                k_stream_post_pt<<<a.n_words, 32, 0, st>>>(a, meas, t, do_meas ? 1 : 0, do_swap ? 1 : 0);
            else
                k_stream_finalize<<<(a.n_chains_padded + 255) / 256, 256, 0, st>>>(a, meas,
                                                                                   static_cast<int64_t>(t) + 1);
            *launches += 2;
            if (do_meas) ++meas;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace crbm
