// Streamed sweep for lattices too large for shared memory (canonical SS
// filters, even periodic L): spins and hidden units live in HBM and one sweep
// is two launches, the hidden half-step (Eq. 9) then the visible half-step
// (Eq. 10).  Spins are stored as 64-chain words, two 32-bit halves per site
// ([group][site][2]); a CTA works on one 32-chain half and one tile of cells,
// staging its tile (plus a one-site / one-cell halo) in shared memory with
// plain coalesced loads, and reuses the per-cell cores of the SMEM path.
#include "crbm_canon_core.cuh"

namespace crbm {
namespace {

using namespace dev;
using namespace canon;

constexpr int kTI = 16;  // tile rows of cells
constexpr int kTJ = 16;  // tile columns of cells
constexpr int kStreamThreads = 256;

__device__ __forceinline__ size_t vidx(int w, int N, int s) {
    return (static_cast<size_t>(w >> 1) * N + s) * 2 + (w & 1);
}

// Hidden half-step of one tile: v tile rows 2 i0 .. 2 i0 + 2 TI and columns
// 2 j0 .. 2 j0 + 2 TJ (wrapped), the lanes' hidden words out to
// h[word][cell][32].
__global__ void __launch_bounds__(kStreamThreads, 4) k_stream_hidden(const SweepArgs a, uint32_t t) {
    __shared__ __align__(16) uint32_t s_th[kCanonTh];
    __shared__ uint32_t s_v[(2 * kTI + 1) * (2 * kTJ + 1)];
    __shared__ uint32_t s_h[kTI * kTJ * 32];
    const Geometry& g = a.g;
    const int L = g.L, W = g.W, N = g.N;
    const int w = blockIdx.y;
    const int tiles_j = (W + kTJ - 1) / kTJ;
    const int i0 = (blockIdx.x / tiles_j) * kTI, j0 = (blockIdx.x % tiles_j) * kTJ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const uint32_t* gt = a.ctab + static_cast<size_t>(w) * kCanonTab;
    for (int x = threadIdx.x; x < kCanonTh; x += blockDim.x) s_th[x] = gt[x];
    constexpr int VS = 2 * kTJ + 1;
    for (int x = threadIdx.x; x < (2 * kTI + 1) * VS; x += blockDim.x) {
        const int r = x / VS, c = x - (x / VS) * VS;
        const int R = (2 * i0 + r) % L, C = (2 * j0 + c) % L;
        s_v[x] = a.v[vidx(w, N, R * L + C)];
    }
    const uint32_t chain = static_cast<uint32_t>(w) * 32u + lane;
    const LaneConst lc = lane_const(lane, lane);
    const Round0Lane r0l = round0_lane(chain);
    const uint32_t X = r0l.hi ^ t ^ a.rk[0];
    __syncthreads();
    for (int lcell = warp; lcell < kTI * kTJ; lcell += nwarp) {
        const int li = lcell / kTJ, lj = lcell - (lcell / kTJ) * kTJ;
        const int gi = i0 + li, gj = j0 + lj;
        if (gi >= W || gj >= W) continue;
        const int r0 = 2 * li * VS, c0 = 2 * lj;
        s_h[lcell * 32 + lane] =
            hidden_cell(s_v, r0, r0 + VS, r0 + 2 * VS, c0, c0 + 1, c0 + 2, s_th, X, r0l.lo,
                        round0_cell(static_cast<uint32_t>(gi * W + gj), a.rk[1]), a.rk, lc);
    }
    __syncthreads();
    const int nj = min(kTJ, W - j0);
    for (int x = threadIdx.x; x < kTI * kTJ * 32; x += blockDim.x) {
        const int li = x / (kTJ * 32), rest = x - li * (kTJ * 32);
        if (i0 + li >= W || rest >= nj * 32) continue;
        a.h[(static_cast<size_t>(w) * g.n_cells + (i0 + li) * W + j0) * 32 + rest] = s_h[x];
    }
}

// Visible half-step of one tile: hidden words of the tile cells plus the row
// of cells above and the column to the left (wrapped), new spins out.
__global__ void __launch_bounds__(kStreamThreads, 4) k_stream_visible(const SweepArgs a, uint32_t t) {
    __shared__ __align__(16) uint32_t s_tv[4 * 32 * 32];
    __shared__ uint32_t s_h[(kTI + 1) * (kTJ + 1) * 32];
    __shared__ uint32_t s_o[2 * kTI * 2 * kTJ];
    const Geometry& g = a.g;
    const int L = g.L, W = g.W, N = g.N;
    const int w = blockIdx.y;
    const int tiles_j = (W + kTJ - 1) / kTJ;
    const int i0 = (blockIdx.x / tiles_j) * kTI, j0 = (blockIdx.x % tiles_j) * kTJ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const uint4* gt = reinterpret_cast<const uint4*>(a.ctab + static_cast<size_t>(w) * kCanonTab + kCanonTh);
    for (int x = threadIdx.x; x < 4 * 32 * 32 / 4; x += blockDim.x) reinterpret_cast<uint4*>(s_tv)[x] = gt[x];
    constexpr int HS = kTJ + 1;
    for (int x = threadIdx.x; x < (kTI + 1) * HS * 32; x += blockDim.x) {
        const int lcell = x >> 5, k = x & 31;
        const int li = lcell / HS, lj = lcell - (lcell / HS) * HS;
        const int gi = (i0 - 1 + li + W) % W, gj = (j0 - 1 + lj + W) % W;
        s_h[x] = a.h[(static_cast<size_t>(w) * g.n_cells + gi * W + gj) * 32 + k];
    }
    const uint32_t chain = static_cast<uint32_t>(w) * 32u + lane;
    const LaneConst lc = lane_const(lane, lane);
    const Round0Lane r0l = round0_lane(chain);
    const uint32_t X = r0l.hi ^ t ^ a.rk[0];
    __syncthreads();
    constexpr int VO = 2 * kTJ;
    for (int lcell = warp; lcell < kTI * kTJ; lcell += nwarp) {
        const int li = lcell / kTJ, lj = lcell - (lcell / kTJ) * kTJ;
        const int gi = i0 + li, gj = j0 + lj;
        if (gi >= W || gj >= W) continue;
        const uint32_t* ho = s_h + ((li + 1) * HS + lj + 1) * 32 + lane;
        visible_cell(s_o + 2 * li * VO + 2 * lj, VO, ho[0], ho[-HS * 32], ho[-32], s_tv, X, r0l.lo,
                     round0_cell(static_cast<uint32_t>(gi * W + gj), a.rk[1]), a.rk, lc);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < 2 * kTI * VO; x += blockDim.x) {
        const int r = x / VO, c = x - (x / VO) * VO;
        const int R = 2 * i0 + r, C = 2 * j0 + c;
        if (R >= L || C >= L) continue;
        a.v[vidx(w, N, R * L + C)] = s_o[x];
    }
}

// Measurement counts of one tile (anti-aligned J / J' filters and +1 spins
// per chain), summed over the CTA in shared memory, then into cnt[chain][3].
__global__ void __launch_bounds__(kStreamThreads, 4) k_stream_count(const SweepArgs a) {
    __shared__ uint32_t s_v[(2 * kTI + 1) * (2 * kTJ + 1)];
    __shared__ int s_cnt[96];
    const Geometry& g = a.g;
    const int L = g.L, W = g.W, N = g.N;
    const int w = blockIdx.y;
    const int tiles_j = (W + kTJ - 1) / kTJ;
    const int i0 = (blockIdx.x / tiles_j) * kTI, j0 = (blockIdx.x % tiles_j) * kTJ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    constexpr int VS = 2 * kTJ + 1;
    for (int x = threadIdx.x; x < (2 * kTI + 1) * VS; x += blockDim.x) {
        const int r = x / VS, c = x - (x / VS) * VS;
        const int R = (2 * i0 + r) % L, C = (2 * j0 + c) % L;
        s_v[x] = a.v[vidx(w, N, R * L + C)];
    }
    for (int x = threadIdx.x; x < 96; x += blockDim.x) s_cnt[x] = 0;
    __syncthreads();
    int anti0 = 0, anti1 = 0, pos = 0;
    for (int lcell = warp; lcell < kTI * kTJ; lcell += nwarp) {
        const int li = lcell / kTJ, lj = lcell - (lcell / kTJ) * kTJ;
        if (i0 + li >= W || j0 + lj >= W) continue;
        const int r0 = 2 * li * VS, c0 = 2 * lj;
        count_cell(s_v, r0, r0 + VS, r0 + 2 * VS, c0, c0 + 1, c0 + 2, lane, anti0, anti1, pos);
    }
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
__global__ void k_stream_finalize(const SweepArgs a, int64_t meas) {
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
}

}  // namespace

cudaError_t launch_sweep_stream(const SweepArgs& a, cudaStream_t st, int64_t* launches) {
    const int tiles = ((a.g.W + kTI - 1) / kTI) * ((a.g.W + kTJ - 1) / kTJ);
    const dim3 grid(tiles, a.n_words);
    int64_t meas = a.meas0;
    for (int it = 0; it < a.n_sweeps; ++it) {
        const uint32_t t = a.t0 + static_cast<uint32_t>(it);
        k_stream_hidden<<<grid, kStreamThreads, 0, st>>>(a, t);
        k_stream_visible<<<grid, kStreamThreads, 0, st>>>(a, t);
        *launches += 2;
        if (a.measure_every > 0 && (t + 1u) % static_cast<uint32_t>(a.measure_every) == 0u) {
            k_stream_count<<<grid, kStreamThreads, 0, st>>>(a);
            k_stream_finalize<<<(a.n_chains_padded + 255) / 256, 256, 0, st>>>(a, meas);
            *launches += 2;
            ++meas;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace crbm
