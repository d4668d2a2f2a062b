// SMEM-resident sweep, canonical SS fast path: a CTA holds one packed word
// (32 chains) -- the whole even, periodic lattice, its hidden layer and the
// lane-expanded tables -- in shared memory and runs a chunk of sweeps on it.
// The sweep body is in crbm_canon_body.cuh, the per-cell cores in
// crbm_canon_core.cuh.
#include <algorithm>

#include "crbm_canon_body.cuh"

#ifndef CRBM_SWEEP_MIN_BLOCKS
#define CRBM_SWEEP_MIN_BLOCKS (CRBM_SWEEP_MAX_THREADS <= 512 ? 2 : 1)  // 64 registers a thread either way
#endif

namespace crbm {
namespace {

using namespace dev;
using namespace canon;

// Persistent form: a grid that fits on the GPU at once works through items
// (word, chunk of `chunk` sweeps).  Chunks of a word run in order, one CTA at
// a time.  state[w] = 2 (chunks of w done) + (1 while a CTA holds w).  A CTA
// claims, with a compare-and-swap on state, the free word with the fewest
// chunks done (warp 0 scans all states with 16-byte loads; ties go to the
// first word in a CTA-dependent scan order), runs its next chunk, publishes
// the word's spins and sums, then releases it with the new count and claims
// again.  A CTA that finds no free unfinished word exits: every unfinished
// word is then held by a running CTA, which claims again after its chunk, so
// no work is left behind and nothing waits.
//
// Two instantiations per variant: one for CTAs of at most kSmallCta threads
// (12 warps, the shape the L=18 grid tunes to) at two CTAs per SM, which may
// take 80 registers a thread and keeps the sweep loop free of spills, and one
// for any CTA, at 64 registers.  A launch takes the first wherever its CTA
// fits it and it holds as many CTAs per SM as the second.
constexpr int kSmallCta = 384;
template <bool kSmemRec, bool kPaper, int kMaxThreads>
__global__ void __launch_bounds__(kMaxThreads, kMaxThreads <= kSmallCta ? 2 : CRBM_SWEEP_MIN_BLOCKS)
    k_sweep_canon_persistent(const SweepArgs a, int chunk, int* state) {
    __shared__ int s_word, s_chunk;
    const int n_chunks = (a.n_sweeps + chunk - 1) / chunk;
    const int nw = a.n_words, nq = (nw + 3) / 4;
    const int K = a.measure_every;
    const int lane = threadIdx.x & 31;
    const unsigned int start = (blockIdx.x * 97u) % static_cast<unsigned int>(nw);
    for (;;) {
        if (threadIdx.x < 32) {
            int word = -1, c = 0;
            for (int tries = 0; tries < (1 << 20) && word < 0; ++tries) {
                int best = 0x7fffffff, bk = 0x7fffffff, bw = -1;  // (chunks done, scan rank, word)
                for (int q = lane; q < nq; q += 32) {
                    const int4 v = __ldcg(reinterpret_cast<const int4*>(state) + q);
                    const int sv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int w = 4 * q + j;
                        const int dw = sv[j] >> 1;
                        const int rank = static_cast<int>((static_cast<unsigned int>(w) + nw - start) %
                                                          static_cast<unsigned int>(nw));
                        if (w < nw && (sv[j] & 1) == 0 && dw < n_chunks &&
                            (dw < best || (dw == best && rank < bk))) {
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
                if (bw < 0) break;  // every unfinished word is held by a running CTA
                if (lane == 0 && atomicCAS(state + bw, 2 * best, 2 * best + 1) == 2 * best) {
                    __threadfence();  // acquire: the previous chunk's stores precede its release
                    word = bw;
                    c = best;
                }
                word = __shfl_sync(0xffffffffu, word, 0);
                c = __shfl_sync(0xffffffffu, c, 0);
            }
            if (lane == 0) {
                s_word = word;
                s_chunk = c;
            }
        }
        __syncthreads();
        const int word = s_word, c = s_chunk;
        if (word < 0) break;
        const uint32_t t0 = a.t0 + static_cast<uint32_t>(c * chunk);
        const int n = min(chunk, a.n_sweeps - c * chunk);
        const int64_t meas0 =
            K > 0 ? a.meas0 + static_cast<int64_t>(t0 / K) - static_cast<int64_t>(a.t0 / K) : a.meas0;
        sweep_canon_body<kSmemRec, false, kPaper>(a, word, t0, n, meas0);
        __syncthreads();  // every thread's state stores are issued
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(state + word, 2 * (c + 1));
        }
    }
}

}  // namespace

bool canon_smem_records(const Geometry& g) {
    constexpr size_t kSmemPerSm = 228 * 1024, kCtaMax = 227 * 1024, kReserve = 1024;
    const size_t base = smem_bytes_canon(g);
    const size_t with = sizeof(uint32_t) * canon_smem_rec_offset(g) + sizeof(uint4) * g.n_cells * kCellRec;
    if (with > kCtaMax) return false;
    const size_t per_sm_base = std::min<size_t>(2, kSmemPerSm / (base + kReserve));
    return kSmemPerSm / (with + kReserve) >= per_sm_base;
}

size_t smem_bytes_canon_launch(const Geometry& g) {
    return canon_smem_records(g)
               ? sizeof(uint32_t) * canon_smem_rec_offset(g) + sizeof(uint4) * g.n_cells * kCellRec
               : smem_bytes_canon(g);
}

size_t smem_bytes_canon(const Geometry& g) { return sizeof(uint32_t) * canon_smem_rec_offset(g); }

namespace {
template <bool kSmemRec, bool kPaper>
cudaError_t launch_persistent(const SweepArgs& a, int warps_per_cta, int chunk, int* sched, cudaStream_t st) {
    const size_t smem = smem_bytes_canon_launch(a.g);
    using Kernel = void (*)(const SweepArgs, int, int*);
    const Kernel big = k_sweep_canon_persistent<kSmemRec, kPaper, CRBM_SWEEP_MAX_THREADS>;
    const Kernel small = k_sweep_canon_persistent<kSmemRec, kPaper, kSmallCta>;
    const int threads = warps_per_cta * 32;
    // the spill-free instantiation where the CTA fits it and it keeps as many CTAs per SM
    int per_sm = 0, per_sm_small = 0, dev = 0, sms = 0;
    cudaError_t e = cudaSuccess;
    for (const Kernel k : {big, small}) {
        if (k == small && threads > kSmallCta) break;
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(k == big ? &per_sm : &per_sm_small, k, threads, smem);
        if (e != cudaSuccess) return e;
    }
    const Kernel kernel = per_sm_small >= per_sm && per_sm_small > 0 ? small : big;
    if (kernel == small) per_sm = per_sm_small;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int n_items = ((a.n_sweeps + chunk - 1) / chunk) * a.n_words;
    const int grid = std::min(std::min(n_items, a.n_words), per_sm * sms);
    e = cudaMemsetAsync(sched, 0, sizeof(int) * (4 + static_cast<size_t>(a.n_words)), st);
    if (e != cudaSuccess) return e;
    kernel<<<grid, warps_per_cta * 32, smem, st>>>(a, chunk, sched);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_canon_persistent(const SweepArgs& a, int warps_per_cta, int chunk, int* sched,
                                          cudaStream_t st) {
    if (a.g.paper)
        return canon_smem_records(a.g) ? launch_persistent<true, true>(a, warps_per_cta, chunk, sched, st)
                                       : launch_persistent<false, true>(a, warps_per_cta, chunk, sched, st);
    return canon_smem_records(a.g) ? launch_persistent<true, false>(a, warps_per_cta, chunk, sched, st)
                                   : launch_persistent<false, false>(a, warps_per_cta, chunk, sched, st);
}

}  // namespace crbm
