// SMEM-resident sweep, canonical SS fast path: a CTA holds one packed word
// (32 chains) -- the whole even, periodic lattice, its hidden layer and the
// lane-expanded tables -- in shared memory and runs a chunk of sweeps on it.
// The sweep body is in crbm_canon_body.cuh, the per-cell cores in
// crbm_canon_core.cuh.
#include <algorithm>

#include "crbm_canon_body.cuh"

#ifndef CRBM_SWEEP_MIN_BLOCKS
#define CRBM_SWEEP_MIN_BLOCKS 2
#endif

namespace crbm {
namespace {

using namespace dev;
using namespace canon;

// Persistent form: a grid that fits on the GPU at once takes work items
// (word, chunk of `chunk` sweeps) in ticket order from a global counter.
// Chunk c of a word waits until chunk c-1 of that word is done (its ticket
// is n_words lower, held by a resident CTA, so the wait ends); the wait is
// bounded and, if it gives up, sets the error word and the CTA stops.  Every
// SM stays busy until the last chunks, whatever the number of words.
template <bool kSmemRec>
__global__ void __launch_bounds__(CRBM_SWEEP_MAX_THREADS, CRBM_SWEEP_MIN_BLOCKS)
    k_sweep_canon_persistent(const SweepArgs a, int chunk, int* counter, int* done, int* err) {
    __shared__ int s_item, s_ok;
    const int n_chunks = (a.n_sweeps + chunk - 1) / chunk;
    const int n_items = n_chunks * a.n_words;
    const int K = a.measure_every;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(counter, 1);
            s_ok = 1;
            const int item = s_item;
            if (item < n_items) {
                const int word = item % a.n_words, c = item / a.n_words;
                unsigned int spins = 0;
                while (ld_acquire(done + word) < c) {
                    if (++spins > (1u << 26)) {  // about 7 s: the predecessor never finished
                        atomicExch(err, 1);
                        s_ok = 0;
                        break;
                    }
                    __nanosleep(100);
                }
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item >= n_items || !s_ok) break;
        const int word = item % a.n_words, c = item / a.n_words;
        const uint32_t t0 = a.t0 + static_cast<uint32_t>(c * chunk);
        const int n = min(chunk, a.n_sweeps - c * chunk);
        const int64_t meas0 =
            K > 0 ? a.meas0 + static_cast<int64_t>(t0 / K) - static_cast<int64_t>(a.t0 / K) : a.meas0;
        sweep_canon_body<kSmemRec>(a, word, t0, n, meas0);
        __syncthreads();  // every thread's state stores are issued
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(done + word, c + 1);
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

size_t smem_bytes_canon(const Geometry& g) {
    return sizeof(uint32_t) * (static_cast<size_t>(kAccWords) + kCanonTab + g.N + static_cast<size_t>(g.n_cells) * 32 +
                               96 + 33 + 32 + 64);
}

namespace {
template <bool kSmemRec>
cudaError_t launch_persistent(const SweepArgs& a, int warps_per_cta, int chunk, int* sched, int* err,
                              cudaStream_t st) {
    const size_t smem = smem_bytes_canon_launch(a.g);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_sweep_canon_persistent<kSmemRec>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_canon_persistent<kSmemRec>,
                                                                  warps_per_cta * 32, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int n_items = ((a.n_sweeps + chunk - 1) / chunk) * a.n_words;
    const int grid = std::min(n_items, per_sm * sms);  // all CTAs resident: the waits always end
    e = cudaMemsetAsync(sched, 0, sizeof(int) * (1 + static_cast<size_t>(a.n_words)), st);
    if (e != cudaSuccess) return e;
    k_sweep_canon_persistent<kSmemRec><<<grid, warps_per_cta * 32, smem, st>>>(a, chunk, sched, sched + 1, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_canon_persistent(const SweepArgs& a, int warps_per_cta, int chunk, int* sched,
                                          int* err, cudaStream_t st) {
    return canon_smem_records(a.g) ? launch_persistent<true>(a, warps_per_cta, chunk, sched, err, st)
                                   : launch_persistent<false>(a, warps_per_cta, chunk, sched, err, st);
}

}  // namespace crbm
