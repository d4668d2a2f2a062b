// Bit-plane sweep (CRBM_RNG_BITPLANE), ten SS filters on an even periodic
// lattice, SMEM layout.  A persistent CTA claims one packed word (32 chains)
// at a time, for a chunk of sweeps, and works on it word-parallel: a thread takes one node (hidden unit or spin) for all 32
// chains at once, with the chains in the bits of every 32-bit value.
//
// A node's 32 uniforms are the bit-transpose of plane words drawn from
// Philox((cell, sweep, word, kTagBitplane + 8 node + j)), four planes per
// call, most significant plane first.  The thresholds are held the same way
// (per word, one bit-plane word per configuration and plane), so the 32
// comparisons u_l < t_l run as one word-parallel comparison, most significant
// bit first: a chain is decided at the first plane where its uniform and
// threshold bits differ (below when the threshold bit is the 1).  Every node
// draws two calls (eight planes); the nodes with chains still open after them
// (about 12 %) go to a straggler list, which the CTA's warps then take 32 at a
// time, drawing further calls while any of a warp's stragglers is open.  The
// result equals the full 32-bit comparison, bit for bit, whichever call a
// node stops at.
//
// Hidden unit k of a cell: its endpoints e1, e2 (spin words; e2 flipped on
// the chains whose class coupling is negative) select the threshold of m = e1
// + s e2 in {-2, 0, 2} per chain.  Spin x: its four J incidences (flipped
// where the spin is a second endpoint of a negative coupling) are counted in
// bit-sliced form (three count bits), its J' incidence gives one bit, and
// these select one of the 5 x 2 visible thresholds per chain.
#include <algorithm>

#include "crbm_bitplane_body.cuh"

namespace crbm {
namespace {

using namespace dev;
using namespace bp;

constexpr int kBpMaxThreads = CRBM_SWEEP_MAX_THREADS;  // largest CTA the launch takes

// Persistent grid over (word, chunk of sweeps) items (claim_word): the node
// records are staged once per CTA, then each claimed chunk runs the body.
// At most 56 registers a thread, so that three CTAs of 12 warps (the shape
// the L=18 grid tunes to) fit on an SM; CTAs of up to kBpMaxThreads threads.
template <bool kSmemRec, bool kSwap>
__global__ void __maxnreg__(56) k_sweep_bitplane(const SweepArgs a, int chunk, int* state) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_word, s_chunk;
    const Geometry& g = a.g;
    const int lane = threadIdx.x & 31;
    const int nh = g.n_cells * kBpNodes;
    const uint32_t* rec = reinterpret_cast<const uint32_t*>(a.crec);
    if (kSmemRec) {
        uint32_t* s_rec = smem + kBpSmemV + g.N + bp_hid_words(g) + bp_strag_words(g);  // N: a multiple of 4
        for (int x = threadIdx.x; x < static_cast<int>(bp_rec_words(g) / 4); x += blockDim.x)
            reinterpret_cast<uint4*>(s_rec)[x] = __ldg(a.crec + x);
        rec = s_rec;
    }
    const int n_chunks = (a.n_sweeps + chunk - 1) / chunk;
    const int nw = a.n_words;
    const int K = a.measure_every;
    const unsigned int start = (blockIdx.x * 97u) % static_cast<unsigned int>(nw);
    for (;;) {
        if (threadIdx.x < 32) {
            int word, c;
            claim_word(state, nw, n_chunks, start, lane, word, c);
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
        sweep_bitplane_body<kSwap>(a, rec, rec + nh, word, t0, n, meas0);
        __syncthreads();  // every thread's state stores are issued
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(state + word, 2 * (c + 1));
        }
    }
}

}  // namespace

size_t smem_bytes_bitplane(const Geometry& g, bool with_records) {
    return sizeof(uint32_t) * (kBpSmemV + static_cast<size_t>(g.N) + bp_hid_words(g) + bp_strag_words(g) +
                               (with_records ? bp_rec_words(g) : 0));
}

cudaError_t launch_sweep_bitplane(const SweepArgs& a, int warps_per_cta, int chunk, int* sched, cudaStream_t st) {
    const int warps = std::max(1, std::min(kBpMaxThreads / 32, warps_per_cta));
    const bool staged = smem_bytes_bitplane(a.g, true) <= 227 * 1024;
    const size_t smem = smem_bytes_bitplane(a.g, staged);
    const bool swap = a.swap_every > 0;  // replica exchange compiled in only where used
    auto kernel = staged ? (swap ? k_sweep_bitplane<true, true> : k_sweep_bitplane<true, false>)
                         : (swap ? k_sweep_bitplane<false, true> : k_sweep_bitplane<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    int per_sm = 0, dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * warps, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int n_items = ((a.n_sweeps + chunk - 1) / chunk) * a.n_words;
    const int grid = std::min(std::min(n_items, a.n_words), per_sm * sms);
    e = cudaMemsetAsync(sched, 0, sizeof(int) * (4 + static_cast<size_t>(a.n_words)), st);
    if (e != cudaSuccess) return e;
    kernel<<<grid, 32 * warps, smem, st>>>(a, chunk, sched);
    return cudaGetLastError();
}

}  // namespace crbm
