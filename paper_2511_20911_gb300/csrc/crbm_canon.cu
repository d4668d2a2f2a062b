// SMEM-resident sweep, canonical SS fast path: one CTA per packed word (32
// chains) holding the whole even, periodic lattice, its hidden layer and the
// lane-expanded tables in shared memory, all n_sweeps sweeps on device.  The
// per-cell cores are in crbm_canon_core.cuh.
#include "crbm_canon_body.cuh"

#ifndef CRBM_SWEEP_MIN_BLOCKS
#define CRBM_SWEEP_MIN_BLOCKS 2
#endif

namespace crbm {
namespace {

using namespace dev;
using namespace canon;

__global__ void __launch_bounds__(512, CRBM_SWEEP_MIN_BLOCKS) k_sweep_canon(const SweepArgs a) {
    sweep_canon_body(a, blockIdx.x);
}

}  // namespace

size_t smem_bytes_canon(const Geometry& g) {
    return sizeof(uint32_t) * (static_cast<size_t>(kCanonTab) + g.N + static_cast<size_t>(g.n_cells) * 32 +
                               96 + 33 + 32 + 64);
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
