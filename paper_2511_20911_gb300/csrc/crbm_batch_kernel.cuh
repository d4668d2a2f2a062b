// The batched sweep kernel (see crbm_batch.cu), instantiated for two CTA
// size limits: up to CRBM_SWEEP_MAX_THREADS threads (crbm_batch.cu; 64
// registers a thread), and up to 512 (crbm_batch_small.cu), where a thread
// may take 128 registers and keeps the bodies' state in registers instead of
// spilling it.  Batches with large members hold one CTA per SM either way
// (their shared memory); the batch autotuner weighs the two against each
// other through the CTA sizes it times.
#pragma once

#include "crbm_bitplane_body.cuh"
#include "crbm_canon_body.cuh"
#include "crbm_generic_body.cuh"

namespace crbm {
namespace {

namespace cg = cooperative_groups;

// One CTA per task (descriptor, word, band, bands), of at most kMaxThreads
// threads.  kCluster: the launch
// has thread-block clusters.  A word split into bands > 1 occupies
// consecutive ranks of a cluster that holds only words of its context (and
// padding ranks of that context, band >= bands), all synchronising with
// cluster barriers; every other cluster holds whole words, one per CTA,
// which synchronise within their CTA only; tasks with descriptor -1 return
// at once.  kModes: the member kinds besides exact lane-uniform and generic
// ones that the batch holds (kBatchPaper, kBatchBitplane), so that a batch
// without them runs code that carries neither body.
template <bool kCluster, int kModes, int kMaxThreads>
__global__ void __launch_bounds__(kMaxThreads, 1) k_sweep_batch(const __grid_constant__ BatchArgs b) {
    const int4 task = b.items[blockIdx.x];
    if (task.x < 0) return;
    const SweepArgs& a = b.d[task.x];
    const uint32_t t0 = static_cast<uint32_t>(a.clock[0]);
    if (!a.g.canonical) {
        if ((kModes & kBatchPaper) && a.g.paper)
            generic::sweep_generic_body<true>(a, task.y);
        else
            generic::sweep_generic_body<false>(a, task.y);
    } else if ((kModes & kBatchBitplane) && a.g.bitplane) {  // whole words; node records from global memory
        const uint32_t* hrec = reinterpret_cast<const uint32_t*>(a.crec);
        const uint32_t* vrec = hrec + static_cast<size_t>(a.g.n_cells) * bp::kBpNodes;
        if (a.swap_every > 0)
            bp::sweep_bitplane_body<true>(a, hrec, vrec, task.y, t0, a.n_sweeps, a.clock[1]);
        else
            bp::sweep_bitplane_body<false>(a, hrec, vrec, task.y, t0, a.n_sweeps, a.clock[1]);
    } else if ((kModes & kBatchPaper) && a.g.paper) {  // whole words
        if (b.smem_rec)
            canon::sweep_canon_body<true, false, true>(a, task.y, t0, a.n_sweeps, a.clock[1]);
        else
            canon::sweep_canon_body<false, false, true>(a, task.y, t0, a.n_sweeps, a.clock[1]);
    } else if (kCluster && task.w > 1) {
        const int rank = static_cast<int>(cg::this_cluster().block_rank());
        const int rank0 = task.z < task.w ? rank - task.z : 0;
        if (b.smem_rec)
            canon::sweep_canon_body<true, true>(a, task.y, t0, a.n_sweeps, a.clock[1], task.z, rank0);
        else
            canon::sweep_canon_body<false, true>(a, task.y, t0, a.n_sweeps, a.clock[1], task.z, rank0);
    } else if (b.smem_rec) {
        canon::sweep_canon_body<true, false>(a, task.y, t0, a.n_sweeps, a.clock[1]);
    } else {
        canon::sweep_canon_body<false, false>(a, task.y, t0, a.n_sweeps, a.clock[1]);
    }
}

// The instantiation for a cluster flag, a set of member kinds and a CTA size limit.
using BatchKernel = void (*)(const BatchArgs);
template <bool kCluster, int kMaxThreads>
BatchKernel batch_kernel_for(int modes) {
    switch (modes & (kBatchPaper | kBatchBitplane)) {
        case kBatchPaper: return k_sweep_batch<kCluster, kBatchPaper, kMaxThreads>;
        case kBatchBitplane: return k_sweep_batch<kCluster, kBatchBitplane, kMaxThreads>;
        case kBatchPaper | kBatchBitplane: return k_sweep_batch<kCluster, kBatchPaper | kBatchBitplane, kMaxThreads>;
        default: return k_sweep_batch<kCluster, 0, kMaxThreads>;
    }
}

}  // namespace
}  // namespace crbm
