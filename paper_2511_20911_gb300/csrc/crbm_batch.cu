// Batched sweep: several contexts (mixed lattice sizes, filter lists,
// precisions, uniform modes and tempering ladders) in one kernel launch.
// Each CTA (or cluster of CTAs) takes one (context, word) item of the work
// list and runs the canonical (exact or paper precision), bit-plane or
// generic SMEM-resident body for it; the contexts' descriptors travel by
// value in the kernel parameters.  Sweep and measurement counters come from a device
// clock per context, advanced by a one-thread epilogue, so the pair of
// launches can be captured once in a CUDA graph and replayed.
#include "crbm_bitplane_body.cuh"
#include "crbm_canon_body.cuh"
#include "crbm_generic_body.cuh"

namespace crbm {
namespace {

namespace cg = cooperative_groups;

// One CTA per task (descriptor, word, band, bands).  kCluster: the launch
// has thread-block clusters.  A word split into bands > 1 occupies
// consecutive ranks of a cluster that holds only words of its context (and
// padding ranks of that context, band >= bands), all synchronising with
// cluster barriers; every other cluster holds whole words, one per CTA,
// which synchronise within their CTA only; tasks with descriptor -1 return
// at once.  kModes: the member kinds besides exact lane-uniform and generic
// ones that the batch holds (kBatchPaper, kBatchBitplane), so that a batch
// without them runs code that carries neither body.
template <bool kCluster, int kModes>
__global__ void __launch_bounds__(CRBM_SWEEP_MAX_THREADS, CRBM_SWEEP_MAX_THREADS <= 512 ? 2 : 1) k_sweep_batch(const __grid_constant__ BatchArgs b) {
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

// The instantiation for a cluster flag and a set of member kinds.
using BatchKernel = void (*)(const BatchArgs);
template <bool kCluster>
BatchKernel batch_kernel(int modes) {
    switch (modes & (kBatchPaper | kBatchBitplane)) {
        case kBatchPaper: return k_sweep_batch<kCluster, kBatchPaper>;
        case kBatchBitplane: return k_sweep_batch<kCluster, kBatchBitplane>;
        case kBatchPaper | kBatchBitplane: return k_sweep_batch<kCluster, kBatchPaper | kBatchBitplane>;
        default: return k_sweep_batch<kCluster, 0>;
    }
}

// clocks[c] = {sweep, measurements}; every[c] = measure_every of context c.
__global__ void k_batch_advance(int64_t* clocks, const int* every, int n_ctx, int64_t n) {
    const int c = threadIdx.x;
    if (c >= n_ctx) return;
    const int64_t t0 = clocks[2 * c], t1 = t0 + n;
    const int64_t k = every[c];
    if (k > 0) clocks[2 * c + 1] += t1 / k - t0 / k;
    clocks[2 * c] = t1;
}

}  // namespace

cudaError_t launch_sweep_batch(const BatchArgs& b, int n_tasks, int cluster, int threads, size_t smem, int modes,
                               cudaStream_t st) {
    const BatchKernel kernel = cluster <= 1 ? batch_kernel<false>(modes) : batch_kernel<true>(modes);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    if (cluster <= 1) {
        kernel<<<n_tasks, threads, smem, st>>>(b);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned int>(n_tasks));
    cfg.blockDim = dim3(static_cast<unsigned int>(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned int>(cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, b);
}

int batch_max_active_clusters(int cluster, int threads, size_t smem, int modes) {
    const BatchKernel kernel = batch_kernel<true>(modes);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
            cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned int>(cluster));
    cfg.blockDim = dim3(static_cast<unsigned int>(threads));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned int>(cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_batch_advance(int64_t* clocks, const int* every, int n_ctx, int64_t n_sweeps, cudaStream_t st) {
    k_batch_advance<<<1, 32, 0, st>>>(clocks, every, n_ctx, n_sweeps);
    return cudaGetLastError();
}

}  // namespace crbm
