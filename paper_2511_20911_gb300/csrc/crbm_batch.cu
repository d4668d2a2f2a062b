// Batched sweep: several contexts (mixed lattice sizes, filter lists,
// precisions, uniform modes and tempering ladders) in one kernel launch.
// Each CTA (or cluster of CTAs) takes one (context, word) item of the work
// list and runs the canonical (exact or paper precision), bit-plane or
// generic SMEM-resident body for it; the contexts' descriptors travel by
// value in the kernel parameters.  Sweep and measurement counters come from a device
// clock per context, advanced by a one-thread epilogue, so the pair of
// launches can be captured once in a CUDA graph and replayed.
#include "crbm_batch_kernel.cuh"

namespace crbm {

// CTAs of up to 512 threads: the instantiations of crbm_batch_small.cu.
BatchKernel batch_kernel_small(bool cluster, int modes);

namespace {

// The kernel for a launch: the 512-thread instantiation for CTAs that fit it.
BatchKernel batch_kernel(bool cluster, int modes, int threads) {
    if (threads <= 512) return batch_kernel_small(cluster, modes);
    return cluster ? batch_kernel_for<true, CRBM_SWEEP_MAX_THREADS>(modes)
                   : batch_kernel_for<false, CRBM_SWEEP_MAX_THREADS>(modes);
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
    const BatchKernel kernel = batch_kernel(cluster > 1, modes, threads);
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
    const BatchKernel kernel = batch_kernel(true, modes, threads);
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
