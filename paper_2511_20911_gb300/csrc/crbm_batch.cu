// Batched sweep: several contexts (mixed lattice sizes, filter lists and
// tempering ladders) in one kernel launch.  Each CTA takes one (context,
// word) item of the work list and runs the canonical or the generic
// SMEM-resident body for it; the contexts' descriptors travel by value in
// the kernel parameters.  Sweep and measurement counters come from a device
// clock per context, advanced by a one-thread epilogue, so the pair of
// launches can be captured once in a CUDA graph and replayed.
#include "crbm_canon_body.cuh"
#include "crbm_generic_body.cuh"

namespace crbm {
namespace {

__global__ void __launch_bounds__(512, 1) k_sweep_batch(const __grid_constant__ BatchArgs b) {
    const int2 item = b.items[blockIdx.x];
    const SweepArgs& a = b.d[item.x];
    if (a.g.canonical)
        canon::sweep_canon_body<false>(a, item.y, static_cast<uint32_t>(a.clock[0]), a.n_sweeps, a.clock[1]);
    else
        generic::sweep_generic_body(a, item.y);
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

cudaError_t launch_sweep_batch(const BatchArgs& b, int n_items, int threads, size_t smem, cudaStream_t st) {
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_sweep_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_sweep_batch<<<n_items, threads, smem, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_batch_advance(int64_t* clocks, const int* every, int n_ctx, int64_t n_sweeps, cudaStream_t st) {
    k_batch_advance<<<1, 32, 0, st>>>(clocks, every, n_ctx, n_sweeps);
    return cudaGetLastError();
}

}  // namespace crbm
