// The batched sweep kernel for CTAs of at most 512 threads (a thread may
// take 128 registers), in its own translation unit so that it compiles in
// parallel with crbm_batch.cu.
#include "crbm_batch_kernel.cuh"

namespace crbm {

BatchKernel batch_kernel_small(bool cluster, int modes) {
    return cluster ? batch_kernel_for<true, 512>(modes) : batch_kernel_for<false, 512>(modes);
}

}  // namespace crbm
