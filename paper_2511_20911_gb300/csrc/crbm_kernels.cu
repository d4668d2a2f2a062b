// CUDA kernels of the CRBM block-Gibbs sampler (sm_103a): the generic
// SMEM-resident sweep (any filter list, odd L, open boundaries), the initial
// spins, packing/unpacking and the Philox check.  The canonical SS fast path
// lives in crbm_canon.cu.
//
// Work mapping: 32 chains share one packed 32-bit word per site (bit l =
// chain 32w + l); a warp works on one word, lane l owning chain 32w + l.  The
// packed words are warp-uniform, so every shared-memory read of the lattice is
// a broadcast, and each lane only extracts its own bit, draws its own Philox
// words and compares against its own threshold column; __ballot_sync packs
// the 32 decisions back into one word.  Everything is integer arithmetic.
#include "crbm_generic_body.cuh"

namespace crbm {
namespace {

using namespace dev;

template <bool kPaper>
__global__ void __launch_bounds__(512, 1) k_sweep_generic(const SweepArgs a) {
    generic::sweep_generic_body<kPaper>(a, blockIdx.x);
}

// Initial spins: site (R, C) of chain c is +1 iff word 2(R&1)+(C&1) of
// Philox((cell, 0, c, tag 5)) < 2^31.  One warp per (word, site).
__global__ void k_init(const Geometry g, uint32_t* v, int n_words, uint32_t k0, uint32_t k1) {
    const int lane = threadIdx.x & 31;
    const long long nw = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long x = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         x < static_cast<long long>(n_words) * g.N; x += nw) {
        const int word = static_cast<int>(x / g.N), s = static_cast<int>(x - static_cast<long long>(word) * g.N);
        const int R = s / g.Lc, C = s - (s / g.Lc) * g.Lc;
        const uint32_t cell = static_cast<uint32_t>((R >> 1) * g.Wc + (C >> 1));
        const U4 q = philox(cell, 0u, static_cast<uint32_t>(word) * 32u + lane, kTagInit, k0, k1);
        const uint32_t b = __ballot_sync(0xffffffffu, pick(q, 2 * (R & 1) + (C & 1)) < 0x80000000u);
        if (lane == 0) v[word_index(g.vil, word, g.N, s)] = b;
    }
}

__global__ void k_unpack(const Geometry g, const uint32_t* v, int8_t* out, int n_words) {
    const long long total = static_cast<long long>(n_words) * 32 * g.N;
    for (long long x = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long chain = x / g.N;
        const int s = static_cast<int>(x - chain * g.N);
        const uint32_t w = v[word_index(g.vil, static_cast<int>(chain >> 5), g.N, s)];
        out[x] = ((w >> (chain & 31)) & 1u) ? 1 : -1;
    }
}

__global__ void k_pack(const Geometry g, const int8_t* in, uint32_t* v, int n_words, const int* skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const long long nw = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    for (long long x = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         x < static_cast<long long>(n_words) * g.N; x += nw) {
        const long long word = x / g.N;
        const int s = static_cast<int>(x - word * g.N);
        const int8_t val = in[(word * 32 + lane) * g.N + s];
        const uint32_t b = __ballot_sync(0xffffffffu, val > 0);
        if (lane == 0) v[word_index(g.vil, static_cast<int>(word), g.N, s)] = b;
    }
}

// *flag = 1 when a byte of in[0 .. n) is neither +1 (0x01) nor -1 (0xFF):
// four bytes per load (the staging buffer is 256-byte aligned), a byte is
// valid iff its bits 1..7 all equal its bit 7 and its bit 0 is set.
__global__ void k_check_spins(const int8_t* in, size_t n, int* flag) {
    const size_t words = n / 4, stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    const uint32_t* w4 = reinterpret_cast<const uint32_t*>(in);
    bool bad = false;
    for (size_t x = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; x < words; x += stride) {
        const uint32_t w = w4[x];
        const uint32_t sign = (w >> 7) & 0x01010101u;      // bit 7 of each byte
        bad |= w != ((sign * 0xFEu) | 0x01010101u);        // 0xFF where the sign is set, else 0x01
    }
    for (size_t x = 4 * words + blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; x < n; x += stride)
        bad |= in[x] != 1 && in[x] != -1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

__global__ void k_philox(const uint32_t* in, uint32_t* out, int n) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint32_t* a = in + 6 * static_cast<size_t>(x);
    const U4 q = philox(a[0], a[1], a[2], a[3], a[4], a[5]);
    uint32_t* o = out + 4 * static_cast<size_t>(x);
    o[0] = q.x;
    o[1] = q.y;
    o[2] = q.z;
    o[3] = q.w;
}

// Philox throughput probe: thread t runs `calls` Philox-4x32-10 calls on the
// counters (i, t, i ^ t, 0x9E3779B9), i = 0 .. calls - 1, and stores the XOR
// of all their output words.  Every round's two wide products depend on i,
// so none can leave the loop: 20 32x32->64 products per call.
__global__ void k_philox_stream(uint32_t* sink, int calls, uint32_t k0, uint32_t k1) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0u;
#pragma unroll 2
    for (int i = 0; i < calls; ++i) {
        const uint32_t c = static_cast<uint32_t>(i);
        const U4 q = philox(c, t, c ^ t, 0x9E3779B9u, k0, k1);
        acc ^= q.x ^ q.y ^ q.z ^ q.w;
    }
    sink[t] = acc;
}

}  // namespace

cudaError_t launch_philox_stream(uint32_t* sink, int n_blocks, int threads, int calls, uint32_t k0,
                                 uint32_t k1, cudaStream_t st) {
    k_philox_stream<<<n_blocks, threads, 0, st>>>(sink, calls, k0, k1);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* in, uint32_t* out, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_philox<<<(n + 255) / 256, 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

size_t smem_bytes_generic(const Geometry& g) { return sizeof(uint32_t) * generic_smem(g).total; }

cudaError_t launch_init(const Geometry& g, uint32_t* v, int n_words, uint32_t key0, uint32_t key1,
                        cudaStream_t st) {
    const long long work = static_cast<long long>(n_words) * g.N;
    const int blocks = static_cast<int>((work + 7) / 8 < 152 * 64 ? (work + 7) / 8 : 152 * 64);
    k_init<<<blocks, 256, 0, st>>>(g, v, n_words, key0, key1);
    return cudaGetLastError();
}

cudaError_t launch_sweep_generic(const SweepArgs& a, int warps_per_cta, cudaStream_t st) {
    const size_t smem = smem_bytes_generic(a.g);
    auto kernel = a.g.paper ? k_sweep_generic<true> : k_sweep_generic<false>;
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    kernel<<<a.n_words, warps_per_cta * 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geometry& g, const uint32_t* v, int8_t* out, int n_words,
                          cudaStream_t st) {
    const long long total = static_cast<long long>(n_words) * 32 * g.N;
    const int blocks = static_cast<int>((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    k_unpack<<<blocks, 256, 0, st>>>(g, v, out, n_words);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Geometry& g, const int8_t* in, uint32_t* v, int n_words, const int* skip,
                        cudaStream_t st) {
    const long long work = static_cast<long long>(n_words) * g.N;
    const int blocks = static_cast<int>((work + 7) / 8 < 152 * 64 ? (work + 7) / 8 : 152 * 64);
    k_pack<<<blocks, 256, 0, st>>>(g, in, v, n_words, skip);
    return cudaGetLastError();
}

cudaError_t launch_check_spins(const int8_t* in, size_t n, int* flag, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const size_t words = n / 4;  // 4 spins per 32-bit load, the tail bytes one at a time
    const size_t want = (words + 255) / 256 + 1;
    const int blocks = static_cast<int>(want < 152 * 16 ? want : 152 * 16);
    k_check_spins<<<blocks, 256, 0, st>>>(in, n, flag);
    return cudaGetLastError();
}

}  // namespace crbm
