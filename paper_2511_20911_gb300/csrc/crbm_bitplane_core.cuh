// Word-parallel pieces of the bit-plane sweeps (CRBM_RNG_BITPLANE), shared by
// the SMEM sweep (crbm_bitplane.cu) and the streamed one (crbm_stream.cu).
// Every 32-bit value holds one bit per chain of a 32-chain word.
#pragma once

#include "crbm_device.cuh"

namespace crbm {
namespace bp {

using dev::U4;

// One plane of the comparison u < t, most significant bit first: lt collects
// the chains found below, eq the chains whose uniform and threshold agree on
// every plane so far (still open).  U, T: the plane of the uniforms and of
// the thresholds.
__device__ __forceinline__ void plane_step(uint32_t U, uint32_t T, uint32_t& lt, uint32_t& eq) {
    lt |= eq & T & ~U;
    eq &= ~(T ^ U);
}

// The four planes of one Philox call of a hidden node: P, M select the chains
// with m = 2 and m = -2, tb points at the call's first plane of the m = -2 row
// (m = 2 row 64 words further); Z0 = the chains with m = 0 on the first call
// (their threshold 2^31 has only its top plane set), 0 on later calls.
__device__ __forceinline__ void hidden_planes(const U4& q, const uint32_t* tb, uint32_t P, uint32_t M, uint32_t Z0,
                                              uint32_t& lt, uint32_t& eq) {
    plane_step(q.x, (P & tb[64]) | (M & tb[0]) | Z0, lt, eq);
    plane_step(q.y, (P & tb[65]) | (M & tb[1]), lt, eq);
    plane_step(q.z, (P & tb[66]) | (M & tb[2]), lt, eq);
    plane_step(q.w, (P & tb[67]) | (M & tb[3]), lt, eq);
}

// Count of set bits among h0..h3 per chain, c0 + 2 c1 + 4 c2, bit-sliced.
struct Count4 {
    uint32_t c0, c1, c2;
};
__device__ __forceinline__ Count4 count4(uint32_t h0, uint32_t h1, uint32_t h2, uint32_t h3) {
    const uint32_t s01 = h0 ^ h1, a01 = h0 & h1, s23 = h2 ^ h3, a23 = h2 & h3;
    const uint32_t cy = s01 & s23;
    return {s01 ^ s23, a01 ^ a23 ^ cy, (a01 & a23) | (cy & (a01 | a23))};
}

// The threshold plane of a spin: tb points at the plane in the [count][J' bit]
// rows (32 words apart); hp is the J' bit, n the count of the J incidences.
// A mux tree: the J' bit, then count bits 0, 1, 2.
__device__ __forceinline__ uint32_t visible_plane(const uint32_t* tb, uint32_t hp, const Count4& n) {
    auto sel = [&](int c) { return (hp & tb[(2 * c + 1) * 32]) | (~hp & tb[2 * c * 32]); };
    const uint32_t m01 = (n.c0 & sel(1)) | (~n.c0 & sel(0)), m23 = (n.c0 & sel(3)) | (~n.c0 & sel(2));
    return (n.c2 & sel(4)) | (~n.c2 & ((n.c1 & m23) | (~n.c1 & m01)));
}

// 32 x 32 bit transpose across a warp: lane c returns the word whose bit l is
// bit c of lane l's x (block swaps of 16, 8, 4, 2 and 1 rows and columns).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
    constexpr uint32_t kLow[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int j = 16 >> i;
        const uint32_t m = kLow[i];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y << j) & ~m));
    }
    return x;
}

// Appends the lanes whose comparison is still open (open != 0: its
// undecided chains) to a straggler list of (node, open chains) pairs, with
// one atomic per warp; returns true on the lanes whose node went to the list
// (false where the list is full: that lane finishes its node itself).
__device__ __forceinline__ bool push_straggler(uint32_t node, uint32_t open, int* count, uint2* list, int cap,
                                               int lane) {
    const uint32_t bal = __ballot_sync(0xffffffffu, open != 0u);
    if (bal == 0u) return false;
    int first = 0;
    if (lane == 0) first = atomicAdd(count, __popc(bal));
    first = __shfl_sync(0xffffffffu, first, 0);
    const int slot = first + __popc(bal & ((1u << lane) - 1u));
    if (open == 0u || slot >= cap) return false;
    list[slot] = make_uint2(node, open);
    return true;
}

}  // namespace bp
}  // namespace crbm
