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

// Four consecutive threshold planes of one row: the planes of one Philox
// call, read with one 16-byte shared-memory load (rows start on a 16-byte
// boundary and calls on a multiple of four planes).
__device__ __forceinline__ uint4 planes4(const uint32_t* p) { return *reinterpret_cast<const uint4*>(p); }

// The four planes of one Philox call of a hidden node: P, M select the chains
// with m = 2 and m = -2, tb points at the call's first plane of the m = -2 row
// (m = 2 row 64 words further); Z0 = the chains with m = 0 on the first call
// (their threshold 2^31 has only its top plane set), 0 on later calls.
__device__ __forceinline__ void hidden_planes(const U4& q, const uint32_t* tb, uint32_t P, uint32_t M, uint32_t Z0,
                                              uint32_t& lt, uint32_t& eq) {
    const uint4 tm = planes4(tb), tp = planes4(tb + 64);
    plane_step(q.x, (P & tp.x) | (M & tm.x) | Z0, lt, eq);
    plane_step(q.y, (P & tp.y) | (M & tm.y), lt, eq);
    plane_step(q.z, (P & tp.z) | (M & tm.z), lt, eq);
    plane_step(q.w, (P & tp.w) | (M & tm.w), lt, eq);
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

// The four threshold planes of one Philox call of a spin: tb points at the
// call's first plane in the [count][J' bit] rows (32 words apart); hp is the
// J' bit, n the count of the J incidences.  A mux tree per plane: the J' bit,
// then count bits 0, 1, 2 (a count of 4 has bits 0 and 1 clear).
__device__ __forceinline__ uint4 visible_planes(const uint32_t* tb, uint32_t hp, const Count4& n) {
    auto mux = [](uint32_t s, const uint4& x1, const uint4& x0) {
        return make_uint4((s & x1.x) | (~s & x0.x), (s & x1.y) | (~s & x0.y), (s & x1.z) | (~s & x0.z),
                          (s & x1.w) | (~s & x0.w));
    };
    auto sel = [&](int c) { return mux(hp, planes4(tb + (2 * c + 1) * 32), planes4(tb + 2 * c * 32)); };
    const uint4 m01 = mux(n.c0, sel(1), sel(0));
    const uint4 m23 = mux(n.c0, sel(3), sel(2));
    return mux(n.c2, sel(4), mux(n.c1, m23, m01));
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
