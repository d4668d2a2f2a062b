// Per-cell cores of the canonical SS fast path (the ten filters of Fig. 1 on
// an even, periodic lattice), shared by the SMEM-resident sweep
// (crbm_canon_body.cuh), the streamed two-phase sweep (crbm_stream.cu) and
// the batched launch.
//
// Mapping: warp = 32 chains of one packed word, lane = chain.
//
// Hidden half-step (Eq. 9): each packed spin word of the 3x3 window is masked
// to the lane's bit and rotated (funnel shift) into address bit 7 (first
// endpoint) or 8 (second endpoint) of the lane-expanded hidden table
// [cls][e1 + 2 e2][lane]; one OR with the lane's column offset makes the
// address.  The ten decisions are not packed across lanes: each lane ORs
// them into ONE per-lane word W whose bits are already the slots of the
// visible-table indices that use them (layout below), for the cell's own four
// spins and for the spins of the cell below and the cell to the right.
//
// Visible half-step (Eq. 10): C = (W_own & kOwn) | (W_up & kDown) |
// (W_left & kRight) holds the 5-bit filter index of spin (r, c) at bits
// 7 + 5 (2r + c) .. +4; a shift and a mask place it in address bits 7..11 of
// the visible table [spin position][idx][lane].  The host builds both tables
// so that they absorb the coefficient signs s and the field sums, so a node
// costs one address merge, one shared load, one compare and one bit merge
// (hidden) or ballot (visible), plus its share of a Philox call.
#pragma once

#include "crbm_device.cuh"

namespace crbm {
namespace canon {

using namespace dev;

// Bit of W for each filter unit k (see the slot table kCanonSlot):
//   spin (0,0): b0 b4 b8 l.b1 u.b5 -> bits  7  8  9 10 11
//   spin (0,1): b0 b6 b1 u.b7 u.b9 -> bits 12 13 14 15 16
//   spin (1,0): b2 b4 b5 l.b3 l.b9 -> bits 17 18 19 20 21
//   spin (1,1): b2 b6 b8 b3 b7     -> bits 22 23 24 25 26
// A unit of the own cell sets its own-spin bits; b1, b3, b9 also set the bits
// the cell to the right reads, b5, b7, b9 those the cell below reads.
constexpr uint32_t kBit0 = (1u << 7) | (1u << 12);
constexpr uint32_t kBit1 = (1u << 14) | (1u << 10);  // own (0,1) slot 2; right's (0,0) slot 3
constexpr uint32_t kBit2 = (1u << 17) | (1u << 22);
constexpr uint32_t kBit3 = (1u << 25) | (1u << 20);  // own (1,1) slot 3; right's (1,0) slot 3
constexpr uint32_t kBit4 = (1u << 8) | (1u << 18);
constexpr uint32_t kBit5 = (1u << 19) | (1u << 11);  // own (1,0) slot 2; below's (0,0) slot 4
constexpr uint32_t kBit6 = (1u << 13) | (1u << 23);
constexpr uint32_t kBit7 = (1u << 26) | (1u << 15);  // own (1,1) slot 4; below's (0,1) slot 3
constexpr uint32_t kBit8 = (1u << 9) | (1u << 24);
constexpr uint32_t kBit9 = (1u << 16) | (1u << 21);  // below's (0,1) slot 4; right's (1,0) slot 4
constexpr uint32_t kDownBits = (1u << 11) | (1u << 15) | (1u << 16);
constexpr uint32_t kRightBits = (1u << 10) | (1u << 20) | (1u << 21);
constexpr uint32_t kOwnBits = ((1u << 27) - (1u << 7)) & ~kDownBits & ~kRightBits;

// w | K when q < t, as one compare and one predicated OR (the conditional
// expression form compiles to a compare, a select and an OR).
template <uint32_t K>
__device__ __forceinline__ uint32_t or_if_less(uint32_t w, uint32_t q, uint32_t t) {
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
        : "+r"(w)
        : "r"(q), "r"(t), "n"(K));
    return w;
}

// Byte-addressed 32-bit shared-memory load.
__device__ __forceinline__ uint32_t lds_at(const uint32_t* base, uint32_t byte_off) {
    return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(base) + byte_off);
}

struct LaneConst {
    uint32_t lm;      // 1 << lane
    uint32_t lb;      // 4 * column: the lane's column in a [.][32] table
    uint32_t rot[2];  // rotate-right amounts taking bit `lane` to bit 7 / 8
};

__device__ __forceinline__ LaneConst lane_const(int lane, int col) {
    LaneConst lc;
    lc.lm = 1u << lane;
    lc.lb = 4u * static_cast<uint32_t>(col);
    lc.rot[0] = static_cast<uint32_t>(lane - 7) & 31u;
    lc.rot[1] = static_cast<uint32_t>(lane - 8) & 31u;
    return lc;
}

// Shared-memory word at a byte offset from the start of dynamic shared
// memory (per-cell records hold such offsets).
__device__ __forceinline__ uint32_t lds_off(const char* sm, uint32_t off) {
    return *reinterpret_cast<const uint32_t*>(sm + off);
}
__device__ __forceinline__ void sts_off(char* sm, uint32_t off, uint32_t x) {
    *reinterpret_cast<uint32_t*>(sm + off) = x;
}

// Hidden half-step of one cell from its eight window words v_rc (row r,
// column c of the 3x3 window; (2,2) is not used), the cell's round-0 Philox
// word rcb = lo(M0 cell) and the round-1 call products of its three calls;
// returns the lane's word W.
__device__ __forceinline__ uint32_t hidden_core(uint32_t v00, uint32_t v01, uint32_t v02, uint32_t v10,
                                                uint32_t v11, uint32_t v12, uint32_t v20, uint32_t v21,
                                                const uint32_t* s_th, const Round1Sweep& r1, uint32_t Y,
                                                uint32_t rcb, const Round1Call& c0, const Round1Call& c1,
                                                const Round1Call& c2, const uint32_t (&rk)[20],
                                                const LaneConst& lc) {
    const uint32_t m00 = v00 & lc.lm, m01 = v01 & lc.lm, m02 = v02 & lc.lm, m10 = v10 & lc.lm;
    const uint32_t m11 = v11 & lc.lm, m12 = v12 & lc.lm, m20 = v20 & lc.lm, m21 = v21 & lc.lm;
    // first endpoints at bit 7
    const uint32_t a00 = rotr(m00, lc.rot[0]), a01 = rotr(m01, lc.rot[0]);
    const uint32_t a10 = rotr(m10, lc.rot[0]), a11 = rotr(m11, lc.rot[0]);
    const uint32_t a12 = rotr(m12, lc.rot[0]);
    // second endpoints at bit 8
    const uint32_t b01 = rotr(m01, lc.rot[1]), b02 = rotr(m02, lc.rot[1]);
    const uint32_t b10 = rotr(m10, lc.rot[1]), b11 = rotr(m11, lc.rot[1]);
    const uint32_t b12 = rotr(m12, lc.rot[1]), b20 = rotr(m20, lc.rot[1]);
    const uint32_t b21 = rotr(m21, lc.rot[1]);
    const Round2Cell r2 = round2_cell(r1.hik ^ rcb);  // shared by the cell's calls
    const U4 q0 = philox_from_call(Y, r1, r2, c0, rk);
    const U4 q1 = philox_from_call(Y, r1, r2, c1, rk);
    const U4 q2 = philox_from_call(Y, r1, r2, c2, rk);
    const uint32_t* thJ = s_th;
    const uint32_t* thP = s_th + 128;
    uint32_t w = 0u;
    // filters 0..7 (J) and 8..9 (J'): (first endpoint, second endpoint)
    w = or_if_less<kBit0>(w, q0.x, lds_at(thJ, a00 | b01 | lc.lb));
    w = or_if_less<kBit1>(w, q0.y, lds_at(thJ, a01 | b02 | lc.lb));
    w = or_if_less<kBit2>(w, q0.z, lds_at(thJ, a10 | b11 | lc.lb));
    w = or_if_less<kBit3>(w, q0.w, lds_at(thJ, a11 | b12 | lc.lb));
    w = or_if_less<kBit4>(w, q1.x, lds_at(thJ, a00 | b10 | lc.lb));
    w = or_if_less<kBit5>(w, q1.y, lds_at(thJ, a10 | b20 | lc.lb));
    w = or_if_less<kBit6>(w, q1.z, lds_at(thJ, a01 | b11 | lc.lb));
    w = or_if_less<kBit7>(w, q1.w, lds_at(thJ, a11 | b21 | lc.lb));
    w = or_if_less<kBit8>(w, q2.x, lds_at(thP, a00 | b11 | lc.lb));
    w = or_if_less<kBit9>(w, q2.y, lds_at(thP, a12 | b21 | lc.lb));
    return w;
}

// Hidden half-step of one cell.  Window rows at s_v + 0, vs, 2 vs; q0 =
// (rc.lo, Q0.h, Q0.l, Q1.h), q1 = (Q1.l, Q2.h, Q2.l, -): the cell's round-0
// word and round-1 call products (as in the per-cell records).  Returns the
// lane's word W.
__device__ __forceinline__ uint32_t hidden_cell(const uint32_t* s_v, int vs, const uint32_t* s_th,
                                                const Round1Sweep& rs, uint32_t Y, const uint4& q0,
                                                const uint4& q1, const uint32_t (&rk)[20], const LaneConst& lc) {
    return hidden_core(s_v[0], s_v[1], s_v[2], s_v[vs], s_v[vs + 1], s_v[vs + 2], s_v[2 * vs], s_v[2 * vs + 1],
                       s_th, rs, Y, q0.x, {q0.y, q0.z}, {q0.w, q1.x}, {q1.y, q1.z}, rk, lc);
}

// The (rc.lo, Q0.h, Q0.l, Q1.h), (Q1.l, Q2.h, Q2.l, 0) words of cell `cell`
// for hidden_cell, and (rc.lo, Qv.h, Qv.l, 0) for visible_cell.
__device__ __forceinline__ void hidden_call_words(uint32_t cell, const uint32_t (&rk)[20], uint4& q0, uint4& q1) {
    const Round0Cell rc = round0_cell(cell, rk[1]);
    const Round1Call c0 = round1_call(rc.a, rk), c1 = round1_call(rc.a ^ 1u, rk), c2 = round1_call(rc.a ^ 2u, rk);
    q0 = make_uint4(rc.b, c0.h, c0.l, c1.h);
    q1 = make_uint4(c1.l, c2.h, c2.l, 0u);
}
__device__ __forceinline__ uint4 visible_call_words(uint32_t cell, const uint32_t (&rk)[20]) {
    const Round0Cell rc = round0_cell(cell, rk[1]);
    const Round1Call cv = round1_call(rc.a ^ kTagVis, rk);
    return make_uint4(rc.b, cv.h, cv.l, 0u);
}

// Hidden half-step of one cell described by its records h0, h1, h2 and the
// first word h5 of its record 5 (layout in crbm_internal.h); returns the
// lane's word W.
__device__ __forceinline__ uint32_t hidden_cell_rec(const char* sm, const uint4& h0, const uint4& h1,
                                                    const uint4& h2, uint32_t h5, const uint32_t* s_th,
                                                    const Round1Sweep& rs, uint32_t Y, const uint32_t (&rk)[20],
                                                    const LaneConst& lc) {
    return hidden_core(lds_off(sm, h0.x), lds_off(sm, h0.x + 4u), lds_off(sm, h0.w), lds_off(sm, h0.y),
                       lds_off(sm, h0.y + 4u), lds_off(sm, h1.x), lds_off(sm, h0.z), lds_off(sm, h0.z + 4u),
                       s_th, rs, Y, h1.z, {h2.x, h2.y}, {h2.z, h2.w}, {h1.w, h5}, rk, lc);
}

// Visible half-step of one cell from the lanes' words of this cell (wo), the
// cell above (wu) and the cell to the left (wl), with the cell's round-0 word
// rcb = lo(M0 cell) and the round-1 product cv of its visible call; returns
// the four new spin words (0,0) (0,1) (1,0) (1,1) of the cell.
__device__ __forceinline__ U4 visible_core(uint32_t wo, uint32_t wu, uint32_t wl, const uint32_t* s_tv,
                                           const Round1Sweep& r1, uint32_t Y, uint32_t rcb,
                                           const Round1Call& cv, const uint32_t (&rk)[20], const LaneConst& lc) {
    const uint32_t c = (wo & kOwnBits) | (wu & kDownBits) | (wl & kRightBits);
    const U4 q = philox_from_call(Y, r1, round2_cell(r1.hik ^ rcb), cv, rk);
    const uint32_t f = 31u << 7;
    const uint32_t t00 = lds_at(s_tv, (c & f) | lc.lb);
    const uint32_t t01 = lds_at(s_tv + 1024, ((c >> 5) & f) | lc.lb);
    const uint32_t t10 = lds_at(s_tv + 2048, ((c >> 10) & f) | lc.lb);
    const uint32_t t11 = lds_at(s_tv + 3072, ((c >> 15) & f) | lc.lb);
    return {__ballot_sync(0xffffffffu, q.x < t00), __ballot_sync(0xffffffffu, q.y < t01),
            __ballot_sync(0xffffffffu, q.z < t10), __ballot_sync(0xffffffffu, q.w < t11)};
}

// Visible half-step of one cell with qv = visible_call_words(cell); the four
// new spin words go to out[0], out[1], out[row], out[row + 1].
__device__ __forceinline__ void visible_cell(uint32_t* out, int row, uint32_t wo, uint32_t wu,
                                             uint32_t wl, const uint32_t* s_tv, const Round1Sweep& rs,
                                             uint32_t Y, const uint4& qv, const uint32_t (&rk)[20],
                                             const LaneConst& lc) {
    const U4 o = visible_core(wo, wu, wl, s_tv, rs, Y, qv.x, {qv.y, qv.z}, rk, lc);
    out[0] = o.x;
    out[1] = o.y;
    out[row] = o.z;
    out[row + 1] = o.w;
}

// Visible half-step of one cell described by its records 3 and 4 (v0, v1); lane4 =
// 4 * lane (the lane's column of the hidden rows).  Stores the four new spin
// words and returns them.
__device__ __forceinline__ U4 visible_cell_rec(char* sm, const uint4& v0, const uint4& v1, uint32_t lane4,
                                               const uint32_t* s_tv, const Round1Sweep& rs, uint32_t Y,
                                               const uint32_t (&rk)[20], const LaneConst& lc) {
    const U4 o = visible_core(lds_off(sm, v0.z + lane4), lds_off(sm, v0.w + lane4), lds_off(sm, v1.x + lane4),
                              s_tv, rs, Y, v1.y, {v1.z, v1.w}, rk, lc);
    sts_off(sm, v0.x, o.x);
    sts_off(sm, v0.x + 4u, o.y);
    sts_off(sm, v0.y, o.z);
    sts_off(sm, v0.y + 4u, o.w);
    return o;
}

// Paper precision (CRBM_PRECISION_PAPER): every Philox word carries two
// 16-bit uniforms and a threshold holds its 16-bit value in the upper half,
// so a word's high-half uniform compares as the whole word and its low half
// after a shift by 16.  The hidden half-step of a cell draws two calls (tags
// 0 and 1): filter k takes half k&1 of word k>>1 of tag 0, filters 8 and 9
// the halves of word 0 of tag 1; words 1 and 2 of tag 1 carry the cell's
// four visible uniforms and are returned in `vis` for the visible half-step.
__device__ __forceinline__ uint32_t hidden_core_paper(uint32_t v00, uint32_t v01, uint32_t v02, uint32_t v10,
                                                      uint32_t v11, uint32_t v12, uint32_t v20, uint32_t v21,
                                                      const uint32_t* s_th, const Round1Sweep& r1, uint32_t Y,
                                                      uint32_t rcb, const Round1Call& c0, const Round1Call& c1,
                                                      const uint32_t (&rk)[20], const LaneConst& lc, uint2& vis) {
    const uint32_t m00 = v00 & lc.lm, m01 = v01 & lc.lm, m02 = v02 & lc.lm, m10 = v10 & lc.lm;
    const uint32_t m11 = v11 & lc.lm, m12 = v12 & lc.lm, m20 = v20 & lc.lm, m21 = v21 & lc.lm;
    const uint32_t a00 = rotr(m00, lc.rot[0]), a01 = rotr(m01, lc.rot[0]);
    const uint32_t a10 = rotr(m10, lc.rot[0]), a11 = rotr(m11, lc.rot[0]);
    const uint32_t a12 = rotr(m12, lc.rot[0]);
    const uint32_t b01 = rotr(m01, lc.rot[1]), b02 = rotr(m02, lc.rot[1]);
    const uint32_t b10 = rotr(m10, lc.rot[1]), b11 = rotr(m11, lc.rot[1]);
    const uint32_t b12 = rotr(m12, lc.rot[1]), b20 = rotr(m20, lc.rot[1]);
    const uint32_t b21 = rotr(m21, lc.rot[1]);
    const Round2Cell r2 = round2_cell(r1.hik ^ rcb);
    const U4 q0 = philox_from_call(Y, r1, r2, c0, rk);
    const U4 q1 = philox_from_call(Y, r1, r2, c1, rk);
    const uint32_t* thJ = s_th;
    const uint32_t* thP = s_th + 128;
    uint32_t w = 0u;
    w = or_if_less<kBit0>(w, q0.x << 16, lds_at(thJ, a00 | b01 | lc.lb));
    w = or_if_less<kBit1>(w, q0.x, lds_at(thJ, a01 | b02 | lc.lb));
    w = or_if_less<kBit2>(w, q0.y << 16, lds_at(thJ, a10 | b11 | lc.lb));
    w = or_if_less<kBit3>(w, q0.y, lds_at(thJ, a11 | b12 | lc.lb));
    w = or_if_less<kBit4>(w, q0.z << 16, lds_at(thJ, a00 | b10 | lc.lb));
    w = or_if_less<kBit5>(w, q0.z, lds_at(thJ, a10 | b20 | lc.lb));
    w = or_if_less<kBit6>(w, q0.w << 16, lds_at(thJ, a01 | b11 | lc.lb));
    w = or_if_less<kBit7>(w, q0.w, lds_at(thJ, a11 | b21 | lc.lb));
    w = or_if_less<kBit8>(w, q1.x << 16, lds_at(thP, a00 | b11 | lc.lb));
    w = or_if_less<kBit9>(w, q1.x, lds_at(thP, a12 | b21 | lc.lb));
    vis = make_uint2(q1.y, q1.z);
    return w;
}

// Paper-precision hidden half-step of one cell from its records (the cell's
// row of visible draws is at byte offset h1.w); stores the lane's two
// visible-draw words there and returns its word W.
__device__ __forceinline__ uint32_t hidden_cell_rec_paper(char* sm, const uint4& h0, const uint4& h1,
                                                          const uint4& h2, const uint32_t* s_th,
                                                          const Round1Sweep& rs, uint32_t Y,
                                                          const uint32_t (&rk)[20], const LaneConst& lc,
                                                          uint32_t lane8) {
    uint2 vis;
    const uint32_t w =
        hidden_core_paper(lds_off(sm, h0.x), lds_off(sm, h0.x + 4u), lds_off(sm, h0.w), lds_off(sm, h0.y),
                          lds_off(sm, h0.y + 4u), lds_off(sm, h1.x), lds_off(sm, h0.z), lds_off(sm, h0.z + 4u),
                          s_th, rs, Y, h1.z, {h2.x, h2.y}, {h2.z, h2.w}, rk, lc, vis);
    *reinterpret_cast<uint2*>(sm + h1.w + lane8) = vis;
    return w;
}

// Paper-precision hidden half-step of one cell from its window rows (the
// streamed layout), with q0, q1 as for hidden_cell (the tag-2 product is not
// used); the visible half-step draws the tag-1 call again.
__device__ __forceinline__ uint32_t hidden_cell_paper(const uint32_t* s_v, int vs, const uint32_t* s_th,
                                                      const Round1Sweep& rs, uint32_t Y, const uint4& q0,
                                                      const uint4& q1, const uint32_t (&rk)[20],
                                                      const LaneConst& lc) {
    uint2 vis;
    return hidden_core_paper(s_v[0], s_v[1], s_v[2], s_v[vs], s_v[vs + 1], s_v[vs + 2], s_v[2 * vs],
                             s_v[2 * vs + 1], s_th, rs, Y, q0.x, {q0.y, q0.z}, {q0.w, q1.x}, rk, lc, vis);
}

// (rc.lo, Q1.h, Q1.l, 0): the cell's round-0 word and the round-1 product of
// its tag-1 call, whose words 1 and 2 carry the visible uniforms in paper
// precision.
__device__ __forceinline__ uint4 visible_call_words_paper(uint32_t cell, const uint32_t (&rk)[20]) {
    const Round0Cell rc = round0_cell(cell, rk[1]);
    const Round1Call c1 = round1_call(rc.a ^ 1u, rk);
    return make_uint4(rc.b, c1.h, c1.l, 0u);
}

// The four paper-precision decisions of a cell with site-class fields c
// (own, down and right bits merged) from its visible uniform words vis.
__device__ __forceinline__ U4 visible_decide_paper(uint32_t c, uint2 vis, const uint32_t* s_tv,
                                                   const LaneConst& lc) {
    const uint32_t f = 31u << 7;
    const uint32_t t00 = lds_at(s_tv, (c & f) | lc.lb);
    const uint32_t t01 = lds_at(s_tv + 1024, ((c >> 5) & f) | lc.lb);
    const uint32_t t10 = lds_at(s_tv + 2048, ((c >> 10) & f) | lc.lb);
    const uint32_t t11 = lds_at(s_tv + 3072, ((c >> 15) & f) | lc.lb);
    return {__ballot_sync(0xffffffffu, (vis.x << 16) < t00), __ballot_sync(0xffffffffu, vis.x < t01),
            __ballot_sync(0xffffffffu, (vis.y << 16) < t10), __ballot_sync(0xffffffffu, vis.y < t11)};
}

// Paper-precision visible half-step of one cell in the streamed layout, with
// qv = visible_call_words_paper(cell): the tag-1 call is drawn again for its
// words 1 and 2.  Stores as visible_cell.
__device__ __forceinline__ void visible_cell_paper(uint32_t* out, int row, uint32_t wo, uint32_t wu,
                                                   uint32_t wl, const uint32_t* s_tv, const Round1Sweep& rs,
                                                   uint32_t Y, const uint4& qv, const uint32_t (&rk)[20],
                                                   const LaneConst& lc) {
    const uint32_t c = (wo & kOwnBits) | (wu & kDownBits) | (wl & kRightBits);
    const U4 q = philox_from_call(Y, rs, round2_cell(rs.hik ^ qv.x), {qv.y, qv.z}, rk);
    const U4 o = visible_decide_paper(c, make_uint2(q.y, q.z), s_tv, lc);
    out[0] = o.x;
    out[1] = o.y;
    out[row] = o.z;
    out[row + 1] = o.w;
}

// Paper-precision visible half-step of one cell: the four uniforms are the
// halves of the two words its hidden half-step left at byte offset v1.z.
__device__ __forceinline__ U4 visible_cell_rec_paper(char* sm, const uint4& v0, const uint4& v1, uint32_t lane4,
                                                     const uint32_t* s_tv, const LaneConst& lc) {
    const uint32_t c = (lds_off(sm, v0.z + lane4) & kOwnBits) | (lds_off(sm, v0.w + lane4) & kDownBits) |
                       (lds_off(sm, v1.x + lane4) & kRightBits);
    const uint2 vis = *reinterpret_cast<const uint2*>(sm + v1.z + 2u * lane4);
    const U4 o = visible_decide_paper(c, vis, s_tv, lc);
    sts_off(sm, v0.x, o.x);
    sts_off(sm, v0.x + 4u, o.y);
    sts_off(sm, v0.y, o.z);
    sts_off(sm, v0.y + 4u, o.w);
    return o;
}

// Per-lane counts of one cell for the measurement from its eight window
// words: anti-aligned J and J' filters of the window, and +1 spins of the cell.
__device__ __forceinline__ void count_core(uint32_t w00, uint32_t w01, uint32_t w02, uint32_t w10, uint32_t w11,
                                           uint32_t w12, uint32_t w20, uint32_t w21, int lane, int& anti0,
                                           int& anti1, int& pos) {
    anti0 += bit_of(w00 ^ w01, lane) + bit_of(w01 ^ w02, lane) + bit_of(w10 ^ w11, lane) +
             bit_of(w11 ^ w12, lane) + bit_of(w00 ^ w10, lane) + bit_of(w10 ^ w20, lane) +
             bit_of(w01 ^ w11, lane) + bit_of(w11 ^ w21, lane);
    anti1 += bit_of(w00 ^ w11, lane) + bit_of(w12 ^ w21, lane);
    pos += bit_of(w00, lane) + bit_of(w01, lane) + bit_of(w10, lane) + bit_of(w11, lane);
}

__device__ __forceinline__ void count_cell(const uint32_t* s_v, int r0, int r1, int r2, int c0,
                                           int c1, int c2, int lane, int& anti0, int& anti1, int& pos) {
    count_core(s_v[r0 + c0], s_v[r0 + c1], s_v[r0 + c2], s_v[r1 + c0], s_v[r1 + c1], s_v[r1 + c2],
               s_v[r2 + c0], s_v[r2 + c1], lane, anti0, anti1, pos);
}

__device__ __forceinline__ void count_cell_rec(const char* sm, const uint4& h0, const uint4& h1, int lane,
                                               int& anti0, int& anti1, int& pos) {
    count_core(lds_off(sm, h0.x), lds_off(sm, h0.x + 4u), lds_off(sm, h0.w), lds_off(sm, h0.y),
               lds_off(sm, h0.y + 4u), lds_off(sm, h1.x), lds_off(sm, h0.z), lds_off(sm, h0.z + 4u), lane,
               anti0, anti1, pos);
}

}  // namespace canon
}  // namespace crbm
