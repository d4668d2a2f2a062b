// Per-cell cores of the canonical SS fast path (the ten filters of Fig. 1 on
// an even, periodic lattice), shared by the SMEM-resident sweep
// (crbm_canon.cu) and the streamed two-phase sweep (crbm_stream.cu).
//
// Mapping: warp = 32 chains of one packed word, lane = chain.  Each packed
// word a node depends on is masked to the lane's bit and rotated (funnel
// shift) straight into the address bits of a lane-expanded threshold table;
// OR-ing those bits with the lane's column offset gives the table address.
// The host builds the tables so that they absorb the coefficient signs s and
// the field sums (Eqs. 9-10): a node costs one address merge, one shared
// load, one compare and one ballot, plus its share of a Philox call.
#pragma once

#include "crbm_device.cuh"

namespace crbm {
namespace canon {

using namespace dev;

// Byte-addressed 32-bit shared-memory load.
__device__ __forceinline__ uint32_t lds_at(const uint32_t* base, uint32_t byte_off) {
    return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(base) + byte_off);
}

struct LaneConst {
    uint32_t lm;      // 1 << lane
    uint32_t lb;      // 4 * lane: the lane's column in a [.][32] table
    uint32_t rot[5];  // rotate-right amounts taking bit `lane` to bit 7 + j
};

// Hidden half-step of one cell (Eq. 9).  Table s_th[cls][e1 + 2 e2][lane]
// (byte offset cls*512 + idx*128 + 4 lane): the e1 bit is rotated to bit 7,
// the e2 bit to bit 8.
// Window rows are at s_v + r0, r1, r2 (offsets of window rows 0..2) and
// columns c0, c1, c2; the ten results go to h[0..9].
__device__ __forceinline__ void hidden_cell(const uint32_t* s_v, int r0, int r1, int r2, int c0,
                                            int c1, int c2, uint32_t* h, const uint32_t* s_th,
                                            uint32_t X, uint32_t Y, const Round0Cell rc,
                                            const uint32_t (&rk)[20], const LaneConst& lc) {
    const uint32_t m00 = s_v[r0 + c0] & lc.lm, m01 = s_v[r0 + c1] & lc.lm;
    const uint32_t m02 = s_v[r0 + c2] & lc.lm, m10 = s_v[r1 + c0] & lc.lm;
    const uint32_t m11 = s_v[r1 + c1] & lc.lm, m12 = s_v[r1 + c2] & lc.lm;
    const uint32_t m20 = s_v[r2 + c0] & lc.lm, m21 = s_v[r2 + c1] & lc.lm;
    // first endpoints at bit 7
    const uint32_t a00 = rotr(m00, lc.rot[0]), a01 = rotr(m01, lc.rot[0]);
    const uint32_t a10 = rotr(m10, lc.rot[0]), a11 = rotr(m11, lc.rot[0]);
    const uint32_t a12 = rotr(m12, lc.rot[0]);
    // second endpoints at bit 8
    const uint32_t b01 = rotr(m01, lc.rot[1]), b02 = rotr(m02, lc.rot[1]);
    const uint32_t b10 = rotr(m10, lc.rot[1]), b11 = rotr(m11, lc.rot[1]);
    const uint32_t b12 = rotr(m12, lc.rot[1]), b20 = rotr(m20, lc.rot[1]);
    const uint32_t b21 = rotr(m21, lc.rot[1]);
    const U4 q0 = philox_rounds1to9(X, Y, rc.a, rc.b, rk);
    const U4 q1 = philox_rounds1to9(X, Y, rc.a ^ 1u, rc.b, rk);
    const U4 q2 = philox_rounds1to9(X, Y, rc.a ^ 2u, rc.b, rk);
    const uint32_t* thJ = s_th;
    const uint32_t* thP = s_th + 128;
    // filters 0..7 (J) and 8..9 (J'): (first endpoint, second endpoint)
    h[0] = __ballot_sync(0xffffffffu, q0.x < lds_at(thJ, a00 | b01 | lc.lb));
    h[1] = __ballot_sync(0xffffffffu, q0.y < lds_at(thJ, a01 | b02 | lc.lb));
    h[2] = __ballot_sync(0xffffffffu, q0.z < lds_at(thJ, a10 | b11 | lc.lb));
    h[3] = __ballot_sync(0xffffffffu, q0.w < lds_at(thJ, a11 | b12 | lc.lb));
    h[4] = __ballot_sync(0xffffffffu, q1.x < lds_at(thJ, a00 | b10 | lc.lb));
    h[5] = __ballot_sync(0xffffffffu, q1.y < lds_at(thJ, a10 | b20 | lc.lb));
    h[6] = __ballot_sync(0xffffffffu, q1.z < lds_at(thJ, a01 | b11 | lc.lb));
    h[7] = __ballot_sync(0xffffffffu, q1.w < lds_at(thJ, a11 | b21 | lc.lb));
    h[8] = __ballot_sync(0xffffffffu, q2.x < lds_at(thP, a00 | b11 | lc.lb));
    h[9] = __ballot_sync(0xffffffffu, q2.y < lds_at(thP, a12 | b21 | lc.lb));
}

// Visible half-step of one cell (Eq. 10).  Each spin's five filter units sit
// in slots 0..4 (bits 7..11) of a 5-bit index into s_tv[site][idx][lane]
// (byte offset site*4096 + idx*128 + 4 lane).  Slot assignment (own cell /
// cell above "u" / cell to the left "l"), chosen so that a unit shared by two
// spins of the cell sits in the same slot for both:
//   spin (0,0): b0 b4 b8 l.b1 u.b5     spin (0,1): b0 b6 b1 u.b7 u.b9
//   spin (1,0): b2 b4 b5 l.b3 l.b9     spin (1,1): b2 b6 b8 b3 b7
// ho, hu, hl: the ten hidden words of this cell, the cell above and the cell
// to the left; the four new spin words go to out[0], out[1], out[row],
// out[row + 1].
__device__ __forceinline__ void visible_cell(uint32_t* out, int row, const uint32_t* ho,
                                             const uint32_t* hu, const uint32_t* hl,
                                             const uint32_t* s_tv, uint32_t X, uint32_t Y,
                                             const Round0Cell rc, const uint32_t (&rk)[20],
                                             const LaneConst& lc) {
    const uint32_t o0 = rotr(ho[0] & lc.lm, lc.rot[0]), o2 = rotr(ho[2] & lc.lm, lc.rot[0]);
    const uint32_t o4 = rotr(ho[4] & lc.lm, lc.rot[1]), o6 = rotr(ho[6] & lc.lm, lc.rot[1]);
    const uint32_t o8 = rotr(ho[8] & lc.lm, lc.rot[2]), o1 = rotr(ho[1] & lc.lm, lc.rot[2]);
    const uint32_t o5 = rotr(ho[5] & lc.lm, lc.rot[2]), o3 = rotr(ho[3] & lc.lm, lc.rot[3]);
    const uint32_t o7 = rotr(ho[7] & lc.lm, lc.rot[4]);
    const uint32_t l1 = rotr(hl[1] & lc.lm, lc.rot[3]), l3 = rotr(hl[3] & lc.lm, lc.rot[3]);
    const uint32_t l9 = rotr(hl[9] & lc.lm, lc.rot[4]);
    const uint32_t u5 = rotr(hu[5] & lc.lm, lc.rot[4]), u7 = rotr(hu[7] & lc.lm, lc.rot[3]);
    const uint32_t u9 = rotr(hu[9] & lc.lm, lc.rot[4]);
    const U4 q = philox_rounds1to9(X, Y, rc.a ^ kTagVis, rc.b, rk);
    const uint32_t t00 = lds_at(s_tv, o0 | o4 | o8 | l1 | u5 | lc.lb);
    const uint32_t t01 = lds_at(s_tv + 1024, o0 | o6 | o1 | u7 | u9 | lc.lb);
    const uint32_t t10 = lds_at(s_tv + 2048, o2 | o4 | o5 | l3 | l9 | lc.lb);
    const uint32_t t11 = lds_at(s_tv + 3072, o2 | o6 | o8 | o3 | o7 | lc.lb);
    out[0] = __ballot_sync(0xffffffffu, q.x < t00);
    out[1] = __ballot_sync(0xffffffffu, q.y < t01);
    out[row] = __ballot_sync(0xffffffffu, q.z < t10);
    out[row + 1] = __ballot_sync(0xffffffffu, q.w < t11);
}

// Per-lane counts of one cell for the measurement: anti-aligned J and J'
// filters of the window, and +1 spins of the cell.
__device__ __forceinline__ void count_cell(const uint32_t* s_v, int r0, int r1, int r2, int c0,
                                           int c1, int c2, int lane, int& anti0, int& anti1, int& pos) {
    const uint32_t w00 = s_v[r0 + c0], w01 = s_v[r0 + c1], w02 = s_v[r0 + c2];
    const uint32_t w10 = s_v[r1 + c0], w11 = s_v[r1 + c1], w12 = s_v[r1 + c2];
    const uint32_t w20 = s_v[r2 + c0], w21 = s_v[r2 + c1];
    anti0 += bit_of(w00 ^ w01, lane) + bit_of(w01 ^ w02, lane) + bit_of(w10 ^ w11, lane) +
             bit_of(w11 ^ w12, lane) + bit_of(w00 ^ w10, lane) + bit_of(w10 ^ w20, lane) +
             bit_of(w01 ^ w11, lane) + bit_of(w11 ^ w21, lane);
    anti1 += bit_of(w00 ^ w11, lane) + bit_of(w12 ^ w21, lane);
    pos += bit_of(w00, lane) + bit_of(w01, lane) + bit_of(w10, lane) + bit_of(w11, lane);
}

}  // namespace canon
}  // namespace crbm
