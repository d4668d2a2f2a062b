// Learned block proposal (Metropolis-Hastings block moves mixed with the
// Gibbs sweeps), canonical SS lattice (even L, periodic).
//
// A k x k block (k = 4) is proposed from a small convolutional net over the
// (k+6) x (k+6) patch around it: input channels 0 spin (0 inside the block),
// 1 block mask, 2 row parity, 3 column parity, 4 beta, 5 h; three valid 3x3
// convolutions 6 -> 16 -> 16 -> 1 with ReLU, one logit per block site,
// q_s = sigmoid(logit) = P(spin s = +1).  The net never sees the block's own
// spins, so the forward and reverse proposal probabilities come from the same
// q and the Metropolis-Hastings ratio exp(-beta dE/16) q(x) / q(x') is exact
// up to floating point (dE is an exact integer).  Blocks of one pass are at
// least 8 sites apart, so no block lies in another's receptive field or
// energy halo and the moves of a pass commute.
//
// The MH pass runs the three convolutions as implicit GEMMs on the tensor
// cores (mma.sync m16n8k16, bf16 operands, fp32 accumulation): rows are
// (chain, output position) of the 32 chains of a packed word, columns the 16
// output channels, K = (tap, input channel).  Layer 1's five constant planes
// are folded into per-position and per-chain constants, so its convolution
// runs on the spin plane alone (one k-tile).  Training runs one example per
// thread in fp32 (bf16-rounded weights and activations), back-propagates the
// binary cross-entropy and updates with Adam.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "crbm_context.h"
#include "crbm_device.cuh"

namespace crbm {
namespace {

using namespace dev;

constexpr int kK = 4;              // block side
constexpr int kP = kK + 6;         // patch side (10)
constexpr int kS1 = kK + 4;        // layer-1 output side (8)
constexpr int kS2 = kK + 2;        // layer-2 output side (6)
constexpr int kNP = 3345;          // parameters
constexpr uint32_t kTagOffset = 8u, kTagBits = 9u, kTagAccept = 13u, kTagExample = 14u;
constexpr int kPassThreads = 256;  // 8 warps

// Parameter offsets (W1[16][6][3][3], b1, W2[16][16][3][3], b2, W3[16][3][3], b3).
constexpr int oW1 = 0, oB1 = 864, oW2 = 880, oB2 = 3184, oW3 = 3200, oB3 = 3344;

// B-operand fragments of the three layers for mma m16n8k16 (per lane 2 x u32):
// layer 1: 1 k-tile (the nine taps of the spin plane) x 2 n-tiles, layer 2:
// 9 x 2, layer 3: 9 x 1.
constexpr int kFrag1 = 2, kFrag2 = 9 * 2, kFrag3 = 9;
constexpr int kFrags = kFrag1 + kFrag2 + kFrag3;

// Layer 1 on the five constant planes (block mask, row and column parity,
// beta, h) is linear in them and the same for every chain of a pass, so it is
// folded out of the convolution: per output position and channel a constant
// for each parity of the patch's first row and column ([4][64][16]), and the
// tap sums of the beta and h kernels ([2][16]).  Only the spin plane remains
// a convolution (K = 9 taps).
constexpr int kC1Pos = 4 * kS1 * kS1 * 16, kC1 = kC1Pos + 2 * 16;

// Shared memory of the pass, 32-bit words.  A1 and A2 hold bf16 activations,
// one 32-byte row per (chain, position) of 16 channels; the two 16-byte halves
// of row R are swapped when bit 2 of R is set, so the eight rows an ldmatrix
// phase reads (mostly consecutive) fall in distinct banks.
constexpr int kSmA1 = 0, kSmA2 = 32 * kS1 * kS1 * 8, kSmFr = kSmA2 + 32 * kS2 * kS2 * 8;
constexpr int kSmPw = kSmFr + kFrags * 32 * 2, kSmWords = kSmPw + kP * kP;

// Per (word, block, lane) record of a pass run in inspection mode: the
// logits, the proposed and current block bits, the exact dE and log alpha.
struct PassRecord {
    float logit[16];
    int32_t dE;
    uint32_t cur_bits, new_bits;
    float log_alpha;
    int32_t bR, bC;
    uint32_t thr[16];
};

struct PassArgs {
    Geometry g;
    PassRecord* rec;          // inspection mode when non-null: records, no move
    uint32_t* v;
    const uint2* frag;        // [kFrags][32] B fragments (bf16 pairs)
    const float* bias;        // b1[16], b2[16], b3
    const float* c1;          // folded layer-1 constants [kC1]
    const float* chain_bh;    // [chains][4] beta, h (bf16-rounded net inputs), beta (fp32), 0
    const int32_t* chain_q;   // [chains][3] Q.4 J, J', h
    unsigned long long* stats;  // {proposed, accepted}
    uint32_t key0, key1;
    uint32_t pass;
    int nb1, spacing;         // blocks per side, block spacing
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// The A fragment of one m16k16 tile from four 8x8 bf16 matrices in shared
// memory; each lane passes the address of one 16-byte matrix row.
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&p);
}

// Word offset of 16-byte half h of activation row R (see the layout above).
__device__ __forceinline__ int act_half(int R, int h) { return R * 8 + ((h ^ (R >> 2)) & 1) * 4; }

// One pass of MH block moves: CTA = (block of the pass, packed word).
__global__ void __launch_bounds__(kPassThreads, 2) k_prop_pass(const __grid_constant__ PassArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    const int L = a.g.L, N = a.g.N;
    const int word = blockIdx.y, b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    uint32_t* A1 = sm + kSmA1;                 // [32][64] rows, layer-1 output
    uint32_t* A2 = sm + kSmA2;                 // [32][36] rows, layer-2 output
    // layer-1 inputs, in A2's space until layer 2 writes it
    uint16_t* sp = reinterpret_cast<uint16_t*>(A2);        // [32][100] spin plane, bf16
    float* c1s = reinterpret_cast<float*>(A2 + 1600);       // [64][16] position constants
    float* cbs = c1s + kS1 * kS1 * 16;                      // [32][16] b1 + beta w_beta + h w_h
    uint2* fr = reinterpret_cast<uint2*>(sm + kSmFr);       // [kFrags][32]
    uint32_t* pw = sm + kSmPw;                              // [100] patch words
    // after layer 2 (A1 is free): logits and the Metropolis-Hastings terms
    // ([site][lane], so a warp's 32 chains fall in distinct banks)
    float* logit = reinterpret_cast<float*>(A1);   // [16][32]
    float* lqc = logit + 512;                      // [16][32] log q of the current spin
    float* lqn = lqc + 512;                        // [16][32] log q of the proposed spin
    int* s_xx = reinterpret_cast<int*>(lqn + 512);  // [16][32] bit 0: current +1, bit 1: proposed +1
    long long* s_de = reinterpret_cast<long long*>(s_xx + 512);  // [16][32] energy-change terms
    uint32_t* s_thr = reinterpret_cast<uint32_t*>(s_de + 512);    // [16][32] proposal thresholds
    const uint32_t a1_base = static_cast<uint32_t>(__cvta_generic_to_shared(A1));
    const uint32_t a2_base = static_cast<uint32_t>(__cvta_generic_to_shared(A2));

    // block origin of this pass
    const U4 off = philox(a.pass, 0u, 0u, kTagOffset, a.key0, a.key1);
    const int bR = static_cast<int>((off.x % static_cast<uint32_t>(L) + a.spacing * (b / a.nb1)) % L);
    const int bC = static_cast<int>((off.y % static_cast<uint32_t>(L) + a.spacing * (b % a.nb1)) % L);
    for (int x = threadIdx.x; x < kP * kP; x += blockDim.x) {  // per patch position
        const int R = (bR - 3 + x / kP + 2 * L) % L, C = (bC - 3 + x % kP + 2 * L) % L;
        pw[x] = a.v[static_cast<size_t>(word) * N + R * L + C];
    }
    {
        const int var = ((bR + 1) & 1) * 2 + ((bC + 1) & 1);  // parity of the patch's first row, column
        const float* c1v = a.c1 + var * (kS1 * kS1 * 16);
        for (int i = threadIdx.x; i < kS1 * kS1 * 16; i += blockDim.x) c1s[i] = c1v[i];
        for (int i = threadIdx.x; i < 32 * 16; i += blockDim.x) {
            const int c = i >> 4, n = i & 15, chain = word * 32 + c;
            cbs[i] = a.bias[n] + a.chain_bh[4 * chain] * a.c1[kC1Pos + n] +
                     a.chain_bh[4 * chain + 1] * a.c1[kC1Pos + 16 + n];
        }
    }
    for (int x = threadIdx.x; x < kFrags * 32; x += blockDim.x) fr[x] = a.frag[x];
    __syncthreads();
    // spin plane: +-1 outside the block, 0 inside
    for (int x = threadIdx.x; x < 32 * kP * kP; x += blockDim.x) {
        const int c = x / (kP * kP), pos = x - c * (kP * kP);
        const int y = pos / kP, xx = pos - y * kP;
        const bool in = y >= 3 && y < 3 + kK && xx >= 3 && xx < 3 + kK;
        sp[x] = in ? 0 : (((pw[pos] >> c) & 1u) ? 0x3F80 : 0xBF80);
    }
    __syncthreads();
    // ---- layer 1: rows (chain, y*8+x) = 2048 (128 m-tiles), K = 9 taps
    for (int mt = warp; mt < 128; mt += kPassThreads / 32) {
        const int chain = mt >> 2, p0 = (mt & 3) * 16;
        const int pA = p0 + gq, pB = p0 + gq + 8;  // the two rows of this lane
        const uint16_t* sc = sp + chain * kP * kP;
        const int oA = (pA >> 3) * kP + (pA & 7), oB = (pB >> 3) * kP + (pB & 7);
        const int t0 = 2 * tq, t1 = 2 * tq + 1;
        const int d0 = (t0 / 3) * kP + t0 % 3, d1 = (t1 / 3) * kP + t1 % 3;
        uint32_t af[4];
        af[0] = sc[oA + d0] | (static_cast<uint32_t>(sc[oA + d1]) << 16);
        af[1] = sc[oB + d0] | (static_cast<uint32_t>(sc[oB + d1]) << 16);
        af[2] = tq == 0 ? sc[oA + 2 * kP + 2] : 0u;  // tap 8; taps 9-15 are padding
        af[3] = tq == 0 ? sc[oB + 2 * kP + 2] : 0u;
        float d[2][4] = {};
        mma_bf16(d[0], af, fr[0 * 32 + lane]);
        mma_bf16(d[1], af, fr[1 * 32 + lane]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int n = 8 * nt + 2 * tq;
            const float2 cb = *reinterpret_cast<const float2*>(cbs + chain * 16 + n);
            const float2 cA = *reinterpret_cast<const float2*>(c1s + pA * 16 + n);
            const float2 cB = *reinterpret_cast<const float2*>(c1s + pB * 16 + n);
            const int RA = chain * 64 + pA, RB = chain * 64 + pB;
            A1[act_half(RA, nt) + tq] = pack_bf16(fmaxf(d[nt][0] + (cA.x + cb.x), 0.f), fmaxf(d[nt][1] + (cA.y + cb.y), 0.f));
            A1[act_half(RB, nt) + tq] = pack_bf16(fmaxf(d[nt][2] + (cB.x + cb.x), 0.f), fmaxf(d[nt][3] + (cB.y + cb.y), 0.f));
        }
    }
    __syncthreads();
    // ---- layer 2: rows (chain, y*6+x) = 1152 (72 m-tiles), K = 9 taps x 16 ch.
    // ldmatrix: lane l gives the row (l & 7) + 8 ((l >> 3) & 1), half l >> 4.
    const int lrow = (lane & 7) + 8 * ((lane >> 3) & 1), lhalf = lane >> 4;
    uint2 b2[kFrag2];  // this lane's B fragments of layer 2, kept for all its m-tiles
#pragma unroll
    for (int f = 0; f < kFrag2; ++f) b2[f] = fr[(kFrag1 + f) * 32 + lane];
    for (int mt = warp; mt < 72; mt += kPassThreads / 32) {
        const int r = mt * 16 + lrow;
        const int c = r / 36, q = r - c * 36;
        const int R0 = c * 64 + (q / 6) * 8 + q % 6;
        float d[2][4] = {};
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int R = R0 + (tap / 3) * 8 + tap % 3;
            uint32_t af[4];
            ldmatrix_x4(af, a1_base + 4u * static_cast<uint32_t>(act_half(R, lhalf)));
            mma_bf16(d[0], af, b2[tap * 2 + 0]);
            mma_bf16(d[1], af, b2[tap * 2 + 1]);
        }
        const int rA = mt * 16 + gq, rB = rA + 8;
        const int cA = rA / 36, qA = rA - cA * 36, cB = rB / 36, qB = rB - cB * 36;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int n = 8 * nt + 2 * tq;
            const float b0 = a.bias[16 + n], b1 = a.bias[16 + n + 1];
            A2[act_half(cA * 36 + qA, nt) + tq] = pack_bf16(fmaxf(d[nt][0] + b0, 0.f), fmaxf(d[nt][1] + b1, 0.f));
            A2[act_half(cB * 36 + qB, nt) + tq] = pack_bf16(fmaxf(d[nt][2] + b0, 0.f), fmaxf(d[nt][3] + b1, 0.f));
        }
    }
    __syncthreads();
    // ---- layer 3: rows (chain, y*4+x) = 512 (32 m-tiles), one output channel
    for (int mt = warp; mt < 32; mt += kPassThreads / 32) {
        const int ch = mt;  // one m-tile = the 16 block sites of chain mt
        const int R0 = ch * 36 + (lrow >> 2) * 6 + (lrow & 3);
        float d[4] = {};
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int R = R0 + (tap / 3) * 6 + tap % 3;
            uint32_t af[4];
            ldmatrix_x4(af, a2_base + 4u * static_cast<uint32_t>(act_half(R, lhalf)));
            mma_bf16(d, af, fr[(kFrag1 + kFrag2 + tap) * 32 + lane]);
        }
        if (tq == 0) {
            logit[gq * 32 + ch] = d[0] + a.bias[32];
            logit[(gq + 8) * 32 + ch] = d[2] + a.bias[32];
        }
    }
    __syncthreads();
    // ---- Metropolis-Hastings, phase A on every warp: lane = chain, warp w
    // draws Philox call w / 2 of its chain (4 sites) and takes sites
    // 4 (w / 2) + 2 (w % 2) + {0, 1}: threshold, log q of the current and the
    // proposed spin, the proposed spin.
    const int chain = word * 32 + lane;
    const uint32_t cell_id = static_cast<uint32_t>(b);
    const int qJ = a.chain_q[3 * chain], qJp = a.chain_q[3 * chain + 1], qh = a.chain_q[3 * chain + 2];
    {
        const int call = warp >> 1;
        const U4 u = philox(cell_id, a.pass, static_cast<uint32_t>(chain), kTagBits + call, a.key0, a.key1);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int s = 4 * call + 2 * (warp & 1) + j;
            const int pos = (3 + s / kK) * kP + 3 + s % kK;
            const int xc = ((pw[pos] >> lane) & 1u) ? 1 : -1;
            const float q = 1.f / (1.f + __expf(-logit[s * 32 + lane]));
            float tf = q * 4294967296.f;
            tf = fminf(fmaxf(tf, 1.f), 4294967040.f);
            const uint32_t thr = static_cast<uint32_t>(tf);
            const float p1 = static_cast<float>(thr) * 2.3283064365386963e-10f;
            const float lp = __logf(p1), lm = log1pf(-p1);
            const int xp = pick(u, s & 3) < thr ? 1 : -1;
            lqc[s * 32 + lane] = xc > 0 ? lp : lm;
            lqn[s * 32 + lane] = xp > 0 ? lp : lm;
            s_xx[s * 32 + lane] = (xc > 0 ? 1 : 0) | (xp > 0 ? 2 : 0);
            s_thr[s * 32 + lane] = thr;
        }
    }
    __syncthreads();
    // phase A': each site's share of the exact energy change (1/16 units) over
    // the bonds touching the block; a bond inside the block is counted by its
    // left / upper endpoint (right and down neighbours, and the dimer partner
    // of higher index)
    {
        auto spin_at = [&](int pr, int pc) -> int { return ((pw[pr * kP + pc] >> lane) & 1u) ? 1 : -1; };
        auto xs = [&](int t) { return (s_xx[t * 32 + lane] & 1) ? 1 : -1; };
        auto ns = [&](int t) { return (s_xx[t * 32 + lane] & 2) ? 1 : -1; };
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int s = 4 * (warp >> 1) + 2 * (warp & 1) + j;
            const int ar = s / kK, ac = s % kK;
            const int x0 = xs(s), n0 = ns(s), d = n0 - x0;
            long long dE = -static_cast<long long>(qh) * d;
            if (ac + 1 < kK) dE += static_cast<long long>(qJ) * (n0 * ns(s + 1) - x0 * xs(s + 1));
            else dE += static_cast<long long>(qJ) * d * spin_at(3 + ar, 3 + ac + 1);
            if (ar + 1 < kK) dE += static_cast<long long>(qJ) * (n0 * ns(s + kK) - x0 * xs(s + kK));
            else dE += static_cast<long long>(qJ) * d * spin_at(3 + ar + 1, 3 + ac);
            if (ac == 0) dE += static_cast<long long>(qJ) * d * spin_at(3 + ar, 2);
            if (ar == 0) dE += static_cast<long long>(qJ) * d * spin_at(2, 3 + ac);
            // the orthogonal dimer of this site
            const int R = bR + ar, C = bC + ac;
            const int dR = (R & 1) ? ((C & 1) ? -1 : 1) : ((C & 1) ? -1 : 1);
            const int dC = (R & 1) ? -1 : 1;
            const int pr = ar + dR, pc = ac + dC;
            if (pr >= 0 && pr < kK && pc >= 0 && pc < kK) {
                const int t = pr * kK + pc;
                if (t > s) dE += static_cast<long long>(qJp) * (n0 * ns(t) - x0 * xs(t));
            } else {
                dE += static_cast<long long>(qJp) * d * spin_at(3 + pr, 3 + pc);
            }
            s_de[s * 32 + lane] = dE;
        }
    }
    __syncthreads();
    // ---- phase B, warp 0, lane = chain: sums over the sites in site order,
    // the exact MH test and the move
    if (warp != 0) return;
    float logq_cur = 0.f, logq_new = 0.f;
    long long dE = 0;
    uint32_t cb = 0, nb = 0;
#pragma unroll
    for (int s = 0; s < kK * kK; ++s) {
        logq_cur += lqc[s * 32 + lane];
        logq_new += lqn[s * 32 + lane];
        dE += s_de[s * 32 + lane];
        const int xx = s_xx[s * 32 + lane];
        cb |= static_cast<uint32_t>(xx & 1) << s;
        nb |= static_cast<uint32_t>((xx >> 1) & 1) << s;
    }
    const float beta = a.chain_bh[4 * chain + 2];  // the exact beta: the MH test targets exp(-beta H)
    const float log_alpha = -beta * static_cast<float>(dE) * 0.0625f + logq_cur - logq_new;
    const U4 ua = philox(cell_id, a.pass, static_cast<uint32_t>(chain), kTagAccept, a.key0, a.key1);
    const bool accept = log_alpha >= 0.f ||
                        static_cast<float>(ua.x >> 8) * 5.9604644775390625e-08f < __expf(log_alpha);
    if (a.rec) {  // inspection: record, do not move
        PassRecord* r = a.rec + (static_cast<size_t>(word) * gridDim.x + b) * 32 + lane;
#pragma unroll
        for (int s = 0; s < kK * kK; ++s) {
            r->logit[s] = logit[s * 32 + lane];
            r->thr[s] = s_thr[s * 32 + lane];
        }
        r->dE = static_cast<int32_t>(dE);
        r->cur_bits = cb;
        r->new_bits = nb;
        r->log_alpha = log_alpha;
        r->bR = bR;
        r->bC = bC;
        return;
    }
    const uint32_t am = __ballot_sync(0xffffffffu, accept);
#pragma unroll
    for (int s = 0; s < kK * kK; ++s) {
        const uint32_t wv = __ballot_sync(0xffffffffu, ((accept ? nb : cb) >> s) & 1u);
        if (lane == s) {
            const int R = (bR + s / kK) % L, C = (bC + s % kK) % L;
            a.v[static_cast<size_t>(word) * N + R * L + C] = wv;
        }
    }
    if (lane == 0) {
        atomicAdd(&a.stats[0], 32ull);
        atomicAdd(&a.stats[1], static_cast<unsigned long long>(__popc(am)));
    }
}


// ---------------------------------------------------------------- training
// One training example: the patch around a block of one chain, compactly.
struct Example {
    int8_t spin[kP * kP];     // +-1 outside the block, 0 inside
    uint8_t inside[kP * kP];  // block mask
    int8_t target[kK * kK];   // the block's spins
    uint8_t pr, pc;           // row / column parity of the patch's first site
    uint8_t pad[2];
    float beta, h;            // bf16-rounded
};

// Draw examples from a context's chains: chain and block origin from Philox.
__global__ void k_prop_extract(Geometry g, const uint32_t* v, const float* chain_bh, int n_chains,
                               Example* ex, int n, uint32_t step, uint32_t k0, uint32_t k1) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int L = g.L;
    const U4 r = philox(static_cast<uint32_t>(e), step, 0u, kTagExample, k0, k1);
    const int c = static_cast<int>(r.x % static_cast<uint32_t>(n_chains));
    const int bR = static_cast<int>(r.y % static_cast<uint32_t>(L)), bC = static_cast<int>(r.z % static_cast<uint32_t>(L));
    Example& x = ex[e];
    for (int pos = 0; pos < kP * kP; ++pos) {
        const int R = (bR - 3 + pos / kP + 2 * L) % L, C = (bC - 3 + pos % kP + 2 * L) % L;
        const bool in = ((R - bR + L) % L) < kK && ((C - bC + L) % L) < kK;
        const int sp = ((v[static_cast<size_t>(c >> 5) * g.N + R * L + C] >> (c & 31)) & 1u) ? 1 : -1;
        x.spin[pos] = in ? 0 : static_cast<int8_t>(sp);
        x.inside[pos] = in ? 1 : 0;
    }
    for (int s = 0; s < kK * kK; ++s) {
        const int R = (bR + s / kK) % L, C = (bC + s % kK) % L;
        x.target[s] = ((v[static_cast<size_t>(c >> 5) * g.N + R * L + C] >> (c & 31)) & 1u) ? 1 : -1;
    }
    x.pr = static_cast<uint8_t>((bR + 1) & 1);  // parity of row bR - 3 (L even)
    x.pc = static_cast<uint8_t>((bC + 1) & 1);
    x.beta = chain_bh[4 * c];
    x.h = chain_bh[4 * c + 1];
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Forward + backward of the mean binary cross-entropy, one example per
// thread, fp32 arithmetic on bf16-rounded weights and activations (the
// roundings pass gradients straight through).  grad and loss accumulate.
__global__ void __launch_bounds__(128) k_prop_train(const float* __restrict__ w, const Example* ex, int n,
                                                    float* grad, float* loss) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const Example& x = ex[e];
    float in[6][kP * kP];
    for (int pos = 0; pos < kP * kP; ++pos) {
        in[0][pos] = x.spin[pos];
        in[1][pos] = x.inside[pos];
        in[2][pos] = static_cast<float>((x.pr + pos / kP) & 1);
        in[3][pos] = static_cast<float>((x.pc + pos % kP) & 1);
        in[4][pos] = x.beta;
        in[5][pos] = x.h;
    }
    float a1[16][kS1 * kS1], a2[16][kS2 * kS2];
    for (int o = 0; o < 16; ++o)
        for (int p = 0; p < kS1 * kS1; ++p) {
            const int y = p / kS1, xx = p % kS1;
            float acc = w[oB1 + o];
            for (int c = 0; c < 6; ++c)
                for (int t = 0; t < 9; ++t) acc += w[oW1 + (o * 6 + c) * 9 + t] * in[c][(y + t / 3) * kP + xx + t % 3];
            a1[o][p] = bf16r(fmaxf(acc, 0.f));
        }
    for (int o = 0; o < 16; ++o)
        for (int p = 0; p < kS2 * kS2; ++p) {
            const int y = p / kS2, xx = p % kS2;
            float acc = w[oB2 + o];
            for (int c = 0; c < 16; ++c)
                for (int t = 0; t < 9; ++t) acc += w[oW2 + (o * 16 + c) * 9 + t] * a1[c][(y + t / 3) * kS1 + xx + t % 3];
            a2[o][p] = bf16r(fmaxf(acc, 0.f));
        }
    float lsum = 0.f, dl[kK * kK];
    for (int p = 0; p < kK * kK; ++p) {
        const int y = p / kK, xx = p % kK;
        float acc = w[oB3];
        for (int c = 0; c < 16; ++c)
            for (int t = 0; t < 9; ++t) acc += w[oW3 + c * 9 + t] * a2[c][(y + t / 3) * kS2 + xx + t % 3];
        const float yv = x.target[p] > 0 ? 1.f : 0.f;
        lsum += (acc > 0.f ? acc + log1pf(__expf(-acc)) : log1pf(__expf(acc))) - yv * acc;
        dl[p] = (1.f / (1.f + __expf(-acc)) - yv) / (static_cast<float>(n) * kK * kK);
    }
    atomicAdd(loss, lsum / (static_cast<float>(n) * kK * kK));
    // layer 3
    float d2[16][kS2 * kS2];
    for (int c = 0; c < 16; ++c)
        for (int p = 0; p < kS2 * kS2; ++p) d2[c][p] = 0.f;
    float gb3 = 0.f;
    for (int p = 0; p < kK * kK; ++p) gb3 += dl[p];
    atomicAdd(&grad[oB3], gb3);
    for (int c = 0; c < 16; ++c)
        for (int t = 0; t < 9; ++t) {
            float gsum = 0.f;
            const float wv = w[oW3 + c * 9 + t];
            for (int p = 0; p < kK * kK; ++p) {
                const int q = (p / kK + t / 3) * kS2 + p % kK + t % 3;
                gsum += dl[p] * a2[c][q];
                d2[c][q] += dl[p] * wv;
            }
            atomicAdd(&grad[oW3 + c * 9 + t], gsum);
        }
    for (int c = 0; c < 16; ++c)
        for (int p = 0; p < kS2 * kS2; ++p)
            if (!(a2[c][p] > 0.f)) d2[c][p] = 0.f;
    // layer 2
    float d1[16][kS1 * kS1];
    for (int c = 0; c < 16; ++c)
        for (int p = 0; p < kS1 * kS1; ++p) d1[c][p] = 0.f;
    for (int o = 0; o < 16; ++o) {
        float gb = 0.f;
        for (int p = 0; p < kS2 * kS2; ++p) gb += d2[o][p];
        atomicAdd(&grad[oB2 + o], gb);
        for (int c = 0; c < 16; ++c)
            for (int t = 0; t < 9; ++t) {
                float gsum = 0.f;
                const float wv = w[oW2 + (o * 16 + c) * 9 + t];
                for (int p = 0; p < kS2 * kS2; ++p) {
                    const int q = (p / kS2 + t / 3) * kS1 + p % kS2 + t % 3;
                    gsum += d2[o][p] * a1[c][q];
                    d1[c][q] += d2[o][p] * wv;
                }
                atomicAdd(&grad[oW2 + (o * 16 + c) * 9 + t], gsum);
            }
    }
    for (int c = 0; c < 16; ++c)
        for (int p = 0; p < kS1 * kS1; ++p)
            if (!(a1[c][p] > 0.f)) d1[c][p] = 0.f;
    // layer 1
    for (int o = 0; o < 16; ++o) {
        float gb = 0.f;
        for (int p = 0; p < kS1 * kS1; ++p) gb += d1[o][p];
        atomicAdd(&grad[oB1 + o], gb);
        for (int c = 0; c < 6; ++c)
            for (int t = 0; t < 9; ++t) {
                float gsum = 0.f;
                for (int p = 0; p < kS1 * kS1; ++p)
                    gsum += d1[o][p] * in[c][(p / kS1 + t / 3) * kP + p % kS1 + t % 3];
                atomicAdd(&grad[oW1 + (o * 6 + c) * 9 + t], gsum);
            }
    }
}

// Adam (Kingma & Ba) on the fp32 master weights; also refreshes the
// bf16-rounded copy the kernels read.
__global__ void k_prop_adam(float* w, float* wb, float* m, float* v2, const float* grad, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    m[i] = b1 * m[i] + (1.f - b1) * g;
    v2[i] = b2 * v2[i] + (1.f - b2) * g * g;
    w[i] -= lr * (m[i] / c1) / (sqrtf(v2[i] / c2) + eps);
    wb[i] = bf16r(w[i]);
}

__global__ void k_prop_round(const float* w, float* wb, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = bf16r(w[i]);
}

// mma B fragments and biases from the bf16-rounded weights (device side, so
// the fragments follow the trained weights without a host round trip).
__global__ void k_prop_fragments(const float* wb, uint2* frag, float* bias) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 33) bias[i] = i < 16 ? wb[oB1 + i] : (i < 32 ? wb[oB2 + i - 16] : wb[oB3]);
    if (i >= kFrags * 32) return;
    const int f = i / 32, lane = i % 32, gq = lane >> 2, tq = lane & 3;
    auto Bv = [&](int k, int n) -> float {
        if (f < kFrag1) return k < 9 ? wb[oW1 + n * 6 * 9 + k] : 0.f;  // layer 1: k = tap of the spin plane
        if (f < kFrag1 + kFrag2) {  // layer 2: k = tap * 16 + channel
            return wb[oW2 + (n * 16 + (k & 15)) * 9 + (k >> 4)];
        }
        return n == 0 ? wb[oW3 + (k & 15) * 9 + (k >> 4)] : 0.f;  // layer 3
    };
    int kt, nt;
    if (f < kFrag1) {
        kt = f / 2;
        nt = f % 2;
    } else if (f < kFrag1 + kFrag2) {
        kt = (f - kFrag1) / 2;
        nt = (f - kFrag1) % 2;
    } else {
        kt = f - kFrag1 - kFrag2;
        nt = 0;
    }
    const int n = 8 * nt + gq, k0 = 16 * kt + 2 * tq;
    frag[i] = make_uint2(pack_bf16(Bv(k0, n), Bv(k0 + 1, n)), pack_bf16(Bv(k0 + 8, n), Bv(k0 + 9, n)));
}

// The folded layer-1 constants (see kC1Pos) from the bf16-rounded weights:
// per parity variant (row parity pr, column parity pc of the patch's first
// site), output position and channel, the sum over the nine taps of the mask
// and parity kernels times their planes; then the tap sums of the beta and h
// kernels.
__global__ void k_prop_layer1_consts(const float* wb, float* c1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kC1) return;
    if (i >= kC1Pos) {
        const int ch = 4 + (i - kC1Pos) / 16, n = (i - kC1Pos) % 16;
        float s = 0.f;
        for (int tap = 0; tap < 9; ++tap) s += wb[oW1 + (n * 6 + ch) * 9 + tap];
        c1[i] = s;
        return;
    }
    const int var = i / (kS1 * kS1 * 16), p = (i / 16) % (kS1 * kS1), n = i % 16;
    const int pr = var >> 1, pc = var & 1, y = p / kS1, x = p % kS1;
    float s = 0.f;
    for (int tap = 0; tap < 9; ++tap) {
        const int Y = y + tap / 3, X = x + tap % 3;
        const bool in = Y >= 3 && Y < 3 + kK && X >= 3 && X < 3 + kK;
        if (in) s += wb[oW1 + (n * 6 + 1) * 9 + tap];
        if ((pr + Y) & 1) s += wb[oW1 + (n * 6 + 2) * 9 + tap];
        if ((pc + X) & 1) s += wb[oW1 + (n * 6 + 3) * 9 + tap];
    }
    c1[i] = s;
}

}  // namespace
}  // namespace crbm

// ------------------------------------------------------------------- host
struct crbm_proposal {
    int device = 0;
    float* w = nullptr;      // fp32 master weights
    float* wb = nullptr;     // bf16-rounded copy
    float* m = nullptr;      // Adam moments
    float* v2 = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;
    uint2* frag = nullptr;   // mma B fragments
    float* bias = nullptr;
    float* c1 = nullptr;     // folded layer-1 constants
    unsigned long long* stats = nullptr;
    crbm::Example* ex = nullptr;
    int ex_cap = 0;
    int64_t adam_t = 0;
    uint64_t seed = 0;
};

namespace {

using crbm::Example;
using crbm::kNP;

thread_local std::string g_prop_error;

int prop_fail(int code, const std::string& msg) {
    g_prop_error = msg;
    return code;
}

// splitmix64 (Steele, Lea, Flood) for the initial weights
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double unit_normal(uint64_t& s) {  // Box-Muller
    const double u1 = (static_cast<double>(splitmix(s) >> 11) + 0.5) * 0x1.0p-53;
    const double u2 = (static_cast<double>(splitmix(s) >> 11) + 0.5) * 0x1.0p-53;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

cudaError_t refresh_fragments(crbm_proposal* p, cudaStream_t st) {
    crbm::k_prop_fragments<<<(crbm::kFrags * 32 + 127) / 128, 128, 0, st>>>(p->wb, p->frag, p->bias);
    crbm::k_prop_layer1_consts<<<(crbm::kC1 + 127) / 128, 128, 0, st>>>(p->wb, p->c1);
    return cudaGetLastError();
}

// Per-chain (beta, h) and Q.4 couplings of a context, on the device:
// chain_bh[c] = {bf16(beta), bf16(h), beta, 0} (the net reads the bf16
// inputs, the Metropolis-Hastings test the fp32 beta).
int ensure_chain_params(crbm_ctx* ctx) {
    if (ctx->d.chain_bh) return CRBM_OK;
    const int npad = ctx->n_words * 32;
    std::vector<float> bh(4 * static_cast<size_t>(npad));
    std::vector<int32_t> cq(3 * static_cast<size_t>(npad));
    auto bf16 = [](float x) {  // round to nearest even, 8 significant bits
        uint32_t u;
        std::memcpy(&u, &x, 4);
        u += 0x7fffu + ((u >> 16) & 1u);
        u &= 0xffff0000u;
        std::memcpy(&x, &u, 4);
        return x;
    };
    for (int c = 0; c < npad; ++c) {
        const int p = ctx->chain_param[c < ctx->n_chains ? c : 0];
        bh[4 * c] = bf16(static_cast<float>(ctx->beta[p]));
        bh[4 * c + 1] = bf16(static_cast<float>(ctx->q[2][p]) * 0.0625f);
        bh[4 * c + 2] = static_cast<float>(ctx->beta[p]);
        bh[4 * c + 3] = 0.f;
        cq[3 * c] = ctx->q[0][p];
        cq[3 * c + 1] = ctx->q[1][p];
        cq[3 * c + 2] = ctx->q[2][p];
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&ctx->d.chain_bh), bh.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&ctx->d.chain_q), cq.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d.chain_bh, bh.data(), bh.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d.chain_q, cq.data(), cq.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return prop_fail(CRBM_ECUDA, std::string("chain parameters: ") + cudaGetErrorString(e));
    return CRBM_OK;
}

int check_ctx(const crbm_ctx* ctx) {
    if (!ctx) return prop_fail(CRBM_EINVAL, "null context");
    if (!ctx->g.canonical || ctx->g.Lc != ctx->g.L || ctx->g.L < crbm::kP || ctx->layout != CRBM_LAYOUT_SMEM ||
        ctx->swap_every > 0 || ctx->g.paper || ctx->g.bitplane)
        return prop_fail(CRBM_EUNSUPPORTED,
                         "block proposals need the ten SS filters on an even periodic square lattice of side "
                         ">= 10 (a patch must not wrap onto its own block), the SMEM layout, exact precision, "
                         "lane uniforms and no replica exchange");
    return CRBM_OK;
}

int ensure_examples(crbm_proposal* p, int n) {
    if (n <= p->ex_cap) return CRBM_OK;
    cudaFree(p->ex);
    p->ex = nullptr;
    p->ex_cap = 0;
    if (cudaMalloc(reinterpret_cast<void**>(&p->ex), static_cast<size_t>(n) * sizeof(Example)) != cudaSuccess)
        return prop_fail(CRBM_ENOMEM, "examples");
    p->ex_cap = n;
    return CRBM_OK;
}

cudaError_t launch_pass(crbm_ctx* ctx, crbm_proposal* p, crbm::PassRecord* rec) {
    const int L = ctx->g.L;
    const int nb1 = std::max(1, L / 8);
    crbm::PassArgs a{};
    a.g = ctx->g;
    a.rec = rec;
    a.v = ctx->d.v;
    a.frag = p->frag;
    a.bias = p->bias;
    a.c1 = p->c1;
    a.chain_bh = ctx->d.chain_bh;
    a.chain_q = ctx->d.chain_q;
    a.stats = p->stats;
    a.key0 = static_cast<uint32_t>(ctx->seed);
    a.key1 = static_cast<uint32_t>(ctx->seed >> 32);
    a.pass = static_cast<uint32_t>(ctx->passes);
    a.nb1 = nb1;
    a.spacing = L / nb1;
    const size_t smem = crbm::kSmWords * 4;
    cudaError_t e = cudaFuncSetAttribute(crbm::k_prop_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    crbm::k_prop_pass<<<dim3(nb1 * nb1, ctx->n_words), crbm::kPassThreads, smem, ctx->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int crbm_proposal_create(crbm_proposal** out, int32_t block, uint64_t seed) {
    if (!out) return prop_fail(CRBM_EINVAL, "null argument");
    *out = nullptr;
    if (block != crbm::kK) return prop_fail(CRBM_EUNSUPPORTED, "block side must be 4");
    crbm_proposal* p = new (std::nothrow) crbm_proposal();
    if (!p) return prop_fail(CRBM_ENOMEM, "host allocation");
    p->seed = seed;
    cudaGetDevice(&p->device);
    cudaError_t e = cudaSuccess;
    float** bufs[] = {&p->w, &p->wb, &p->m, &p->v2, &p->grad};
    for (float** b : bufs)
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(b), kNP * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->loss), sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->frag), crbm::kFrags * 32 * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->bias), 33 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->c1), crbm::kC1 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->stats), 2 * sizeof(unsigned long long));
    // He-style initial weights; the output layer starts small (q near 1/2)
    std::vector<float> w(kNP, 0.f);
    uint64_t s = seed ^ 0x243F6A8885A308D3ull;
    for (int i = 0; i < 864; ++i) w[crbm::oW1 + i] = static_cast<float>(unit_normal(s) * std::sqrt(2.0 / 54.0));
    for (int i = 0; i < 2304; ++i) w[crbm::oW2 + i] = static_cast<float>(unit_normal(s) * std::sqrt(2.0 / 144.0));
    for (int i = 0; i < 144; ++i) w[crbm::oW3 + i] = static_cast<float>(unit_normal(s) * 0.01);
    if (e == cudaSuccess) e = cudaMemcpy(p->w, w.data(), kNP * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->m, 0, kNP * 4);
    if (e == cudaSuccess) e = cudaMemset(p->v2, 0, kNP * 4);
    if (e == cudaSuccess) e = cudaMemset(p->stats, 0, 16);
    if (e == cudaSuccess) {
        crbm::k_prop_round<<<(kNP + 255) / 256, 256>>>(p->w, p->wb, kNP);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = refresh_fragments(p, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        crbm_proposal_destroy(p);
        return prop_fail(CRBM_ECUDA, std::string("crbm_proposal_create: ") + cudaGetErrorString(e));
    }
    *out = p;
    return CRBM_OK;
}

void crbm_proposal_destroy(crbm_proposal* p) {
    if (!p) return;
    void* b[] = {p->w, p->wb, p->m, p->v2, p->grad, p->loss, p->frag, p->bias, p->c1, p->stats, p->ex};
    for (void* x : b)
        if (x) cudaFree(x);
    delete p;
}

int crbm_proposal_set_weights(crbm_proposal* p, const float* w, size_t n) {
    if (!p || !w || n != static_cast<size_t>(kNP)) return prop_fail(CRBM_EINVAL, "need 3345 weights");
    cudaError_t e = cudaMemcpy(p->w, w, kNP * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        crbm::k_prop_round<<<(kNP + 255) / 256, 256>>>(p->w, p->wb, kNP);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = refresh_fragments(p, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? CRBM_OK : prop_fail(CRBM_ECUDA, cudaGetErrorString(e));
}

int crbm_proposal_get_weights(crbm_proposal* p, float* w, size_t n) {
    if (!p || !w || n < static_cast<size_t>(kNP)) return prop_fail(CRBM_EINVAL, "need room for 3345 weights");
    const cudaError_t e = cudaMemcpy(w, p->w, kNP * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? CRBM_OK : prop_fail(CRBM_ECUDA, cudaGetErrorString(e));
}

int crbm_proposal_loss_grad(crbm_proposal* p, const int8_t* spins, int32_t L, const int32_t* origins,
                            const float* beta_h, int32_t n, float* loss, float* grad) {
    if (!p || !spins || !origins || !beta_h || n < 1 || L < 4 || (L & 1) || !loss || !grad)
        return prop_fail(CRBM_EINVAL, "bad arguments");
    int rc = ensure_examples(p, n);
    if (rc) return rc;
    std::vector<Example> ex(n);
    for (int e = 0; e < n; ++e) {
        const int8_t* v = spins + static_cast<size_t>(e) * L * L;
        const int bR = ((origins[2 * e] % L) + L) % L, bC = ((origins[2 * e + 1] % L) + L) % L;
        Example& x = ex[e];
        std::memset(&x, 0, sizeof(x));
        for (int pos = 0; pos < crbm::kP * crbm::kP; ++pos) {
            const int R = (bR - 3 + pos / crbm::kP + 2 * L) % L, C = (bC - 3 + pos % crbm::kP + 2 * L) % L;
            const bool in = ((R - bR + L) % L) < crbm::kK && ((C - bC + L) % L) < crbm::kK;
            x.spin[pos] = in ? 0 : v[R * L + C];
            x.inside[pos] = in ? 1 : 0;
        }
        for (int s = 0; s < crbm::kK * crbm::kK; ++s)
            x.target[s] = v[((bR + s / crbm::kK) % L) * L + (bC + s % crbm::kK) % L];
        x.pr = static_cast<uint8_t>((bR + 1) & 1);
        x.pc = static_cast<uint8_t>((bC + 1) & 1);
        x.beta = beta_h[2 * e];
        x.h = beta_h[2 * e + 1];
    }
    cudaError_t e = cudaMemcpy(p->ex, ex.data(), n * sizeof(Example), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->grad, 0, kNP * 4);
    if (e == cudaSuccess) e = cudaMemset(p->loss, 0, 4);
    if (e == cudaSuccess) {
        crbm::k_prop_train<<<(n + 127) / 128, 128>>>(p->wb, p->ex, n, p->grad, p->loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(grad, p->grad, kNP * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(loss, p->loss, 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? CRBM_OK : prop_fail(CRBM_ECUDA, cudaGetErrorString(e));
}

int crbm_proposal_train(crbm_proposal* p, crbm_ctx* ctx, int32_t steps, int32_t batch, float lr,
                        int32_t sweeps_between, float* losses) {
    if (!p || steps < 0 || batch < 1 || batch > (1 << 20) || !(lr > 0.f) || sweeps_between < 0)
        return prop_fail(CRBM_EINVAL, "bad arguments");
    int rc = check_ctx(ctx);
    if (!rc) rc = ensure_chain_params(ctx);
    if (!rc) rc = ensure_examples(p, batch);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    for (int s = 0; s < steps; ++s) {
        if (sweeps_between > 0 && (rc = crbm_sweep(ctx, sweeps_between))) return prop_fail(rc, crbm_last_error(ctx));
        cudaError_t e = cudaSuccess;
        crbm::k_prop_extract<<<(batch + 127) / 128, 128, 0, st>>>(
            ctx->g, ctx->d.v, ctx->d.chain_bh, ctx->n_chains, p->ex, batch,
            static_cast<uint32_t>(p->adam_t), static_cast<uint32_t>(p->seed), static_cast<uint32_t>(p->seed >> 32));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemsetAsync(p->grad, 0, kNP * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(p->loss, 0, 4, st);
        if (e == cudaSuccess) {
            crbm::k_prop_train<<<(batch + 127) / 128, 128, 0, st>>>(p->wb, p->ex, batch, p->grad, p->loss);
            e = cudaGetLastError();
        }
        ++p->adam_t;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, static_cast<float>(p->adam_t));
        const float c2 = 1.f - std::pow(b2, static_cast<float>(p->adam_t));
        if (e == cudaSuccess) {
            crbm::k_prop_adam<<<(kNP + 255) / 256, 256, 0, st>>>(p->w, p->wb, p->m, p->v2, p->grad, kNP, lr,
                                                                  b1, b2, 1e-8f, c1, c2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && losses) {
            e = cudaMemcpyAsync(&losses[s], p->loss, 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
        if (e != cudaSuccess) return prop_fail(CRBM_ECUDA, std::string("train: ") + cudaGetErrorString(e));
    }
    const cudaError_t e = refresh_fragments(p, st);
    if (e == cudaSuccess) cudaStreamSynchronize(st);
    return e == cudaSuccess ? CRBM_OK : prop_fail(CRBM_ECUDA, cudaGetErrorString(e));
}

int crbm_proposal_pass(crbm_ctx* ctx, crbm_proposal* p, int64_t n_passes) {
    if (!p || n_passes < 0) return prop_fail(CRBM_EINVAL, "bad arguments");
    int rc = check_ctx(ctx);
    if (!rc) rc = ensure_chain_params(ctx);
    if (rc) return rc;
    for (int64_t i = 0; i < n_passes; ++i) {
        const cudaError_t e = launch_pass(ctx, p, nullptr);
        if (e != cudaSuccess) return prop_fail(CRBM_ECUDA, std::string("pass: ") + cudaGetErrorString(e));
        ++ctx->passes;
        ++ctx->launches;
    }
    return CRBM_OK;
}

int crbm_sweep_mixed_every(crbm_ctx* ctx, crbm_proposal* p, int64_t n_sweeps, int32_t every) {
    if (!p || n_sweeps < 0 || every < 1) return prop_fail(CRBM_EINVAL, "bad arguments");
    int rc = check_ctx(ctx);
    if (rc) return rc;
    for (int64_t i = 0; i < n_sweeps; i += every) {
        if ((rc = crbm_sweep(ctx, std::min<int64_t>(every, n_sweeps - i)))) return prop_fail(rc, crbm_last_error(ctx));
        if ((rc = crbm_proposal_pass(ctx, p, 1))) return rc;
    }
    return CRBM_OK;
}

int crbm_sweep_mixed(crbm_ctx* ctx, crbm_proposal* p, int64_t n_sweeps) {
    return crbm_sweep_mixed_every(ctx, p, n_sweeps, 1);
}

int crbm_proposal_inspect(crbm_ctx* ctx, crbm_proposal* p, crbm_pass_record* out, size_t n_out) {
    if (!p || !out) return prop_fail(CRBM_EINVAL, "bad arguments");
    int rc = check_ctx(ctx);
    if (!rc) rc = ensure_chain_params(ctx);
    if (rc) return rc;
    const int nb1 = std::max(1, ctx->g.L / 8);
    const size_t need = static_cast<size_t>(ctx->n_words) * nb1 * nb1 * 32;
    if (n_out < need) return prop_fail(CRBM_EINVAL, "output too small");
    static_assert(sizeof(crbm_pass_record) == sizeof(crbm::PassRecord), "record layout");
    crbm::PassRecord* rec = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&rec), need * sizeof(crbm::PassRecord));
    if (e == cudaSuccess) e = launch_pass(ctx, p, rec);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, rec, need * sizeof(crbm::PassRecord), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(rec);
    return e == cudaSuccess ? CRBM_OK : prop_fail(CRBM_ECUDA, cudaGetErrorString(e));
}

int crbm_proposal_stats(crbm_proposal* p, int64_t* proposed, int64_t* accepted) {
    if (!p || !proposed || !accepted) return prop_fail(CRBM_EINVAL, "bad arguments");
    unsigned long long s[2];
    const cudaError_t e = cudaMemcpy(s, p->stats, 16, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return prop_fail(CRBM_ECUDA, cudaGetErrorString(e));
    *proposed = static_cast<int64_t>(s[0]);
    *accepted = static_cast<int64_t>(s[1]);
    return CRBM_OK;
}

const char* crbm_proposal_last_error(void) { return g_prop_error.c_str(); }

}  // extern "C"
