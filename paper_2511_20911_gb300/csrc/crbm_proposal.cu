// Learned block proposal (Metropolis-Hastings block moves mixed with the
// Gibbs sweeps), canonical SS lattice (even L >= 10, periodic).
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
// The pass runs the three convolutions on the tcgen05 tensor cores (bf16
// operands from shared memory, fp32 accumulators in tensor memory).  Four
// independent groups of four warps run on each SM, each working through its
// own work items = (block of the pass, 16 chains of a packed word) with its
// own shared-memory buffers, mbarrier, named barrier and 128 of the SM's 512
// tensor-memory columns; kGroups of them share a persistent CTA (one group
// per CTA measured fastest: four CTAs per SM).  Activations live in an 8 x 8
// frame per chain, stored as "column planes": plane (x, h) holds channels
// 8h .. 8h + 7 of frame column x for the 128 rows (chain, frame row y), 16
// bytes a row.
//  * layer 1 acts on the spin plane alone (its five constant planes are folded
//    into per-position constants added in its epilogue, and b1 + beta w_beta
//    + h w_h enter through constant K columns): one K = 16 MMA per frame
//    column x on a gathered 9-tap operand (M = 128 rows (chain, y), N = 16);
//  * layer 2 is banded: D[(chain, y)][(x, n)] over the six frame columns it
//    needs accumulates, for each tap row dy and input column o, the operand
//    plane o shifted by dy rows (a 3 x 3 convolution's row offset is a
//    shared-memory row offset) against the taps o - x of W2 for the output
//    columns x = o - 2 .. o it feeds (N = 16 .. 48): 24 MMAs into an
//    accumulator zeroed beforehand;
//  * layer 3 (one output channel) is banded the same way with N = the four
//    block columns: its accumulator is the block's logits (18 MMAs);
//  * epilogues read the accumulators with tcgen05.ld, add the bias, apply
//    ReLU and round to bf16 in one conversion, and write the next operand.
// The Metropolis-Hastings step then runs on the CUDA cores: Philox draws of
// the proposed bits against thresholds of q, exact integer dE, log alpha
// with the exact beta, and accepted blocks flipped in place with atomic XOR
// (the two halves of a word are separate items).
//
// Training runs one example per thread in fp32 (bf16-rounded weights and
// activations), back-propagates the binary cross-entropy and updates with
// Adam.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "crbm_context.h"
#include "crbm_device.cuh"
#include "crbm_umma.cuh"

namespace crbm {
namespace {

using namespace dev;

constexpr int kK = 4;              // block side
constexpr int kP = kK + 6;         // patch side (10)
constexpr int kS1 = kK + 4;        // layer-1 output side (8)
constexpr int kS2 = kK + 2;        // layer-2 output side (6)
constexpr int kNP = 3345;          // parameters
constexpr uint32_t kTagOffset = 8u, kTagBits = 9u, kTagAccept = 13u, kTagExample = 14u;

// Parameter offsets (W1[16][6][3][3], b1, W2[16][16][3][3], b2, W3[16][3][3], b3).
constexpr int oW1 = 0, oB1 = 864, oW2 = 880, oB2 = 3184, oW3 = 3200, oB3 = 3344;

// Layer 1 on the five constant planes (block mask, row and column parity,
// beta, h) is linear in them and the same for every chain of a pass, so it is
// folded out of the convolution: per output position and channel a constant
// for each parity of the patch's first row and column ([4][64][16]), and the
// tap sums of the beta and h kernels ([2][16]).  Only the spin plane remains
// a convolution (K = 9 taps).
constexpr int kC1Pos = 4 * kS1 * kS1 * 16, kC1 = kC1Pos + 2 * 16;

// ---- tensor-core pass geometry
constexpr int kPassThreads = 128;              // one group (warpgroup): warp w reads TMEM lanes 32 (w % 4) ..
constexpr int kGroups = 1;                     // groups per CTA (2 or 4 measured slower)
constexpr int kCtasPerSm = 4 / kGroups;        // four groups per SM: 4 x 128 tensor-memory columns
constexpr int kCtaThreads = kGroups * kPassThreads;
constexpr int kItemChains = 16;                // chains of one work item (half a packed word)
constexpr int kFrame = 8;                      // every layer in an 8 x 8 frame per chain
constexpr int kTmemCols = 128;                 // per group; the CTA allocates kGroups x 128 = 512
constexpr int kPlaneRows = 136;                // 128 rows (chain, y) + rows read by the dy = 1, 2 shifts
constexpr int kPlane = kPlaneRows * 16;        // bytes of one column plane (x, h)
// Layer-1 operand (gathered): rows (x, chain, y), K = 9 spin taps, then 1,
// beta, beta, h, h, 0, 0: two planes of 1024 rows.
constexpr int kA0Plane = 1024 * 16;
// B operands (bf16, K-major, element offsets): B1 [n 16][k 16]; layer-2 taps
// per dy: [h 2][row 3 * 16][8] with row = block j * 16 + n, block j = tap
// column 2 - j; layer-3 bands per dy: [h 2][row 24][8], row 7 - dx = tap
// column dx, zero rows elsewhere.
constexpr int kZ2Rows = 3 * 16, kZ3Rows = 24;
constexpr int kB1 = 0, kZ2 = 256, kZ3 = kZ2 + 3 * 2 * kZ2Rows * 8, kBElems = kZ3 + 3 * 2 * kZ3Rows * 8;
constexpr uint32_t kIdesc1 = umma::idesc_bf16_f32(128, 16);
constexpr uint32_t kIdesc3 = umma::idesc_bf16_f32(128, 16);
// Shared memory of the pass (bytes): the B operands (shared by the groups),
// then one region per group.  A group's X holds, in turn, layer 1's gathered
// operand, layer 1's output planes (layer 2's operand), layer 2's output
// planes (layer 3's operand) and the block's logits.  Item data are
// double-buffered (the next item's are fetched during this one); the folded
// layer-1 constants of the item are fetched at its start.
constexpr int kSmB = 0;
constexpr int kSmG0 = ((kBElems * 2 + 127) / 128) * 128;   // first group region
constexpr int kSmX = 0, kSmXBytes = 8 * 2 * kPlane;        // 34816 >= 2 * kA0Plane (offsets in a group)
constexpr int kItemBytes = 104 * 4 + kItemChains * 8 * 4;  // patch [100](+4), chain_bh [16][4], Q.4 [16][4]
constexpr int kC1Stride = 20;                              // floats per (x, y) row of staged constants
constexpr int kC1Bytes = 64 * kC1Stride * 4;
constexpr int kSmItem = kSmX + kSmXBytes;
constexpr int kSmC1 = kSmItem + 2 * kItemBytes;
constexpr int kSmBar = kSmC1 + kC1Bytes, kSmGroup = kSmBar + 16;
constexpr int kSmBytes = kSmG0 + kGroups * kSmGroup + 16;  // + the tensor-memory address slot
static_assert(kSmXBytes >= 2 * kA0Plane, "layer-1 operand fits in X");
static_assert(kSmG0 % 128 == 0 && kSmGroup % 16 == 0 && kSmItem % 16 == 0 && kSmC1 % 16 == 0 && kSmBar % 8 == 0,
              "alignment");
static_assert(kSmBytes * kCtasPerSm <= 226 * 1024, "kCtasPerSm CTAs per SM");
constexpr int kWaitTries = 1 << 22;            // mbarrier polls before the pass gives up

// Per (word, block, lane) record of a pass run in inspection mode: the
// logits, the proposed and current block bits, the exact dE, log alpha and
// the proposal thresholds.
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
    const uint4* bmat;        // [kBElems / 8] B operands (bf16, canonical layout)
    const float* bias;        // b2[16], b3
    const float* c1;          // folded layer-1 constants [kC1]
    const float* chain_bh;    // [chains][4] beta, h (bf16-rounded net inputs), beta (fp32), 0
    const int32_t* chain_q;   // [chains][3] Q.4 J, J', h
    unsigned long long* stats;  // {proposed, accepted, timeouts}
    uint32_t key0, key1;
    uint32_t pass;
    int nb1, spacing;         // blocks per side, block spacing
    int n_items;              // blocks x half-words
};

// Start fetching item `item`'s patch words and chain data into buffer `buf`
// (cp.async: complete at the next cp.async.wait).
__device__ __forceinline__ void prefetch_item(const PassArgs& a, uint8_t* sm, int buf, int item, int bR0, int bC0,
                                              int tid) {
    const int L = a.g.L, n_blocks = a.nb1 * a.nb1;
    const int b = item % n_blocks, hw = item / n_blocks, word = hw >> 1, half = hw & 1;
    const int bR = (bR0 + a.spacing * (b / a.nb1)) % L, bC = (bC0 + a.spacing * (b % a.nb1)) % L;
    uint8_t* ib = sm + kSmItem + buf * kItemBytes;
    if (tid < kP * kP) {
        const int R = (bR - 3 + tid / kP + 2 * L) % L, C = (bC - 3 + tid % kP + 2 * L) % L;
        const uint32_t* src = a.v + static_cast<size_t>(word) * a.g.N + R * L + C;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(umma::smem_addr(ib + 4 * tid)), "l"(src)
                     : "memory");
    } else if (tid < kP * kP + kItemChains) {
        const int c = tid - kP * kP, chain = word * 32 + half * 16 + c;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(umma::smem_addr(ib + 416 + 16 * c)),
                     "l"(a.chain_bh + 4 * static_cast<size_t>(chain))
                     : "memory");
        for (int j = 0; j < 3; ++j)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(umma::smem_addr(ib + 672 + 16 * c + 4 * j)),
                         "l"(a.chain_q + 3 * static_cast<size_t>(chain) + j)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Start fetching the folded layer-1 constants of parity variant `var`: row
// (x, y) of 16 floats at stride kC1Stride (c1 is stored [var][y * 8 + x][16]).
__device__ __forceinline__ void fetch_c1(const PassArgs& a, uint8_t* sm, int var, int tid) {
    uint8_t* cb = sm + kSmC1;
    for (int q = tid; q < 64 * 4; q += kPassThreads) {
        const int row = q >> 2, x = row >> 3, y = row & 7;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(
                         umma::smem_addr(cb + (row * kC1Stride + 4 * (q & 3)) * 4)),
                     "l"(a.c1 + (var * 64 + y * 8 + x) * 16 + 4 * (q & 3))
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Group barrier: the 128 threads of group g (named barrier 1 + g).
__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(kPassThreads) : "memory");
}

// One pass of MH block moves; persistent CTAs of kGroups groups of four
// warps, each group taking items (block b, half-word hw) in turn.
__global__ void __launch_bounds__(kCtaThreads, kCtasPerSm) k_prop_pass(const __grid_constant__ PassArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_all[];
    const int L = a.g.L, N = a.g.N;
    const int g = threadIdx.x / kPassThreads;  // group
    const int tid = threadIdx.x % kPassThreads, lane = tid & 31, warp = tid >> 5;  // within the group
    const int n_blocks = a.nb1 * a.nb1;
    uint8_t* sm = smem_all + kSmG0 + g * kSmGroup;  // the group's region
    uint8_t* X = sm + kSmX;
    uint16_t* Bs = reinterpret_cast<uint16_t*>(smem_all + kSmB);
    const uint32_t bar = umma::smem_addr(sm + kSmBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_all + kSmG0 + kGroups * kSmGroup);
    __shared__ int s_fail[kGroups];
    __shared__ unsigned long long s_stats[2];  // proposed, accepted by this CTA
    // the block's logits in X after layer 3: site s of chain c at (s & 1) * 256 + 8 c + (s >> 1), so
    // that the Metropolis-Hastings lanes (chain c, part p: sites 2 p, 2 p + 1) read them without
    // bank conflicts
    float* logit = reinterpret_cast<float*>(X);

    // set-up: the tensor memory first (a CTA of a kernel that allocates tensor memory starts only
    // after the SM's previous one gave up its allocation permit), B operands, the never-written tail
    // of each X (rows past 128 of the last plane, read by the dy = 1, 2 shifts), mbarriers
    if (threadIdx.x < 32) umma::tmem_alloc(umma::smem_addr(tslot), kGroups * kTmemCols);
    for (int x = threadIdx.x; x < kBElems / 8; x += kCtaThreads) reinterpret_cast<uint4*>(Bs)[x] = a.bmat[x];
    for (int x = 2 * kA0Plane / 16 + tid; x < kSmXBytes / 16; x += kPassThreads)
        reinterpret_cast<uint4*>(X)[x] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        umma::mbar_init(bar, 1);
        s_fail[g] = 0;
    }
    if (threadIdx.x < 2) s_stats[threadIdx.x] = 0ull;
    const U4 off = philox(a.pass, 0u, 0u, kTagOffset, a.key0, a.key1);
    const int bR0 = static_cast<int>(off.x % static_cast<uint32_t>(L));
    const int bC0 = static_cast<int>(off.y % static_cast<uint32_t>(L));
    const int item0 = blockIdx.x * kGroups + g, stride = gridDim.x * kGroups;
    if (item0 < a.n_items) prefetch_item(a, sm, 0, item0, bR0, bC0, tid);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot + static_cast<uint32_t>(kTmemCols * g);
    const uint32_t xs = umma::smem_addr(X), bs = umma::smem_addr(Bs);
    uint32_t phase = 0;
    // this thread's accumulator lane 32 warp + lane = row (chain cl, frame row y)
    const int my_row = 32 * warp + lane, my_c = my_row >> 3, my_y = my_row & 7;
    const uint32_t tl = tmem + (static_cast<uint32_t>(32 * warp) << 16);
    float b2[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) b2[n] = a.bias[n];
    const float b3 = a.bias[16];
    bool ok = true;
    int buf = 0;

    for (int item = item0; item < a.n_items && ok; item += stride, buf ^= 1) {
        const int b = item % n_blocks, hw = item / n_blocks;
        const int word = hw >> 1, half = hw & 1;
        const int bR = (bR0 + a.spacing * (b / a.nb1)) % L, bC = (bC0 + a.spacing * (b % a.nb1)) % L;
        const uint8_t* ib = sm + kSmItem + buf * kItemBytes;
        const uint32_t* pw = reinterpret_cast<const uint32_t*>(ib);               // [100] patch words
        const float* cbh = reinterpret_cast<const float*>(ib + 416);            // [16][4] chain_bh
        const int32_t* cq = reinterpret_cast<const int32_t*>(ib + 672);         // [16][4] Q.4 J, J', h
        const float* c1s = reinterpret_cast<const float*>(sm + kSmC1);
        asm volatile("cp.async.wait_all;" ::: "memory");
        group_sync(g);
        fetch_c1(a, sm, ((bR + 1) & 1) * 2 + ((bC + 1) & 1), tid);
        if (item + stride < a.n_items)   // the next item's data, during this one
            prefetch_item(a, sm, buf ^ 1, item + stride, bR0, bC0, tid);
        else
            asm volatile("cp.async.commit_group;" ::: "memory");
        // ---- layer-1 operand: rows x * 128 + (chain c, y) = tid, K = 9 spin taps (0 inside
        // the block), then 1, beta, beta, h, h (the constant columns), 0, 0
        {
            const int c = my_c, y = my_y, bit = half * 16 + c;
            uint32_t sp[3][kP];  // bf16 spin values of patch rows y .. y + 2
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int Xc = 0; Xc < kP; ++Xc) {
                    const int Y = y + dy;
                    const uint32_t keep = (Y >= 3 && Y < 3 + kK && Xc >= 3 && Xc < 3 + kK) ? 0u : 0xFFFFu;
                    sp[dy][Xc] = (0xBF80u ^ (((pw[Y * kP + Xc] >> bit) & 1u) << 15)) & keep;
                }
            const uint32_t beta_b = __float_as_uint(cbh[4 * c]) >> 16, h_b = __float_as_uint(cbh[4 * c + 1]) >> 16;
            const uint4 k1 = make_uint4(0u, beta_b | (beta_b << 16), h_b | (h_b << 16), 0u);
#pragma unroll
            for (int x = 0; x < kFrame; ++x) {
                const int r = x * 128 + my_row;
                reinterpret_cast<uint4*>(X + r * 16)[0] =
                    make_uint4(sp[0][x] | (sp[0][x + 1] << 16), sp[0][x + 2] | (sp[1][x] << 16),
                               sp[1][x + 1] | (sp[1][x + 2] << 16), sp[2][x] | (sp[2][x + 1] << 16));
                uint4 q = k1;
                q.x = sp[2][x + 2] | (0x3F80u << 16);
                reinterpret_cast<uint4*>(X + kA0Plane + r * 16)[0] = q;
            }
        }
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this item's constants (not the next item's data)
        umma::fence_async_smem();
        umma::fence_before_sync();
        group_sync(g);
        if (tid == 0) {  // layer 1: one K = 16 MMA per frame column x (accumulator columns 16 x)
            umma::fence_after_sync();
            for (int x = 0; x < kFrame; ++x)
                umma::mma(tmem + 16 * x, umma::desc(xs + 2048 * x, kA0Plane, 128), umma::desc(bs + 2 * kB1, 256, 128),
                          kIdesc1, 0u);
            umma::commit(bar);
        }
        if (!umma::mbar_wait(bar, phase, kWaitTries)) s_fail[g] = 1;
        phase ^= 1u;
        umma::fence_after_sync();
        // ---- epilogue 1: + folded constants, ReLU, bf16 -> column planes (x, h), row my_row
        for (int x = 0; x < kFrame; x += 2) {
            uint32_t r0[16], r1[16];
            umma::tmem_ld16(tl + 16 * x, r0);
            umma::tmem_ld16(tl + 16 * (x + 1), r1);
            umma::tmem_ld_wait();
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const uint32_t* r = t ? r1 : r0;
                const float4* cr = reinterpret_cast<const float4*>(c1s + ((x + t) * 8 + my_y) * kC1Stride);
                uint32_t o[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 f = cr[q];
                    o[2 * q] = umma::relu_bf16x2(__uint_as_float(r[4 * q]) + f.x, __uint_as_float(r[4 * q + 1]) + f.y);
                    o[2 * q + 1] =
                        umma::relu_bf16x2(__uint_as_float(r[4 * q + 2]) + f.z, __uint_as_float(r[4 * q + 3]) + f.w);
                }
                uint8_t* pl = X + 2 * (x + t) * kPlane + my_row * 16;
                reinterpret_cast<uint4*>(pl)[0] = make_uint4(o[0], o[1], o[2], o[3]);
                reinterpret_cast<uint4*>(pl + kPlane)[0] = make_uint4(o[4], o[5], o[6], o[7]);
            }
        }
#pragma unroll
        for (int x = 0; x < 6; ++x) umma::tmem_zero16(tl + 16 * x);  // layer 2 accumulates from zero
        umma::tmem_st_wait();
        umma::fence_async_smem();
        umma::fence_before_sync();
        group_sync(g);
        if (s_fail[g]) {
            ok = false;
            break;
        }
        if (tid == 0) {  // layer 2: 3 tap rows x 8 input columns o, output columns o - 2 .. o
            umma::fence_after_sync();
            for (int dy = 0; dy < 3; ++dy)
                for (int o = 0; o < kFrame; ++o) {
                    const int lo = o < 2 ? 0 : o - 2, hi = o < 5 ? o : 5;
                    umma::mma(tmem + 16 * lo, umma::desc(xs + 2 * o * kPlane + 16 * dy, kPlane, 128),
                              umma::desc(bs + 2 * (kZ2 + dy * 2 * kZ2Rows * 8) + (2 - o + lo) * 256, kZ2Rows * 16, 128),
                              umma::idesc_bf16_f32(128, 16 * (hi - lo + 1)), 1u);
                }
            umma::commit(bar);
        }
        if (!umma::mbar_wait(bar, phase, kWaitTries)) s_fail[g] = 1;
        phase ^= 1u;
        umma::fence_after_sync();
        // ---- epilogue 2: + b2, ReLU, bf16 -> column planes 0..5 (layer 3's operand)
        for (int x = 0; x < 6; x += 2) {
            uint32_t r0[16], r1[16];
            umma::tmem_ld16(tl + 16 * x, r0);
            umma::tmem_ld16(tl + 16 * (x + 1), r1);
            umma::tmem_ld_wait();
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const uint32_t* r = t ? r1 : r0;
                uint32_t o[8];
#pragma unroll
                for (int n = 0; n < 8; ++n)
                    o[n] = umma::relu_bf16x2(__uint_as_float(r[2 * n]) + b2[2 * n],
                                             __uint_as_float(r[2 * n + 1]) + b2[2 * n + 1]);
                uint8_t* pl = X + 2 * (x + t) * kPlane + my_row * 16;
                reinterpret_cast<uint4*>(pl)[0] = make_uint4(o[0], o[1], o[2], o[3]);
                reinterpret_cast<uint4*>(pl + kPlane)[0] = make_uint4(o[4], o[5], o[6], o[7]);
            }
        }
        umma::fence_async_smem();
        umma::fence_before_sync();
        group_sync(g);
        if (s_fail[g]) {
            ok = false;
            break;
        }
        if (tid == 0) {  // layer 3: banded, 3 tap rows x 6 input columns, N = the block's 4 columns (+ 12)
            umma::fence_after_sync();
            for (int dy = 0; dy < 3; ++dy)
                for (int o = 0; o < 6; ++o)
                    umma::mma(tmem, umma::desc(xs + 2 * o * kPlane + 16 * dy, kPlane, 128),
                              umma::desc(bs + 2 * (kZ3 + dy * 2 * kZ3Rows * 8) + (7 - o) * 16, kZ3Rows * 16, 128),
                              kIdesc3, (dy | o) ? 1u : 0u);
            umma::commit(bar);
        }
        if (!umma::mbar_wait(bar, phase, kWaitTries)) s_fail[g] = 1;
        phase ^= 1u;
        umma::fence_after_sync();
        // ---- epilogue 3: rows y < 4 hold the logits of block sites (y, 0..3)
        {
            uint32_t r[4];
            umma::tmem_ld4(tl, r);
            umma::tmem_ld_wait();
            if (my_y < kK) {
#pragma unroll
                for (int x = 0; x < kK; ++x)
                    logit[(x & 1) * 256 + 8 * my_c + (my_y * kK + x) / 2] = __uint_as_float(r[x]) + b3;
            }
        }
        umma::fence_before_sync();
        group_sync(g);
        if (s_fail[g]) {
            ok = false;
            break;
        }
        // ---- Metropolis-Hastings: warp w takes chains 4 w .. 4 w + 3, eight lanes per chain,
        // lane part p the sites 2 p and 2 p + 1 (words (2 p) % 4 and (2 p + 1) % 4 of Philox
        // call p / 2).  A lane forms its sites' thresholds, proposals and shares of
        // log q(current) - log q(proposed), and of the exact dE the terms linear in the block's
        // spins (bonds to spins outside the block, and the field); the chain's eight lanes sum
        // them by shuffles, add the bonds inside the block from the current and proposed bit
        // masks, and run the test; accepted sites flip with one atomic XOR per site and warp.
        {
            const int c = 4 * warp + (lane >> 3), part = lane & 7;
            const int chain = word * 32 + half * 16 + c;
            const int cbit = half * 16 + c;
            const uint32_t cell_id = static_cast<uint32_t>(b);
            const int qJ = cq[4 * c], qJp = cq[4 * c + 1], qh = cq[4 * c + 2];
            const U4 u = philox(cell_id, a.pass, static_cast<uint32_t>(chain), kTagBits + (part >> 1), a.key0, a.key1);
            float lq = 0.f;
            int de = 0;
            uint32_t bits = 0u;
            auto spin_at = [&](int pr, int pc) -> int { return ((pw[pr * kP + pc] >> cbit) & 1u) ? 1 : -1; };
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int s = 2 * part + j;
                const int ar = s / kK, ac = s % kK;
                const bool xc = (pw[(3 + ar) * kP + 3 + ac] >> cbit) & 1u;
                const float lg = logit[j * 256 + 8 * c + part];
                const float q = __fdividef(1.f, 1.f + __expf(-lg));
                float tf = q * 4294967296.f;
                tf = fminf(fmaxf(tf, 1.f), 4294967040.f);
                const uint32_t thr = static_cast<uint32_t>(tf);
                // log p and log (1 - p) of p = thr / 2^32, from the exact integers thr and 2^32 - thr
                const float lp = __logf(static_cast<float>(thr)) - 22.18070977791825f;
                const float lm = __logf(static_cast<float>(0u - thr)) - 22.18070977791825f;
                const bool xp = pick(u, s & 3) < thr;
                lq += (xc ? lp : lm) - (xp ? lp : lm);
                bits |= (xc ? 1u : 0u) << s | (xp ? 1u : 0u) << (16 + s);
                // field on site s from outside the block (1/16 units): J to its outside neighbours,
                // J' to an outside dimer partner, -h
                int f = -qh;
                if (ac == 0) f += qJ * spin_at(3 + ar, 2);
                if (ac == kK - 1) f += qJ * spin_at(3 + ar, 3 + kK);
                if (ar == 0) f += qJ * spin_at(2, 3 + ac);
                if (ar == kK - 1) f += qJ * spin_at(3 + kK, 3 + ac);
                const int R = bR + ar, C = bC + ac;
                const int pr = ar + ((C & 1) ? -1 : 1), pc = ac + ((R & 1) ? -1 : 1);  // the dimer partner
                if (pr < 0 || pr >= kK || pc < 0 || pc >= kK) f += qJp * spin_at(3 + pr, 3 + pc);
                de += ((xp ? 1 : -1) - (xc ? 1 : -1)) * f;
                if (a.rec) {  // inspection: this lane's sites of the record
                    PassRecord* r = a.rec + (static_cast<size_t>(word) * n_blocks + b) * 32 + cbit;
                    r->logit[s] = lg;
                    r->thr[s] = thr;
                }
            }
            // the chain's eight lanes: sums in a fixed tree order
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                lq += __shfl_xor_sync(0xffffffffu, lq, o);
                de += __shfl_xor_sync(0xffffffffu, de, o);
                bits |= __shfl_xor_sync(0xffffffffu, bits, o);
            }
            const uint32_t cb = bits & 0xFFFFu, nb = bits >> 16;
            // bonds inside the block: s_i s_j = 1 - 2 [bits differ], counted once per pair
            // (right neighbour, lower neighbour, the dimer partner of the upper site)
            uint32_t d5 = 0u, d3 = 0u;  // sites whose partner is site + 5 / site + 3
#pragma unroll
            for (int s = 0; s < 12; ++s) {
                const int ar = s / kK, ac = s % kK, R = bR + ar, C = bC + ac;
                if (!(C & 1)) {  // the partner lies one row down
                    if (!(R & 1) && ac < kK - 1) d5 |= 1u << s;
                    if ((R & 1) && ac > 0) d3 |= 1u << s;
                }
            }
            auto diffs = [&](uint32_t x) {
                return static_cast<int>(__popc((x ^ (x >> 1)) & 0x7777u) + __popc((x ^ (x >> 4)) & 0x0FFFu));
            };
            auto ddiffs = [&](uint32_t x) { return static_cast<int>(__popc(((x ^ (x >> 5)) & d5) | ((x ^ (x >> 3)) & d3))); };
            de += 2 * qJ * (diffs(cb) - diffs(nb)) + 2 * qJp * (ddiffs(cb) - ddiffs(nb));
            const float beta = cbh[4 * c + 2];  // the exact beta: the MH test targets exp(-beta H)
            const float log_alpha = -beta * static_cast<float>(de) * 0.0625f + lq;
            uint32_t ua = 0u;
            if (part == 0) ua = philox(cell_id, a.pass, static_cast<uint32_t>(chain), kTagAccept, a.key0, a.key1).x;
            ua = __shfl_sync(0xffffffffu, ua, lane & 24);
            const bool accept =
                log_alpha >= 0.f || static_cast<float>(ua >> 8) * 5.9604644775390625e-08f < __expf(log_alpha);
            if (a.rec) {
                if (part == 0) {
                    PassRecord* r = a.rec + (static_cast<size_t>(word) * n_blocks + b) * 32 + cbit;
                    r->dE = de;
                    r->cur_bits = cb;
                    r->new_bits = nb;
                    r->log_alpha = log_alpha;
                    r->bR = bR;
                    r->bC = bC;
                }
            } else {
                const uint32_t flip = accept ? (cb ^ nb) : 0u;
                uint32_t my_fm = 0u;  // lane s < 16: the warp's chains whose site s flips
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    my_fm |= ((__shfl_sync(0xffffffffu, flip, 8 * j) >> (lane & 15)) & 1u) << j;
                if (lane < 16 && my_fm) {
                    const int R = (bR + lane / kK) % L, C = (bC + lane % kK) % L;
                    atomicXor(a.v + static_cast<size_t>(word) * N + R * L + C, my_fm << (16 * half + 4 * warp));
                }
                const uint32_t am = __ballot_sync(0xffffffffu, accept && part == 0);
                if (lane == 0) {
                    atomicAdd(&s_stats[0], 4ull);
                    atomicAdd(&s_stats[1], static_cast<unsigned long long>(__popc(am)));
                }
            }
        }
        group_sync(g);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // a timed-out wait: record it, give the tensor cores one more bounded wait
    // for the group's MMAs in flight, then (every group done) free the tensor memory
    if (!ok) {
        if (tid == 0) atomicAdd(&a.stats[2], 1ull);
        umma::mbar_wait(bar, phase ^ 1u, kWaitTries);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        umma::fence_after_sync();
        umma::tmem_dealloc(*tslot, kGroups * kTmemCols);
    }
    if (threadIdx.x == 32 && s_stats[0]) {
        atomicAdd(&a.stats[0], s_stats[0]);
        atomicAdd(&a.stats[1], s_stats[1]);
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

// Forward + backward of the mean binary cross-entropy in fp32 on
// bf16-rounded weights and activations (the roundings pass gradients straight
// through).  A CTA takes kTrainEx examples in turn, with the weights, its
// gradient sums and one example's activations and deltas in shared memory;
// within an example a thread takes output positions (forward, deltas) or
// parameters (weight gradients), so every gradient sum has one owner thread
// and the CTA adds its sums to grad with one atomic per parameter.  grad and
// loss accumulate.
constexpr int kTrainEx = 16, kTrainThreads = 128;
__global__ void __launch_bounds__(kTrainThreads) k_prop_train(const float* __restrict__ w, const Example* ex, int n,
                                                              float* grad, float* loss) {
    __shared__ float sW[kNP], sG[kNP];
    __shared__ float s_in[6][kP * kP], s_a1[16][kS1 * kS1], s_a2[16][kS2 * kS2];
    __shared__ float s_d1[16][kS1 * kS1], s_d2[16][kS2 * kS2], s_dl[kK * kK];
    __shared__ float s_loss;
    const int tid = threadIdx.x;
    for (int i = tid; i < kNP; i += kTrainThreads) {
        sW[i] = w[i];
        sG[i] = 0.f;
    }
    if (tid == 0) s_loss = 0.f;
    const float inv = 1.f / (static_cast<float>(n) * kK * kK);
    const int e_end = min(n, (blockIdx.x + 1) * kTrainEx);
    for (int e = blockIdx.x * kTrainEx; e < e_end; ++e) {
        const Example& x = ex[e];
        __syncthreads();  // the previous example's buffers are free
        for (int pos = tid; pos < kP * kP; pos += kTrainThreads) {
            s_in[0][pos] = x.spin[pos];
            s_in[1][pos] = x.inside[pos];
            s_in[2][pos] = static_cast<float>((x.pr + pos / kP) & 1);
            s_in[3][pos] = static_cast<float>((x.pc + pos % kP) & 1);
            s_in[4][pos] = x.beta;
            s_in[5][pos] = x.h;
        }
        __syncthreads();
        for (int i = tid; i < 16 * kS1 * kS1; i += kTrainThreads) {  // layer 1
            const int o = i / (kS1 * kS1), p = i % (kS1 * kS1), y = p / kS1, xx = p % kS1;
            float acc = sW[oB1 + o];
            for (int c = 0; c < 6; ++c)
#pragma unroll
                for (int t = 0; t < 9; ++t) acc += sW[oW1 + (o * 6 + c) * 9 + t] * s_in[c][(y + t / 3) * kP + xx + t % 3];
            s_a1[o][p] = bf16r(fmaxf(acc, 0.f));
        }
        __syncthreads();
        for (int i = tid; i < 16 * kS2 * kS2; i += kTrainThreads) {  // layer 2
            const int o = i / (kS2 * kS2), p = i % (kS2 * kS2), y = p / kS2, xx = p % kS2;
            float acc = sW[oB2 + o];
            for (int c = 0; c < 16; ++c)
#pragma unroll
                for (int t = 0; t < 9; ++t) acc += sW[oW2 + (o * 16 + c) * 9 + t] * s_a1[c][(y + t / 3) * kS1 + xx + t % 3];
            s_a2[o][p] = bf16r(fmaxf(acc, 0.f));
        }
        __syncthreads();
        if (tid < 32) {  // layer 3 and the loss: lanes 0 .. 15 take the block sites
            float l = 0.f;
            if (tid < kK * kK) {
                const int y = tid / kK, xx = tid % kK;
                float acc = sW[oB3];
                for (int c = 0; c < 16; ++c)
#pragma unroll
                    for (int t = 0; t < 9; ++t) acc += sW[oW3 + c * 9 + t] * s_a2[c][(y + t / 3) * kS2 + xx + t % 3];
                const float yv = x.target[tid] > 0 ? 1.f : 0.f;
                l = (acc > 0.f ? acc + log1pf(__expf(-acc)) : log1pf(__expf(acc))) - yv * acc;
                s_dl[tid] = (1.f / (1.f + __expf(-acc)) - yv) * inv;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
            if (tid == 0) s_loss += l;
        }
        __syncthreads();
        // layer 3: weight gradients and the deltas of layer 2's outputs (zero where ReLU was off)
        for (int i = tid; i < 16 * 9; i += kTrainThreads) {
            const int c = i / 9, t = i % 9;
            float g = 0.f;
#pragma unroll
            for (int p = 0; p < kK * kK; ++p) g += s_dl[p] * s_a2[c][(p / kK + t / 3) * kS2 + p % kK + t % 3];
            sG[oW3 + i] += g;
        }
        if (tid == 0) {
            float g = 0.f;
            for (int p = 0; p < kK * kK; ++p) g += s_dl[p];
            sG[oB3] += g;
        }
        for (int i = tid; i < 16 * kS2 * kS2; i += kTrainThreads) {
            const int c = i / (kS2 * kS2), q = i % (kS2 * kS2), qy = q / kS2, qx = q % kS2;
            float d = 0.f;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int py = qy - t / 3, px = qx - t % 3;
                if (py >= 0 && py < kK && px >= 0 && px < kK) d += s_dl[py * kK + px] * sW[oW3 + c * 9 + t];
            }
            s_d2[c][q] = s_a2[c][q] > 0.f ? d : 0.f;
        }
        __syncthreads();
        // layer 2: weight and bias gradients, the deltas of layer 1's outputs
        for (int i = tid; i < 16 * 16 * 9; i += kTrainThreads) {
            const int o = i / 144, c = (i / 9) % 16, t = i % 9;
            float g = 0.f;
#pragma unroll 4
            for (int p = 0; p < kS2 * kS2; ++p) g += s_d2[o][p] * s_a1[c][(p / kS2 + t / 3) * kS1 + p % kS2 + t % 3];
            sG[oW2 + i] += g;
        }
        if (tid < 16) {
            float g = 0.f;
            for (int p = 0; p < kS2 * kS2; ++p) g += s_d2[tid][p];
            sG[oB2 + tid] += g;
        }
        for (int i = tid; i < 16 * kS1 * kS1; i += kTrainThreads) {
            const int c = i / (kS1 * kS1), q = i % (kS1 * kS1), qy = q / kS1, qx = q % kS1;
            float d = 0.f;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int py = qy - t / 3, px = qx - t % 3;
                if (py >= 0 && py < kS2 && px >= 0 && px < kS2)
                    for (int o = 0; o < 16; ++o) d += s_d2[o][py * kS2 + px] * sW[oW2 + (o * 16 + c) * 9 + t];
            }
            s_d1[c][q] = s_a1[c][q] > 0.f ? d : 0.f;
        }
        __syncthreads();
        // layer 1: weight and bias gradients
        for (int i = tid; i < 16 * 6 * 9; i += kTrainThreads) {
            const int o = i / 54, c = (i / 9) % 6, t = i % 9;
            float g = 0.f;
#pragma unroll 4
            for (int p = 0; p < kS1 * kS1; ++p) g += s_d1[o][p] * s_in[c][(p / kS1 + t / 3) * kP + p % kS1 + t % 3];
            sG[oW1 + i] += g;
        }
        if (tid < 16) {
            float g = 0.f;
            for (int p = 0; p < kS1 * kS1; ++p) g += s_d1[tid][p];
            sG[oB1 + tid] += g;
        }
    }
    __syncthreads();
    for (int i = tid; i < kNP; i += kTrainThreads) atomicAdd(&grad[i], sG[i]);
    if (tid == 0) atomicAdd(loss, s_loss * inv);
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

// The tensor-core B operands and biases from the bf16-rounded weights (on the
// device, so they follow the trained weights without a host round trip), in
// the layout described at kB1 / kZ2 / kZ3.  B1 (element (n, k) at (k / 8) *
// 128 + n * 8 + k % 8): layer 1 on the spin plane (k < 9: tap k), then the
// constant columns b1 (k = 9) and the tap sums of the beta and h kernels as
// bf16 hi + lo pairs (k = 10, 11 and 12, 13).
__global__ void k_prop_operands(const float* wb, uint16_t* bmat, float* bias) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 17) bias[i] = i < 16 ? wb[oB2 + i] : wb[oB3];
    if (i >= kBElems) return;
    float v = 0.f;
    if (i < kZ2) {
        const int n = (i % 128) / 8, k = (i / 128) * 8 + i % 8;
        if (k < 9) {
            v = wb[oW1 + n * 6 * 9 + k];
        } else if (k == 9) {
            v = wb[oB1 + n];
        } else if (k <= 13) {
            const int ch = k < 12 ? 4 : 5;
            float sum = 0.f;
            for (int tap = 0; tap < 9; ++tap) sum += wb[oW1 + (n * 6 + ch) * 9 + tap];
            const float hi = bf16r(sum);
            v = ((k - 10) & 1) ? bf16r(sum - hi) : hi;
        }
    } else if (i < kZ3) {  // layer-2 taps: [dy][h][row j * 16 + n][8], tap column 2 - j
        const int e = i - kZ2, dy = e / (2 * kZ2Rows * 8), r = e % (2 * kZ2Rows * 8);
        const int h = r / (kZ2Rows * 8), row = (r % (kZ2Rows * 8)) / 8, ch = h * 8 + r % 8;
        const int j = row / 16, n = row % 16, dx = 2 - j;
        v = wb[oW2 + (n * 16 + ch) * 9 + dy * 3 + dx];
    } else {  // layer-3 bands: [dy][h][row][8], row 7 - dx
        const int e = i - kZ3, dy = e / (2 * kZ3Rows * 8), r = e % (2 * kZ3Rows * 8);
        const int h = r / (kZ3Rows * 8), row = (r % (kZ3Rows * 8)) / 8, ch = h * 8 + r % 8;
        const int dx = 7 - row;
        if (dx >= 0 && dx <= 2) v = wb[oW3 + ch * 9 + dy * 3 + dx];
    }
    bmat[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
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
    uint16_t* bmat = nullptr;  // tensor-core B operands (bf16)
    float* bias = nullptr;     // b2, b3
    float* c1 = nullptr;     // folded layer-1 constants
    unsigned long long* stats = nullptr;
    crbm::Example* ex = nullptr;
    int ex_cap = 0;
    int64_t adam_t = 0;
    uint64_t seed = 0;
    int pass_sms = 0, pass_dev = -1;  // SM count of the device the pass kernel was set up on
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
    crbm::k_prop_operands<<<(crbm::kBElems + 127) / 128, 128, 0, st>>>(p->wb, p->bmat, p->bias);
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
    if (e != cudaSuccess) {  // leave neither buffer behind: the next call builds both again
        cudaFree(ctx->d.chain_bh);
        cudaFree(ctx->d.chain_q);
        ctx->d.chain_bh = nullptr;
        ctx->d.chain_q = nullptr;
        cudaGetLastError();  // an allocation error is not sticky; clear it for later launch checks
        return prop_fail(CRBM_ECUDA, std::string("chain parameters: ") + cudaGetErrorString(e));
    }
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
    if (cudaMalloc(reinterpret_cast<void**>(&p->ex), static_cast<size_t>(n) * sizeof(Example)) != cudaSuccess) {
        p->ex = nullptr;
        cudaGetLastError();  // not sticky: clear it for later launch checks
        return prop_fail(CRBM_ENOMEM, "examples");
    }
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
    a.bmat = reinterpret_cast<const uint4*>(p->bmat);
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
    a.n_items = nb1 * nb1 * 2 * ctx->n_words;  // (block, 16-chain half of a word)
    // one persistent CTA per SM (four groups of four warps); the attribute and the SM count are set
    // and read once per proposal
    if (p->pass_sms == 0 || p->pass_dev != ctx->device) {
        cudaError_t e = cudaFuncSetAttribute(crbm::k_prop_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(crbm::kSmBytes));
        if (e == cudaSuccess)  // all of the unified L1 / shared memory as shared memory
            e = cudaFuncSetAttribute(crbm::k_prop_pass, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int sms = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        if (e != cudaSuccess) return e;
        p->pass_sms = sms;
        p->pass_dev = ctx->device;
    }
    const int grid = std::min((a.n_items + crbm::kGroups - 1) / crbm::kGroups, crbm::kCtasPerSm * p->pass_sms);
    crbm::k_prop_pass<<<grid, crbm::kCtaThreads, crbm::kSmBytes, ctx->stream>>>(a);
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
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->bmat), crbm::kBElems * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->bias), 33 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->c1), crbm::kC1 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->stats), 4 * sizeof(unsigned long long));
    // He-style initial weights; the output layer starts small (q near 1/2)
    std::vector<float> w(kNP, 0.f);
    uint64_t s = seed ^ 0x243F6A8885A308D3ull;
    for (int i = 0; i < 864; ++i) w[crbm::oW1 + i] = static_cast<float>(unit_normal(s) * std::sqrt(2.0 / 54.0));
    for (int i = 0; i < 2304; ++i) w[crbm::oW2 + i] = static_cast<float>(unit_normal(s) * std::sqrt(2.0 / 144.0));
    for (int i = 0; i < 144; ++i) w[crbm::oW3 + i] = static_cast<float>(unit_normal(s) * 0.01);
    if (e == cudaSuccess) e = cudaMemcpy(p->w, w.data(), kNP * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->m, 0, kNP * 4);
    if (e == cudaSuccess) e = cudaMemset(p->v2, 0, kNP * 4);
    if (e == cudaSuccess) e = cudaMemset(p->stats, 0, 32);
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
    void* b[] = {p->w, p->wb, p->m, p->v2, p->grad, p->loss, p->bmat, p->bias, p->c1, p->stats, p->ex};
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
        crbm::k_prop_train<<<(n + crbm::kTrainEx - 1) / crbm::kTrainEx, crbm::kTrainThreads>>>(p->wb, p->ex, n,
                                                                                              p->grad, p->loss);
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
            crbm::k_prop_train<<<(batch + crbm::kTrainEx - 1) / crbm::kTrainEx, crbm::kTrainThreads, 0, st>>>(
                p->wb, p->ex, batch, p->grad, p->loss);
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
    unsigned long long s[3];
    const cudaError_t e = cudaMemcpy(s, p->stats, 24, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return prop_fail(CRBM_ECUDA, cudaGetErrorString(e));
    *proposed = static_cast<int64_t>(s[0]);
    *accepted = static_cast<int64_t>(s[1]);
    if (s[2] != 0)
        return prop_fail(CRBM_ETIMEOUT, "a block-move pass gave up waiting for its tensor-core MMAs (" +
                                            std::to_string(s[2]) + " CTAs); its moves are incomplete");
    return CRBM_OK;
}

const char* crbm_proposal_last_error(void) { return g_prop_error.c_str(); }

}  // extern "C"
