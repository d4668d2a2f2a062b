// Internal definitions shared by the host runtime (crbm_host.cpp) and the
// CUDA kernels (crbm_kernels.cu).  Not part of the public ABI (include/crbm.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace crbm {

// Index of the packed word of 32-chain word w at site s in either layout.
__host__ __device__ inline size_t word_index(int vil, int w, int N, int s) {
    return vil ? (static_cast<size_t>(w >> 1) * N + s) * 2 + (w & 1)
               : static_cast<size_t>(w) * N + s;
}

#ifndef CRBM_SWEEP_MAX_THREADS
#define CRBM_SWEEP_MAX_THREADS 1024
#endif
constexpr int kMaxSweepWarps = CRBM_SWEEP_MAX_THREADS / 32;  // warps per CTA of the SMEM sweeps
#ifndef CRBM_CHUNKS_PER_WORD
#define CRBM_CHUNKS_PER_WORD 64  // persistent SMEM sweep: a launch is about this many chunks per word
#endif
constexpr int kMaxBonds = 16;  // filters per 3x3 window -> at most 4 hidden Philox calls
constexpr int kNSum = 11;      // per-chain observable sums
constexpr int kAccWords = kNSum * 32 * 2;  // shared-memory words of the [kNSum][32] int64 running sums
constexpr int kWordBits = 32;  // chains per packed word (one bit per chain)
constexpr uint32_t kTagVis = 4u;   // Philox tag of the visible half-step
constexpr uint32_t kTagInit = 5u;  // Philox tag of the initial spins
constexpr uint32_t kTagSwap = 6u;  // Philox tag of replica-exchange decisions
// Bit-plane uniforms (CRBM_RNG_BITPLANE): call j of node n of a cell has tag
// kTagBitplane + 8 n + j and counter word 2 = the 32-chain word (not a chain).
constexpr uint32_t kTagBitplane = 256u;
// Per word, the bit-plane sweep's threshold planes and sign masks:
// [2 classes][3 m = -2, 0, 2][32 planes] hidden, [5 counts][2 J' bits][32
// planes] visible, [2] chains whose class coupling has a negative sign.
constexpr int kBpHidPlanes = 0, kBpVisPlanes = 192, kBpFlip = 512, kBpTab = 516;
static_assert(kBpHidPlanes % 4 == 0 && kBpVisPlanes % 4 == 0 && kBpTab % 4 == 0 && (kNSum * 64) % 4 == 0,
              "the sweeps read four threshold planes with one 16-byte load");

// Canonical fast-path tables per packed word: hidden [2 cls][4 idx][32 lanes]
// then visible [4 spin positions][32 idx][32 lanes] (see crbm_canon.cu).
constexpr int kCanonTh = 2 * 4 * 32;
constexpr int kCanonTab = kCanonTh + 4 * 32 * 32;
// Canonical SMEM-resident sweep: dynamic shared memory holds, in 32-bit
// words, [kAccWords running sums][kCanonTab tables][N spins]
// [n_cells x 32 per-lane hidden words][counters ...]; kCanonSmemV is the
// offset of the spins.
constexpr int kCanonSmemV = kAccWords + kCanonTab;
// Per-cell records of that sweep, kCellRec uint4 per cell, built on the host
// so that the cell loops do no index arithmetic.  Byte offsets are from the
// start of dynamic shared memory; rc.lo = lo(M0 cell) is a round-0 Philox
// word of the cell (M0, M1 the Philox multipliers).  Round 1 multiplies the
// warp-uniform word rc.hi ^ tag = hi(M0 cell) ^ key1 ^ tag by M1, so that
// product is built here too, per call tag t: Qt = (hi(M1 (rc.hi ^ t)) ^ rk2,
// lo(M1 (rc.hi ^ t)) ^ rk4), with the round keys it is XORed with
// (tags 0, 1, 2: hidden calls; v: the visible call):
//   [0] spins (0,0) (1,0) (2,0) (0,2) of the 3x3 window (site (r,1) is (r,0) + 4)
//   [1] spin (1,2), the cell's hidden row, rc.lo, Q2.hi
//   [2] Q0.hi, Q0.lo, Q1.hi, Q1.lo
//   [3] spins (0,0) (1,0) of the cell, hidden rows of the cell and of the cell above
//   [4] hidden row of the cell to the left, rc.lo, Qv.hi, Qv.lo
//   [5] Q2.lo, 0, 0, 0
// In paper precision (two calls per cell) Q2 and Qv are not used: [1].w and
// [4].z hold the byte offset of the cell's row of visible draws instead.
constexpr int kCellRec = 6;
// (class, second-endpoint flag) of the five filter slots of each spin
// position (0,0), (0,1), (1,0), (1,1) in the canonical visible tables.
constexpr int kCanonSlot[4][5][2] = {{{0, 0}, {0, 0}, {1, 0}, {0, 1}, {0, 1}},
                                     {{0, 1}, {0, 0}, {0, 0}, {0, 1}, {1, 1}},
                                     {{0, 0}, {0, 1}, {0, 0}, {0, 1}, {1, 0}},
                                     {{0, 1}, {0, 1}, {1, 1}, {0, 0}, {0, 0}}};

// Lattice and filter geometry, passed by value to kernels (lives in the
// kernel-parameter constant bank, read uniformly by every warp).
struct Geometry {
    int L;         // rows of spins (the side of a square lattice)
    int W;         // window rows = (L + 1) / 2
    int Lc;        // columns of spins (L for a square lattice)
    int Wc;        // window columns = (Lc + 1) / 2
    int N;         // L * Lc
    int n_cells;   // W * Wc
    int nb;        // filters per window
    int n_calls;   // hidden Philox calls per cell = ceil(nb / 4)
    int periodic;  // rows axis: 1 periodic, 0 open (zero padded)
    int pc;        // columns axis: 1 periodic, 0 open
    int canonical; // 1: the ten SS filters on an even, periodic lattice
    int DJ, DJp;   // visible field ranges n_J in [-DJ, DJ], n_J' in [-DJp, DJp]
    int nTv;       // (2 DJ + 1) (2 DJp + 1)
    int nTab;      // 10 hidden entries + n_vis_tab * nTv visible entries
    int n_vis_tab; // 1, or 2 with an odd-column field (even-column table, then odd)
    int n_real_bonds[2];  // bonds with both endpoints real, per class
    int vil;       // spin storage: 0 = [word][site], 1 = 64-chain words [group][site][2]
    int paper;     // CRBM_PRECISION_PAPER: 16-bit thresholds and uniforms, two per Philox word
    int bitplane;  // CRBM_RNG_BITPLANE: uniforms from bit-plane words shared by the 32 chains of a word
    int8_t r1[kMaxBonds], c1[kMaxBonds], r2[kMaxBonds], c2[kMaxBonds];
    uint8_t cls[kMaxBonds];
};

// Word offset, after [kCanonSmemV][N][n_cells x 32][3 x 32 counters]
// [33 segments][32 masks][32][32] replica tables rounded up to 16 bytes, of
// the paper-precision visible draws: [n_cells][32 lanes] pairs of words, the
// two Philox words of tag 1 that carry a cell's four 16-bit visible uniforms
// (drawn in the hidden half-step, read in the visible one).  The records
// follow them when the sweep copies the records into shared memory.
__host__ __device__ inline size_t canon_smem_pw_offset(const Geometry& g) {
    return (static_cast<size_t>(kCanonSmemV) + g.N + static_cast<size_t>(g.n_cells) * 32 + 96 + 33 + 32 + 64 + 3) &
           ~static_cast<size_t>(3);
}
__host__ __device__ inline size_t canon_smem_rec_offset(const Geometry& g) {
    return canon_smem_pw_offset(g) + (g.paper ? static_cast<size_t>(g.n_cells) * 64 : 0);
}

// Generic SMEM-resident sweep (any filter list, odd L, open boundaries).
// Lane-expanded tables per packed word, [kGenHid + nTv][32]: the hidden rows
// [cls][pad][e1 + 2 e2] (pad bit 0: first endpoint zero-padded, bit 1:
// second), indexed by the raw endpoint bits with the coefficient sign folded
// in, then the visible rows [(n_J + DJ) (2 DJp + 1) + n_J' + DJp].
constexpr int kGenHid = 2 * 4 * 4;
// Host-built records of the generic sweep, byte offsets from the start of
// dynamic shared memory:
//   hidden, per (cell, filter k): {first endpoint word, second endpoint word
//     (the zero word for a padded endpoint), table row of (cls, pad), 0};
//   visible, kGenVisRec per cell: [0] the 16-bit hidden rows of the four
//     cells whose windows can hold the cell's spins (own, above, left,
//     above-left; a zero row where there is none); then per owned spin
//     x = 2 r + c: [1 + 2x] J masks, [2 + 2x] J' masks over the four rows'
//     expanded words (bit k: filter k with the spin as first endpoint, bit
//     16 + k: as second endpoint); [9] the table row of n_J = n_J' = -deg
//     of each spin; [10] each spin's word (a scratch word for a position past
//     the lattice edge).
constexpr int kGenVisRec = 11;
// Word offsets of the generic sweep's dynamic shared memory.
struct GenericSmem {
    size_t tab;      // [kGenHid + n_vis_tab nTv][32] thresholds
    size_t v;        // [N] spins
    size_t zero;     // one zero word (padded endpoints), then one scratch word
    size_t hw;       // [n_cells][32] 16-bit per-lane hidden words (bit k: filter k)
    size_t zrow;     // [32] 16-bit zeros
    size_t cnt;      // [3][32] measurement counters
    size_t seg;      // [33]
    size_t segmask;  // [32]
    size_t sob;      // [32] replica slot of each rung, then [32] rung of each slot
    size_t total;
};
__host__ __device__ inline GenericSmem generic_smem(const Geometry& g) {
    GenericSmem s;
    s.tab = static_cast<size_t>(kAccWords);
    s.v = s.tab + static_cast<size_t>(kGenHid + g.n_vis_tab * g.nTv) * 32;
    s.zero = s.v + g.N;
    s.hw = (s.zero + 2 + 3) & ~static_cast<size_t>(3);
    s.zrow = s.hw + static_cast<size_t>(g.n_cells) * 16;
    s.cnt = s.zrow + 16;
    s.seg = s.cnt + 96;
    s.segmask = s.seg + 33;
    s.sob = s.segmask + 32;
    s.total = s.sob + 64;
    return s;
}

// Device buffers of one context (all owned by the context).
struct DeviceState {
    uint32_t* v = nullptr;        // [n_words][N] packed spins, bit l = chain 32w + l
    uint32_t* tab = nullptr;      // generic: [n_words][kGenHid + nTv][32] lane-expanded thresholds
    uint32_t* ctab = nullptr;     // [n_words][kCanonTab] canonical fast-path tables
    uint4* crec = nullptr;        // SMEM layout: canonical [n_cells][kCellRec] or generic per-cell records
    uint32_t* sneg = nullptr;     // [n_words][2] lanes whose class coefficient s = -1
    uint32_t* gep = nullptr;      // generic: [n_cells][nb] filter endpoint words (measurement)
    int64_t* sums = nullptr;      // [n_words * 32][kNSum]
    int32_t* series = nullptr;    // [series_len][n_words * 32][3]
    int64_t* corr = nullptr;      // [n_params][N] correlation sums
    int32_t* seg = nullptr;       // [n_words][33]: n_seg, then (param << 8 | first lane) ...
    uint32_t* segmask = nullptr;  // [n_words][32] lane mask of each segment
    int8_t* spins8 = nullptr;     // [n_words * 32][N] staging for get/set spins
    int32_t* sob = nullptr;       // tempering: [n_words][32] replica slot holding each rung
    uint32_t* swap_tab = nullptr; // tempering: swap thresholds, per (word, pair) at swap_off
    int32_t* swap_off = nullptr;  // [n_words][32]
    int32_t* swap_len = nullptr;  // [n_words][32]: thresholds for dE = 1 .. len-1 (0 beyond)
    int32_t* wq = nullptr;        // [n_words][3] Q.4 couplings (J, J', h) of each word
    uint32_t* h = nullptr;        // streamed layout: [n_words][n_cells][10] hidden words
    int* cnt = nullptr;           // streamed layout: [n_words * 32][3] measurement counts
    float* chain_bh = nullptr;    // block proposals: [n_words * 32][2] beta, h (bf16-rounded)
    int32_t* chain_q = nullptr;   // block proposals: [n_words * 32][3] Q.4 J, J', h
    int* sched = nullptr;         // persistent scheduler: [n_words + 4] word states (chunks done, held)
    int64_t* hit = nullptr;       // time to solution: [n_words * 32][2] target energy, first hitting sweep
    int32_t* hit_q = nullptr;     // [n_words * 32][4] Q.4 J, J', h of each chain's point
    int* flag = nullptr;          // [1] crbm_set_spins: set when an input spin is not +-1
};

struct SweepArgs {
    Geometry g;
    uint32_t* v;
    const uint32_t* tab;
    const uint32_t* ctab;
    const uint4* crec;
    const uint32_t* sneg;
    const uint32_t* gep;  // generic path: [n_cells][nb] filter endpoint words (see crbm_generic_body.cuh)
    int64_t* sums;
    int32_t* series;
    uint32_t* h;
    int* cnt;
    int32_t* sob;
    const uint32_t* swap_tab;
    const int32_t* swap_off;
    const int32_t* swap_len;
    const int32_t* wq;
    int swap_every;       // 0 = no replica exchange
    int n_bands;          // batched cluster launch: CTAs (bands of cell rows) per word, else 1
    const int64_t* clock; // batch launches: device {sweep, measurements} (else t0 / meas0)
    int64_t* hit;         // time to solution (nullptr = off): per chain {target energy, first hitting sweep}
    const int32_t* hit_q; // per chain {Q.4 J, J', h, 0}
    int64_t* corr;
    const int32_t* seg;
    const uint32_t* segmask;
    int n_words;
    int n_chains_padded;
    uint32_t key0, key1;
    uint32_t rk[20];      // Philox round keys: rk[2r] = key0 + r W0, rk[2r+1] = key1 + r W1
    uint32_t t0;          // first global sweep index of this launch
    int n_sweeps;
    int measure_every;    // 0 = never
    int64_t meas0;        // measurements recorded before this launch (series index)
    int series_len;
    int sq_every;         // 0 = never
    // (kept last: the fields above keep the offsets the sweep kernels were tuned with; rk is
    // read as 8-byte constant pairs)
    int n_chains;         // real chains (replica-exchange ladders: n_chains / 32)
};

// Host model helpers (crbm_host.cpp): Q.4 rounding of a coupling, and the
// ten hidden + (2DJ+1)(2DJp+1) visible thresholds and the two class signs of
// one parameter point.
bool host_to_q4(double x, int32_t& q);
void host_point_tables(const Geometry& g, double beta, int32_t qJ, int32_t qJp, int32_t qh,
                       uint32_t* out, int sgn[2]);

// Batched launch: up to kMaxBatch contexts' descriptors by value (kernel
// parameter space), and a work list of (descriptor, word) per CTA.
constexpr int kMaxBatch = 16;
struct BatchArgs {
    const int4* items;    // per CTA: (descriptor or -1, word, band, bands)
    int n_desc;
    int smem_rec;         // 1: canonical members stage their per-cell records in shared memory
    SweepArgs d[kMaxBatch];
};

// Kernel launchers (crbm_kernels.cu).  All return cudaGetLastError().
size_t smem_bytes_generic(const Geometry& g);
size_t smem_bytes_canon(const Geometry& g);
// Whether the canonical persistent sweep keeps the per-cell records in shared
// memory (when that does not lower the CTAs per SM), and its dynamic shared
// memory with that choice.
bool canon_smem_records(const Geometry& g);
size_t smem_bytes_canon_launch(const Geometry& g);
cudaError_t launch_init(const Geometry& g, uint32_t* v, int n_words, uint32_t key0,
                        uint32_t key1, cudaStream_t st);
cudaError_t launch_sweep_generic(const SweepArgs& a, int warps_per_cta, cudaStream_t st);
cudaError_t launch_sweep_canon_persistent(const SweepArgs& a, int warps_per_cta, int chunk, int* sched,
                                          cudaStream_t st);
cudaError_t launch_sweep_stream(const SweepArgs& a, cudaStream_t st, int64_t* launches);
// Bit-plane sweep (crbm_bitplane.cu): a persistent grid that claims (word,
// chunk) items as the canonical sweep does (sched: 4 + n_words ints), each
// word's lattice, hidden words and threshold planes in shared memory, the
// node records there too when they fit.  Per-CTA dynamic shared memory with
// and without the records.
size_t smem_bytes_bitplane(const Geometry& g, bool with_records);
cudaError_t launch_sweep_bitplane(const SweepArgs& a, int warps_per_cta, int chunk, int* sched, cudaStream_t st);
// modes: the member kinds of the batch besides exact lane-uniform and generic
// ones (kBatchPaper, kBatchBitplane), which pick the kernel instantiation.
constexpr int kBatchPaper = 1, kBatchBitplane = 2;
cudaError_t launch_sweep_batch(const BatchArgs& b, int n_tasks, int cluster, int threads, size_t smem, int modes,
                               cudaStream_t st);
// Clusters of `cluster` batch CTAs that can be resident at once (0: none).
int batch_max_active_clusters(int cluster, int threads, size_t smem, int modes);
cudaError_t launch_batch_advance(int64_t* clocks, const int* every, int n_ctx, int64_t n_sweeps, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* in, uint32_t* out, int n, cudaStream_t st);
cudaError_t launch_philox_stream(uint32_t* sink, int n_blocks, int threads, int calls, uint32_t k0,
                                 uint32_t k1, cudaStream_t st);
cudaError_t launch_unpack(const Geometry& g, const uint32_t* v, int8_t* out, int n_words,
                          cudaStream_t st);
// Sets *flag (zeroed first) when any of the n bytes at `in` is not +1 or -1.
cudaError_t launch_check_spins(const int8_t* in, size_t n, int* flag, cudaStream_t st);
// Packs the staged int8 spins into the packed words, unless skip is non-null
// and *skip is set (an invalid input found by launch_check_spins).
cudaError_t launch_pack(const Geometry& g, const int8_t* in, uint32_t* v, int n_words, const int* skip,
                        cudaStream_t st);

}  // namespace crbm
