/*
 * crbm.h — C ABI of the GB300 block-Gibbs sampler for the convolutional RBM
 * (CRBM) that encodes the classical Shastry–Sutherland (SS) Ising lattice.
 *
 * Method: Brahma, Han, Razzaque, Patel, Salahuddin, "Hardware Acceleration of
 * Frustrated Lattice Systems using Convolutional Restricted Boltzmann
 * Machine", arXiv 2511.20911:
 *   Eq. (1)      SS Hamiltonian H = J1 sum_nn s s + J2 sum_diag s s + h_z sum s
 *   Eqs. (3)-(7) bond -> hidden unit mapping, a = 1/2 arccosh(exp(2|J|))
 *   Eq. (8)      the ten 3x3 stride-2 convolutional filters of the unit cell
 *   Eqs. (9)-(10) hidden | visible and visible | hidden conditionals
 *   Sec. II.C and the appendix: the host writes weights, biases, sizes and
 *   periodicity, runs sampling cycles, and reads samples back.
 *
 * Readings fixed by this library (the CPU oracle in oracle/ implements the
 * same ones independently; trajectories agree bit for bit):
 *   - spins and hidden units are +1/-1; H uses -h sum s (h > 0 favours +1);
 *   - a bond of coupling J has K = -beta J, weight a = 0.5*acosh(exp(2|K|)),
 *     coefficient +1 on its first endpoint and s = (K >= 0 ? +1 : -1) on its
 *     second; hidden bias 0; visible bias beta*h;
 *   - J, J', h are rounded to the nearest 1/16 (Q.4 fixed point,
 *     |16 x| <= 2047), so energies are exact integers in units of 1/16;
 *   - acceptance: a unit becomes +1 iff u < thr(y), u a 32-bit Philox-4x32-10
 *     word, thr(y) = min(2^32-1, nearbyint(2^32 / (1 + exp(-y)))) in double;
 *   - Philox counter (cell, sweep, chain, tag), key (seed lo, seed hi): hidden
 *     bond k uses word k&3 of tag k>>2; the spin at window offset (r, c) uses
 *     word 2r+c of tag 4; the initial spin is +1 iff that word of tag 5 at
 *     sweep 0 is < 2^31.
 *
 * Conventions for every function:
 *   - return CRBM_OK (0) or a negative CRBM_E* code; crbm_last_error() then
 *     holds a message.  No C++ exception crosses this boundary.
 *   - the caller owns every host buffer; the context owns all device memory.
 *   - a context is bound to the CUDA device current at crbm_create and to the
 *     stream given there; calls on one context are not thread-safe.
 *   - crbm_sweep is asynchronous on that stream; every function that returns
 *     data to the host synchronises the stream first.
 */
#ifndef CRBM_H
#define CRBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CRBM_OK 0
#define CRBM_EINVAL -1       /* bad argument or buffer size */
#define CRBM_ENOMEM -2       /* device or host allocation failed */
#define CRBM_ECUDA -3        /* a CUDA runtime call failed */
#define CRBM_ETIMEOUT -4     /* reserved: a bounded device-side wait gave up (no kernel of this build waits) */
#define CRBM_EUNSUPPORTED -5 /* valid request this build cannot serve */

#define CRBM_NSUM 11 /* per-chain observable sums, see crbm_observables */

/* Layout of a context's lattice state on the device. */
#define CRBM_LAYOUT_AUTO 0   /* SMEM when it fits one CTA (L <= CRBM_SMEM_MAX_L), else STREAM */
#define CRBM_LAYOUT_SMEM 1   /* whole lattice resident in shared memory */
#define CRBM_LAYOUT_STREAM 2 /* lattice in HBM, one tiled launch per sweep */
#define CRBM_SMEM_MAX_L 96

/* Arithmetic of the conditionals (Eqs. 9-10). */
#define CRBM_BC_AS_ROWS 0
#define CRBM_BC_PERIODIC 1
#define CRBM_BC_OPEN 2

/* Source of the uniforms. */
#define CRBM_RNG_LANE 0     /* one Philox stream per chain: counter (cell, sweep, chain, tag) */
#define CRBM_RNG_BITPLANE 1 /* bit-plane words shared by the 32 chains of a word (see crbm_params) */

#define CRBM_PRECISION_EXACT 0 /* double-precision weights, 32-bit thresholds and uniforms */
#define CRBM_PRECISION_PAPER 1 /* the paper's FPGA (Sec. III, "Dimension and Precision"):
                                * weights and visible bias in 10-bit fixed point (4 fraction
                                * bits), a 12-bit accumulator, a 16-bit sigmoid table and
                                * 16-bit uniforms, two per Philox word (see crbm_params) */

typedef struct crbm_ctx crbm_ctx;

/* One filter of Eq. (8): the bond between two sites of the 3x3 window
 * (row, col offsets in [0, 2]); cls 0 = J (J1), 1 = J' (J2). */
typedef struct {
    int8_t r1, c1, r2, c2;
    uint8_t cls;
} crbm_bond;

typedef struct {
    int32_t L;        /* L x L spins, 3 <= L <= 4096 */
    int32_t periodic; /* 1 = periodic in both directions, 0 = open (zero padded) */
    const crbm_bond* bonds; /* NULL -> the ten SS filters of Fig. 1 */
    int32_t n_bonds;        /* 1..16 when bonds != NULL */
    /* parameter points p = 0..n_params-1 (host arrays of length n_params) */
    const double* J;
    const double* Jp;
    const double* h;
    const double* beta;
    int32_t n_params;
    /* chain -> parameter point (host array of n_chains), NULL -> contiguous
     * equal blocks: p(c) = c * n_params / n_chains */
    const int32_t* chain_param;
    int32_t n_chains;       /* 1 .. 2^30 */
    uint64_t seed;          /* Philox key */
    int32_t measure_every;  /* accumulate observables after every K-th sweep, 0 = never */
    int32_t series_len;     /* per-chain time-series capacity in measurements, 0 = none */
    int32_t sq_every;       /* accumulate spin correlations every K_S sweeps, 0 = never */
    int32_t layout;         /* CRBM_LAYOUT_* */
    /* Replica exchange (parallel tempering), 0 = off.  > 0: every 32-chain
     * group c = 32 l .. 32 l + 31 is a temperature ladder -- rung k is the
     * parameter point chain_param[32 l + k], all rungs with equal J, J', h and
     * beta strictly increasing in k -- and after every swap_every-th sweep
     * adjacent rungs exchange configurations by the Metropolis rule
     * min(1, exp((beta_k - beta_{k+1}) (E_k - E_{k+1}))) on exact integer
     * energies.  Needs n_chains % 32 == 0 (either layout; in the streamed
     * one a 32-chain half of a 64-chain group is a ladder).  Observables
     * then belong to rungs (row 32 l + k), spins to replica slots (see
     * crbm_get_permutation). */
    int32_t swap_every;
    void* stream;           /* cudaStream_t for all work; NULL = legacy default stream */
    /* CRBM_PRECISION_*.  PAPER: A = q(a_cls), B = q(beta h) with q(x) the
     * nearest multiple of 1/16 clamped to +-511/16; a unit's 16-bit threshold
     * is min(65535, nearbyint(2^16 / (1 + exp(-2 y)))) with y = A m (hidden)
     * or B + A_J n_J + A_J' n_J' (visible), y clamped to +-2047/16; its 16-bit
     * uniform is a half of a Philox word (low half first): hidden filter
     * k < 8 half k&1 of word k>>1 of tag 0, filters 8 and 9 word 0 of tag 1,
     * the spin at window offset (r, c) half (2r+c)&1 of word 1 + ((2r+c)>>1)
     * of tag 1 -- two Philox calls per cell instead of four (three in the
     * streamed layout, whose visible half-step draws the tag-1 call again).
     * Needs at most ten filters (any lattice: the SS fast path, SMEM or
     * streamed, or the generic SMEM sweep, whose visible half-step also draws
     * the tag-1 call again); not with block proposals (a batch runs such a
     * member's words whole, unsplit).  crbm_get_tables returns the 16-bit
     * thresholds in the upper halves of the 32-bit entries. */
    int32_t precision;
    /* Rectangular lattices and a boundary per axis (Sec. III: open boundaries
     * along the lateral direction for laterally confined strips).  L_cols = 0
     * keeps the lattice L x L; otherwise it has L rows and L_cols columns
     * (3..4096).  periodic_cols: CRBM_BC_AS_ROWS (0) takes `periodic` for the
     * columns too, CRBM_BC_PERIODIC (1) or CRBM_BC_OPEN (2) sets the column
     * axis on its own (`periodic` then covers the rows).  Windows (i, j),
     * i < (L+1)/2, j < (L_cols+1)/2, cell index i (L_cols+1)/2 + j; spins
     * [chain][row][column].  Even sides periodic along both axes run on the
     * SS fast path (SMEM or streamed layout); any other lattice on the
     * generic SMEM sweep. */
    int32_t L_cols;
    int32_t periodic_cols;
    /* Field of the odd columns (the appendix's separate odd- and even-column
     * visible biases), host array of n_params, or NULL for h everywhere.  With
     * it, crbm_get_tables returns a second visible table (odd columns) after
     * the first, and crbm_observables' M is still the total magnetisation.
     * Not with replica exchange (its energies use the total M). */
    const double* h_odd;
    /* CRBM_RNG_LANE (0) or CRBM_RNG_BITPLANE.  Bit-plane uniforms: for the
     * 32 chains c = 32 w + l of word w, node n of cell `cell` in sweep t draws
     * plane words P_b, b = 0..31, P_(4j+i) = word i of Philox((cell, t, w,
     * 256 + 8 n + j)), and chain l's uniform is sum_b bit l of P_b << (31 -
     * b): most significant bit first, so a comparison of all 32 uniforms
     * with their thresholds can stop at the first plane on which every chain
     * is decided (two calls per node, then the nodes still open, about 12 %,
     * from a straggler list: 2.2 calls per node and word instead of 8 calls
     * for 32 separate uniforms).  Node n = k for hidden filter k, 10 +
     * 2r + c for the spin at window offset (r, c).  Needs the ten SS filters
     * on an even periodic lattice (SMEM or streamed layout; replica exchange
     * in the SMEM layout, where slot l draws as chain 32 w + l whichever rung
     * it holds), exact precision, no correlations; not with block proposals
     * (a batch runs such a member's words whole, node records read from
     * global memory).  A different random stream: the chains differ from
     * CRBM_RNG_LANE's, with the same law. */
    int32_t rng;
} crbm_params;

/* Build the model (Eqs. 3-8), the threshold tables, allocate device state and
 * draw the initial spins (tag 5) on the stream.  *out receives the context.
 * Errors: CRBM_EINVAL (bad sizes, couplings outside Q.4 range, beta < 0 or
 * NaN, bond outside the window), CRBM_ENOMEM, CRBM_ECUDA. */
int crbm_create(crbm_ctx** out, const crbm_params* params);

/* Free all device memory; NULL is ignored. */
void crbm_destroy(crbm_ctx* ctx);

/* Run n_sweeps sweeps (Sec. II.B: all hidden units from Eq. 9, then all spins
 * from Eq. 10), continuing the global sweep counter.  Asynchronous.
 * Errors: CRBM_EINVAL (n_sweeps < 0 or counter past 2^32-1), CRBM_ECUDA. */
int crbm_sweep(crbm_ctx* ctx, int64_t n_sweeps);

/* Global number of sweeps done since creation (or since crbm_load). */
int64_t crbm_sweep_count(const crbm_ctx* ctx);

/* Per-chain exact integer sums over measurements (measure_every), host array
 * out[n_chains][CRBM_NSUM] int64 = {n, sum NJ, sum NJ', sum M, sum |M|,
 * sum NJ^2, sum NJ'^2, sum M^2, sum NJ NJ', sum NJ M, sum NJ' M}, where for
 * one configuration NJ = sum over J bonds of s_i s_j, NJ' likewise over J'
 * bonds, M = sum s (so E = J NJ + J' NJ' - h M).  n_out = number of int64s.
 * Synchronises the stream. */
int crbm_observables(crbm_ctx* ctx, int64_t* out, size_t n_out);

/* Time to solution (Sec. III, "Hardware Acceleration").  Give every
 * parameter point a target energy in 1/16 units, E = qJ NJ + qJ' NJ' - qh M
 * (Q.4 couplings; e.g. its ground-state energy): from then on every
 * measurement (measure_every) records, per chain, the first global sweep
 * count t + 1 after which the chain's energy was at or below its target.
 * crbm_set_targets (host array of n_params, synchronises) also clears the
 * records; crbm_first_hits writes host out[n_chains] int64, -1 for a chain
 * that has not reached its target.  With replica exchange the records belong
 * to rungs.  Not part of checkpoints.  Errors: CRBM_EINVAL (n_params not the
 * context's; the targets in force stay), CRBM_ENOMEM, CRBM_ECUDA (either of
 * these leaves the context without targets: nothing is recorded until a
 * call succeeds). */
int crbm_set_targets(crbm_ctx* ctx, const int64_t* e_target, int32_t n_params);
int crbm_first_hits(crbm_ctx* ctx, int64_t* out, size_t n_out);

/* Time series, host array out[series_len][n_chains][3] int32 = (NJ, NJ', M)
 * per measurement (entries past the number of measurements are zero). */
int crbm_series(crbm_ctx* ctx, int32_t* out, size_t n_out);

/* Spin-correlation sums of Sec. IV.B, host array out[n_params][L*L] int64:
 * out[p][dR*L+dC] = sum over sampled configurations of chains at p of
 * sum_r s_r s_{r+d} (periodic lattices only), and n_samples[p] (may be NULL). */
int crbm_correlations(crbm_ctx* ctx, int64_t* out, size_t n_out, int64_t* n_samples);

/* Static structure factor per spin, host array out[n_params][L*L] double:
 * S(q) = (1/N) <|sum_r s_r e^{i q.r}|^2>, q = 2 pi (nR, nC) / L, from the
 * correlation sums (Eq. 11 with the 1/N of the text's per-spin plots). */
int crbm_structure_factor(crbm_ctx* ctx, double* out, size_t n_out);

/* Zero every accumulator (sums, series, correlations). */
int crbm_reset_observables(crbm_ctx* ctx);

/* Spins as int8 +-1, host array [n_chains][L][L] (pinned host memory makes
 * the copies direct).  crbm_set_spins checks the values on the device and
 * sets the chains only when every one is +1 or -1 (else CRBM_EINVAL, chains
 * unchanged).  Both synchronise the stream. */
int crbm_get_spins(crbm_ctx* ctx, int8_t* out, size_t n_out);
int crbm_set_spins(crbm_ctx* ctx, const int8_t* in, size_t n_in);

/* Threshold tables, host array [n_params][10 + (2DJ+1)(2DJ'+1)] uint32:
 * Th[cls][m+2] (m in -2..2) then Tv[nJ+DJ][nJ'+DJ'].  dims may be NULL; else
 * dims[0] = DJ, dims[1] = DJ'. */
int crbm_get_tables(crbm_ctx* ctx, uint32_t* out, size_t n_out, int32_t* dims);

/* Replica permutation of a tempering context, host array out[n_chains]
 * int32: out[32 l + k] = replica slot (chain index within ladder l) that
 * holds rung k.  The identity without tempering. */
int crbm_get_permutation(crbm_ctx* ctx, int32_t* out, size_t n_out);

/* Which layout the context runs (CRBM_LAYOUT_SMEM or CRBM_LAYOUT_STREAM). */
int crbm_layout(const crbm_ctx* ctx);

/* Autotuner: time the CTA shapes of the SMEM sweep (2..32 warps per CTA; at
 * most 16 for the generic kernel, at most one per cell) for probe_sweeps sweeps each on scratch copies of the context's
 * spins (its chains, counters and observables are untouched), keep the
 * fastest for this context and append it to the cache file
 * ($CRBM_AUTOTUNE_CACHE, default $HOME/.cache/crbm_autotune.txt), which
 * crbm_create consults for contexts of the same shape on the same GPU model.
 * best_warps may be NULL.  Synchronises the stream.  Errors: CRBM_EINVAL,
 * CRBM_EUNSUPPORTED (streamed layout), CRBM_ECUDA. */
int crbm_autotune(crbm_ctx* ctx, int64_t probe_sweeps, int32_t* best_warps);

/* Warps per CTA the context's SMEM sweep launches with. */
int crbm_warps(const crbm_ctx* ctx);

/* Kernel launches issued by this context since creation. */
int64_t crbm_launch_count(const crbm_ctx* ctx);

/* Checkpoint: serialise spins, sweep counter, seed and accumulators into a
 * caller buffer.  With buf == NULL, *n receives the size needed.  Resume is
 * bit-exact because every draw is a function of (cell, sweep, chain, tag). */
int crbm_save(crbm_ctx* ctx, void* buf, size_t* n);
int crbm_load(crbm_ctx* ctx, const void* buf, size_t n);

/* Evaluate the library's device Philox-4x32-10 (Salmon et al., SC'11) on n
 * host inputs in[n][6] = (c0, c1, c2, c3, k0, k1) into host out[n][4], on the
 * current device's legacy stream.  For verification of the generator that
 * keys every draw; synchronous.  Errors: CRBM_EINVAL, CRBM_ENOMEM, CRBM_ECUDA. */
int crbm_philox(const uint32_t* in, uint32_t* out, size_t n);

/* Philox throughput probe (integer-multiply ceiling of this path): device
 * sink[n_blocks * threads] (caller-owned), thread t of the launch runs `calls`
 * Philox-4x32-10 calls with key = (seed lo, seed hi) on the counters
 * (i, t, i ^ t, 0x9E3779B9), i = 0 .. calls - 1, and stores the XOR of all
 * their output words in sink[t].  Each call is 20 32x32->64 products, none
 * shareable between calls.  Asynchronous on `stream` (a cudaStream_t, NULL =
 * legacy); time it with events there.  threads a multiple of 32 in 32..1024.
 * Errors: CRBM_EINVAL, CRBM_ECUDA. */
int crbm_philox_stream(uint32_t* sink, int32_t n_blocks, int32_t threads, int32_t calls, uint64_t seed,
                       void* stream);

/* Batched sweeps: several SMEM-layout contexts -- mixed lattice sizes,
 * filter lists, precisions, uniform modes and tempering ladders -- advanced
 * together by ONE kernel launch plus a one-thread clock update, captured once
 * in a CUDA graph and replayed on the members' common stream.  The launch has
 * one CTA per packed word of every member, heaviest lattices first, except
 * that with thread-block clusters of C CTAs (environment CRBM_BATCH_CLUSTER,
 * default 8, 1 = none) a canonical exact-precision, lane-uniform word without
 * correlations that has at least C cell rows and 16 cells per band is split
 * into C bands of cell rows, one cluster per word, the bands exchanging their
 * boundary rows through distributed shared memory.  Members keep their own state, counters and getters; each
 * batched call advances every member by n_sweeps sweeps, bit-identical to
 * calling crbm_sweep on each.  The CTA shape is the largest warps count of
 * the members (see crbm_autotune) until crbm_batch_autotune picks one for
 * the batch itself. */
#define CRBM_BATCH_MAX 16
typedef struct crbm_batch crbm_batch;
/* Errors: CRBM_EINVAL (0 or more than CRBM_BATCH_MAX members, a repeated
 * member, a streamed-layout member, members on different devices or
 * streams), CRBM_ENOMEM, CRBM_ECUDA.  The members must outlive the batch. */
int crbm_batch_create(crbm_batch** out, crbm_ctx* const* ctxs, int32_t n_ctx);
/* Asynchronous on the members' stream.  n_sweeps in 0..2^20. */
int crbm_batch_sweep(crbm_batch* batch, int64_t n_sweeps);
int crbm_batch_threads(const crbm_batch* batch);
/* Batch autotuner: time the batched launch with CTAs of 8, 12, ..., 32 warps
 * (the shapes whose clusters can be resident) for probe_sweeps sweeps each
 * and keep the fastest for this batch.  The members' chains, counters,
 * observables, series, correlations, replica permutations and first-hit
 * records are checkpointed to host memory first and put back after every
 * probe, so a tuned batch continues bit-identically.  Synchronises the
 * stream.  best_threads (threads per CTA) may be NULL.  Errors: CRBM_EINVAL
 * (probe_sweeps outside 1..100000, or a member's 32-bit sweep counter would
 * overflow), CRBM_ECUDA (the shape in use before the call is kept). */
int crbm_batch_autotune(crbm_batch* batch, int64_t probe_sweeps, int32_t* best_threads);
/* Cluster size C of the batched launch (1: no clusters, no word split). */
int crbm_batch_cluster(const crbm_batch* batch);
/* Message for the last failed call on batch (or crbm_batch_create if NULL). */
const char* crbm_batch_last_error(const crbm_batch* batch);
void crbm_batch_destroy(crbm_batch* batch);

/* ---- Learned block proposal --------------------------------------------
 * A k x k block (k = 4) of spins is proposed from a small convolutional net
 * over the (k+6) x (k+6) periodic patch around it: input channels spin (0
 * inside the block), block mask, row parity, column parity, beta, h; three
 * valid 3x3 convolutions 6 -> 16 -> 16 -> 1 with ReLU; one logit per block
 * site, q = sigmoid(logit) = P(+1).  Weights and activations are bfloat16,
 * accumulation fp32.  The net never sees the block's own spins, so forward
 * and reverse proposal probabilities are exact and each move passes a
 * Metropolis-Hastings test min(1, exp(-beta dE/16) q(x)/q(x')) on the exact
 * integer energy difference dE (1/16 units).  A pass moves blocks at least 8
 * sites apart (max(1, L/8) per side, random offset), one per 32-chain word
 * and block per CTA.  Not a method of the paper: a learned proposal mixed
 * with its block Gibbs sweeps, judged by it (observables within standard
 * errors) and trained on configurations it generates.
 * Parameter order (3345 floats): W1[16][6][3][3], b1[16], W2[16][16][3][3],
 * b2[16], W3[16][3][3], b3.
 * Contexts used with proposals need the ten SS filters, an even periodic
 * lattice of side L >= 10 (so that a patch does not wrap onto its own
 * block), the SMEM layout and no replica exchange (else CRBM_EUNSUPPORTED).
 * Keying of a pass (Philox key = the context's seed): block b of pass P has
 * origin (o0 % L + S (b / n), o1 % L + S (b % n)) mod L, n = max(1, L / 8)
 * blocks per side, S = L / n, (o0, o1) = words 0, 1 of Philox((P, 0, 0, 8));
 * site s of chain c proposes +1 iff word s % 4 of Philox((b, P, c, 9 + s / 4))
 * is below thr[s] = clamp(2^32 q_s, 1, 2^32 - 256); the move is accepted iff
 * log alpha >= 0 or (word 0 of Philox((b, P, c, 13)) >> 8) / 2^24 <
 * exp(log alpha).
 * Errors of these functions: see crbm_proposal_last_error(). */
typedef struct crbm_proposal crbm_proposal;
typedef struct {
    float logit[16];
    int32_t dE;               /* exact energy change of the proposed block, 1/16 units */
    uint32_t cur_bits, new_bits; /* bit s = site (s / 4, s % 4) of the block is +1 */
    float log_alpha;          /* -beta dE / 16 + sum log q(current) - sum log q(proposed) */
    int32_t bR, bC;           /* block origin */
    uint32_t thr[16];         /* site s proposes +1 iff its Philox draw < thr[s] */
} crbm_pass_record;
/* New net with seeded He-style weights; block must be 4. */
int crbm_proposal_create(crbm_proposal** out, int32_t block, uint64_t seed);
void crbm_proposal_destroy(crbm_proposal* p);
int crbm_proposal_set_weights(crbm_proposal* p, const float* w, size_t n);
int crbm_proposal_get_weights(crbm_proposal* p, float* w, size_t n);
/* Train on the GPU: per step, crbm_sweep(ctx, sweeps_between), draw `batch`
 * (chain, block) examples from ctx's current configurations, back-propagate
 * the mean binary cross-entropy of q against the blocks' spins, Adam step
 * (lr).  losses[steps] (may be NULL) receives the batch losses. */
int crbm_proposal_train(crbm_proposal* p, crbm_ctx* ctx, int32_t steps, int32_t batch, float lr,
                        int32_t sweeps_between, float* losses);
/* Loss and gradient (fp32, GPU) on given examples: host spins[n][L*L] (+-1),
 * block origins[n][2], beta_h[n][2]; grad[3345]. */
int crbm_proposal_loss_grad(crbm_proposal* p, const int8_t* spins, int32_t L, const int32_t* origins,
                            const float* beta_h, int32_t n, float* loss, float* grad);
/* n_passes passes of block moves (asynchronous). */
int crbm_proposal_pass(crbm_ctx* ctx, crbm_proposal* p, int64_t n_passes);
/* n_sweeps times: one Gibbs sweep, then one pass of block moves. */
int crbm_sweep_mixed(crbm_ctx* ctx, crbm_proposal* p, int64_t n_sweeps);
/* n_sweeps Gibbs sweeps with one pass of block moves after every `every`
 * sweeps (the sweeps between passes run in one launch); every >= 1, every =
 * 1 is crbm_sweep_mixed.  A final group shorter than `every` ends with a pass
 * too. */
int crbm_sweep_mixed_every(crbm_ctx* ctx, crbm_proposal* p, int64_t n_sweeps, int32_t every);
/* The next pass, evaluated without moving: records out[n_words][n_blocks][32]. */
int crbm_proposal_inspect(crbm_ctx* ctx, crbm_proposal* p, crbm_pass_record* out, size_t n_out);
/* Cumulative proposed / accepted block moves of p. */
int crbm_proposal_stats(crbm_proposal* p, int64_t* proposed, int64_t* accepted);
const char* crbm_proposal_last_error(void);

/* Size of the fixed device scratch array of crbm_sweep_stream_noalloc. */
#define CRBM_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Streamed sweep that allocates nothing, for callers that cannot call
 * cudaMalloc (code running under another framework's allocator or memory
 * pool, or a service whose device memory is fixed at start-up).  The paper
 * has no counterpart: it is the two-launch streamed sweep of the
 * CRBM_LAYOUT_STREAM contexts, stateless and without a context.
 *
 * p: the model and chains (L even, periodic = 1, bonds = NULL, J, Jp, h,
 *    beta, n_params, chain_param, n_chains, seed, stream, precision);
 *    L_cols 0 or L, periodic_cols CRBM_BC_AS_ROWS or CRBM_BC_PERIODIC,
 *    h_odd NULL, rng CRBM_RNG_LANE; measure_every, series_len, sq_every and layout are ignored:
 *    no observables are kept.
 * v: device spins owned by the caller, in/out, the streamed layout:
 *    u32 v[ceil(n_chains/64)][L*L][2], bit l of v[g][s][k] = spin +1 of chain
 *    64 g + 32 k + l at site s (pad chains of the last group are sampled too).
 * Runs sweeps sweep0 .. sweep0 + n_sweeps - 1 of the same Philox keying as a
 * context, so the result is bit-identical to crbm_sweep on a
 * CRBM_LAYOUT_STREAM context holding the same spins at the same sweep count.
 *
 * Scratch: one static device array of CRBM_NOALLOC_SCRATCH_BYTES per GPU that
 * loads the library, held until exit; it takes the lane threshold tables and
 * the lanes' hidden words, 4 * n_words * (4352 + 32 (L/2)^2) bytes with
 * n_words = 2 ceil(n_chains / 64).  Larger requests return
 * CRBM_EUNSUPPORTED.  Every call shares the array and leaves its contents
 * behind (each call rewrites all of it that it reads), so calls that overlap
 * on the GPU -- on different streams, or from several threads -- race.
 * The first call on a device fetches the array's device address
 * (cudaGetSymbolAddress, with that device current; a failed lookup is tried
 * again by the next call); make that first call before any stream capture.
 * Asynchronous on p->stream apart from the table upload: every call copies
 * the lane tables from pageable host memory, one cudaMemcpyAsync per 32-chain
 * word, and each of those copies may wait on p->stream.  No cudaMalloc,
 * cudaFree or other allocation.
 * Errors (code only, crbm_last_error is not updated): CRBM_EINVAL (bad
 * arguments or parameters, n_chains outside 1..2^30), CRBM_EUNSUPPORTED (needs more scratch than
 * CRBM_NOALLOC_SCRATCH_BYTES), CRBM_ECUDA. */
int crbm_sweep_stream_noalloc(const crbm_params* p, uint32_t* v, int64_t sweep0, int64_t n_sweeps);

/* Message for the last failed call on ctx (or of the last failed
 * crbm_create when ctx is NULL).  Never NULL. */
const char* crbm_last_error(const crbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
