/*
 * crbm_oracle.h — TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, scalar CPU restatement of block Gibbs sampling of the
 * convolutional RBM (CRBM) that encodes the classical Shastry–Sutherland (SS)
 * Ising lattice (Brahma et al., arXiv 2511.20911, Sec. II.A "Mapping to CRBM"
 * and Sec. II.B "Sampling of CRBM").  Only tests/, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
 * library: its bond list, weights, threshold tables, Philox generator and
 * sweep loop are written here from the paper and from the published Philox
 * definition, independently of the library's own.
 *
 * Conventions (the readings of the paper that both sides implement):
 *   - spins and hidden units are +1/-1 (int8); spin bit 1 <-> +1.
 *   - H(s) = J * sum_nn s s + J' * sum_diag s s - h * sum s   (Eq. 1 with the
 *     field sign chosen so that h > 0 favours +1).
 *   - J, J', h are held as signed Q.4 fixed point: q = nearbyint(16 x),
 *     |q| <= 2047; energies in units of 1/16 are then exact integers.
 *   - windows of the stride-2 3x3 filter sit at (2i, 2j), i, j in [0, W),
 *     W = floor((L+1)/2) (the hidden register size of the appendix).
 */
#ifndef CRBM_ORACLE_H
#define CRBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int8_t r1, c1, r2, c2; /* window-relative endpoints, each in [0, 2] */
    uint8_t cls;           /* 0 = J (nearest neighbour), 1 = J' (diagonal) */
} orc_bond;

/* Philox-4x32-10 of Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11: counter ctr[4], key key[2] -> out[4]. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The ten bonds of the SS 3x3 unit cell (8 J bonds then 2 J' diagonals). */
int orc_canonical_bonds(orc_bond out[10]);

/* Q.4 quantisation of a coupling; returns 0, or -1 if out of range / NaN. */
int orc_quantize(double x, int32_t* q);

/* Per-class weight a = 1/2 arccosh(exp(2|K|)), K = -beta * J (Eqs. 5-7), and
 * the sign s of the second endpoint's coefficient (s = +1 iff K >= 0). */
void orc_weight(double beta, double J, double* a, int* s);

/* thr(y) = min(2^32 - 1, nearbyint(2^32 / (1 + exp(-y)))) as uint32. */
uint32_t orc_threshold(double y);

/* Largest number of (cell, bond, endpoint) incidences of class 0 / class 1 on
 * any real site: the visible table spans n_J in [-DJ, DJ], n_J' in [-DJp, DJp]. */
int orc_degrees(int L, int periodic, const orc_bond* bonds, int nb, int* DJ, int* DJp);

/* Threshold tables for one parameter point.
 *   Th[cls*5 + (m+2)] = thr(2 a_cls m),                m in [-2, 2]
 *   Tv[(nJ+DJ)*(2DJp+1) + (nJp+DJp)] = thr(2 x),
 *       x = beta*h + a_J*nJ + a_J'*nJp  (left to right, double). */
int orc_tables(int L, int periodic, const orc_bond* bonds, int nb,
               double J, double Jp, double h, double beta,
               uint32_t* Th, uint32_t* Tv);

/* Uniform +-1 initial spins: site (R, C) of chain c is +1 iff word
 * 2(R&1)+(C&1) of Philox((cell, 0, c, TAG_INIT), seed) < 2^31. */
void orc_init(int L, const uint32_t* chain_ids, int n_chains, uint64_t seed, int8_t* spins);

/* Exact integer counts of one configuration over the bond multiset generated
 * by the windows: NJ = sum over class-0 bonds of s s, NJp likewise, M = sum s. */
void orc_counts(int L, int periodic, const orc_bond* bonds, int nb,
                const int8_t* spins, int64_t* NJ, int64_t* NJp, int64_t* M);

/* Run n_sweeps block-Gibbs sweeps (hidden | visible, then visible | hidden)
 * on each chain, starting at global sweep index sweep0.
 *   params: J, Jp, h, beta arrays of length n_params; chain_param[c] -> p.
 *   chain_ids[c]: global chain index used in the Philox counter.
 *   spins [n_chains][L*L] int8 in/out.
 *   sums [n_chains][11] int64, accumulated (see ORC_SUM_*), may be NULL.
 *   series [n_chains][series_cap][3] int32 (NJ, NJp, M), may be NULL; entry
 *     index = sums[c][0] before the measurement.
 *   sq [n_chains][L*L] double, accumulated S(q) = |sum_r s_r e^{i q.r}|^2 / N
 *     at q = 2 pi (nR, nC) / L, every sq_every sweeps (0 = off), may be NULL.
 * Measurement after sweep t (0-based, global) iff measure_every > 0 and
 * (t + 1) % measure_every == 0.  Returns 0 or a negative error. */
int orc_run(int L, int periodic, const orc_bond* bonds, int nb,
            const double* J, const double* Jp, const double* h, const double* beta,
            int n_params, const int32_t* chain_param, const uint32_t* chain_ids,
            int n_chains, uint64_t seed, int64_t sweep0, int64_t n_sweeps,
            int measure_every, int8_t* spins, int64_t* sums,
            int32_t* series, int64_t series_cap, int sq_every, double* sq);

void orc_set_threads(int n);
int orc_get_threads(void);

/* ---- paper precision (Sec. III, "Dimension and Precision") ----------------
 * The paper's FPGA keeps the convolution weights in 10-bit fixed point (sign,
 * 5 integer and 4 fraction bits), sums them in an accumulator 2 bits wider,
 * maps the sum through a 16-bit sigmoid table and compares it with 16-bit
 * uniform draws.  ORC_PRECISION_PAPER restates that arithmetic:
 *   A_cls = q54(a_cls), B = q54(beta h)   (q54: nearest multiple of 1/16,
 *                                           clamped to +-511/16)
 *   hidden threshold of m:   lut16(A_cls m)
 *   visible threshold:       lut16(B + A_J n_J + A_J' n_J')
 *   lut16(acc) = min(65535, nearbyint(2^16 / (1 + exp(-2 acc / 16)))) << 16,
 *     acc in 1/16 units clamped to the 12-bit range +-2047,
 * so a 32-bit table entry is the 16-bit threshold in its upper half.  Each
 * Philox word carries two 16-bit uniforms, low half first: hidden filter
 * k < 8 takes half k&1 of word k>>1 of tag 0, filters 8 and 9 the halves of
 * word 0 of tag 1, and the spin at window offset (r, c) half (2r+c)&1 of word
 * 1 + ((2r+c)>>1) of tag 1; a unit becomes +1 iff its uniform is below the
 * 16-bit threshold.  Needs at most 10 filters.  The _ex functions take the
 * precision; the others are ORC_PRECISION_EXACT. */
#define ORC_PRECISION_EXACT 0
#define ORC_PRECISION_PAPER 1

/* ---- rectangular lattices, a boundary per axis, odd-column field ----------
 * Sec. III runs laterally confined strips (open boundaries along one axis)
 * and the appendix lets odd and even columns take different visible biases.
 * The _rect functions take Lr rows x Lc columns, pr / pc = 1 for a periodic
 * row (vertical) / column (horizontal) axis, and (for the sampler) h_odd[p],
 * the field of the odd columns (NULL: h on every column).  Windows (i, j),
 * i < (Lr+1)/2, j < (Lc+1)/2; cell index i (Lc+1)/2 + j; spins [R][C] with
 * R < Lr, C < Lc.  The square functions are the _rect ones with Lr = Lc = L,
 * pr = pc = periodic and no odd-column field.  Replica exchange needs equal
 * fields on both column parities (its energies use the total M). */
int orc_degrees_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, int* DJ, int* DJp);
int orc_tables_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, double J, double Jp,
                    double h, double h_odd, double beta, int precision, uint32_t* Th, uint32_t* Tv,
                    uint32_t* Tv_odd);
void orc_init_rect(int Lr, int Lc, const uint32_t* chain_ids, int n_chains, uint64_t seed, int8_t* spins);
void orc_counts_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, const int8_t* v,
                     int64_t* NJ, int64_t* NJp, int64_t* M);
int orc_run_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, const double* J,
                 const double* Jp, const double* h, const double* h_odd, const double* beta, int n_params,
                 const int32_t* chain_param, const uint32_t* chain_ids, int n_chains, uint64_t seed,
                 int64_t sweep0, int64_t n_sweeps, int measure_every, int8_t* spins, int64_t* sums,
                 int32_t* series, int64_t series_cap, int sq_every, double* sq, int precision);
int orc_run_pt_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, const double* J,
                    const double* Jp, const double* h, const double* beta, int n_params,
                    const int32_t* chain_param, int n_chains, uint64_t seed, int64_t sweep0,
                    int64_t n_sweeps, int measure_every, int swap_every, int8_t* spins,
                    int32_t* slot_of_beta, int64_t* sums, int32_t* series, int64_t series_cap,
                    int precision);
int32_t orc_q54(double x);
uint32_t orc_lut16(int32_t acc);
int orc_tables_ex(int L, int periodic, const orc_bond* bonds, int nb,
                  double J, double Jp, double h, double beta, int precision,
                  uint32_t* Th, uint32_t* Tv);
int orc_run_ex(int L, int periodic, const orc_bond* bonds, int nb,
               const double* J, const double* Jp, const double* h, const double* beta,
               int n_params, const int32_t* chain_param, const uint32_t* chain_ids,
               int n_chains, uint64_t seed, int64_t sweep0, int64_t n_sweeps,
               int measure_every, int8_t* spins, int64_t* sums,
               int32_t* series, int64_t series_cap, int sq_every, double* sq, int precision);

/* ---- bit-plane uniforms -----------------------------------------------------
 * A second source of the uniforms, for groups of 32 chains (chain c is bit
 * c % 32 of group c / 32): the uniform of every chain of a group at one node
 * is built from shared bit-plane words, most significant bit first, so that a
 * word-parallel comparison can stop as soon as all 32 decisions are known.
 * The uniform of chain c at node n of cell `cell` in sweep t is
 *   u = sum_b bit (c % 32) of P_b  <<  (31 - b),   b = 0 .. 31,
 * where plane P_(4j+i) is output word i of
 *   Philox((cell, t, c / 32, ORC_TAG_BITPLANE + 8 n + j)),  j = 0 .. 7,
 * and the node of hidden filter k is n = k, the node of the spin at window
 * offset (r, c) is n = 10 + 2r + c.  The unit is +1 iff u < t with the exact
 * thresholds, as in every other mode.  Selected by OR-ing ORC_RNG_BITPLANE
 * into the precision argument of the _ex and _rect samplers (replica exchange
 * included: replica r of ladder l draws as chain 32 l + r, whichever rung it
 * holds); it needs ORC_PRECISION_EXACT and at most 10 filters. */
#define ORC_RNG_BITPLANE 0x10
#define ORC_TAG_BITPLANE 256u

#define ORC_TAG_VIS 4u
#define ORC_TAG_INIT 5u
#define ORC_TAG_SWAP 6u
#define ORC_NSUM 11

#ifdef __cplusplus
}
#endif
#endif

#ifdef __cplusplus
extern "C" {
#endif
/* Parallel tempering (replica exchange) on ladders of 32 chains: chains
 * 32 l .. 32 l + 31 form ladder l.  Chain index 32 l + k of chain_param names
 * the parameter point of temperature rung k (beta strictly increasing in k,
 * equal J, J', h along a ladder).  slot_of_beta[l][k] (in/out) is the replica
 * slot holding rung k; spins are stored per slot and every slot's Gibbs
 * draws use its own chain index 32 l + slot.  After sweep t, if measuring,
 * rung k's configuration is measured into sums / series row 32 l + k; then,
 * if (t + 1) % swap_every == 0 (round m = (t + 1) / swap_every - 1), every
 * pair (k, k+1) with k = m mod 2 (mod 2) exchanges rungs with probability
 * min(1, exp((beta_k - beta_{k+1}) (E_k - E_{k+1}) / 16)), E in 1/16 units:
 * accepted iff E_k <= E_{k+1} or u < nearbyint(2^32 exp(x)), u = word 0 of
 * Philox((k, m, l, ORC_TAG_SWAP)). */
int orc_run_pt(int L, int periodic, const orc_bond* bonds, int nb, const double* J,
               const double* Jp, const double* h, const double* beta, int n_params,
               const int32_t* chain_param, int n_chains, uint64_t seed, int64_t sweep0,
               int64_t n_sweeps, int measure_every, int swap_every, int8_t* spins,
               int32_t* slot_of_beta, int64_t* sums, int32_t* series, int64_t series_cap);
int orc_run_pt_ex(int L, int periodic, const orc_bond* bonds, int nb, const double* J,
                  const double* Jp, const double* h, const double* beta, int n_params,
                  const int32_t* chain_param, int n_chains, uint64_t seed, int64_t sweep0,
                  int64_t n_sweeps, int measure_every, int swap_every, int8_t* spins,
                  int32_t* slot_of_beta, int64_t* sums, int32_t* series, int64_t series_cap,
                  int precision);
uint32_t orc_swap_threshold(double x);
#ifdef __cplusplus
}
#endif

#ifdef __cplusplus
extern "C" {
#endif
/* ---- learned block proposal (test infrastructure) ------------------------
 * A k x k block of spins at origin (bR, bC) is proposed from a small conv net
 * over the (k+6) x (k+6) patch around it (periodic):
 *   input channels: 0 spin (0 inside the block), 1 block mask, 2 row parity,
 *                   3 column parity, 4 beta, 5 h;
 *   three valid 3x3 convolutions 6->16->16->1 with ReLU after the first two,
 *   one logit per block site, q_s = sigmoid(logit) = P(spin s = +1).
 * Parameters (ORC_NET_PARAMS doubles): W1[16][6][3][3], b1[16],
 * W2[16][16][3][3], b2[16], W3[16][3][3], b3.
 * With bf16 != 0, weights and inputs are rounded to bfloat16 (round to
 * nearest even) and so are the two hidden activations (the GPU's storage
 * precision); accumulation is in double.  The proposal draws each site with
 * probability t_s / 2^32, t_s = clamp(nearbyint(q_s 2^32), 1, 2^32 - 1), and
 * the move is accepted with probability
 * min(1, exp(-beta dE / 16) q(x_B) / q(x'_B)) on the exact integer energy
 * difference dE (1/16 units) of the canonical SS lattice (even L, periodic). */
#define ORC_NET_PARAMS 3345
double orc_bf16(double x);
int orc_patch_input(int L, const int8_t* v, int bR, int bC, int k, double beta, double h,
                    double* input);
int orc_net_forward(int k, const double* w, const double* input, int bf16, double* logits);
int orc_net_loss_grad(int k, const double* w, const double* inputs, const int8_t* targets, int n,
                      int bf16, double* loss, double* grad);
int64_t orc_block_delta_e(int L, const int8_t* v, int bR, int bC, int k, const int8_t* newblock,
                          int32_t qJ, int32_t qJp, int32_t qh);
int orc_mh_row(int L, const int8_t* v, int bR, int bC, int k, const double* w, double J,
               double Jp, double h, double beta, int bf16, double* probs);

/* One pass of block moves over n_chains chains, keyed as the library keys
 * it (see orc_prop_pass in crbm_oracle.c for the steps); needs L >= 10. */
#define ORC_TAG_PROP_OFFSET 8u
#define ORC_TAG_PROP_BITS 9u
#define ORC_TAG_PROP_ACCEPT 13u
typedef struct {
    double logit[16];
    uint32_t thr[16];     /* t_s: site s proposes +1 iff its draw < t_s */
    uint32_t draw[16];    /* the Philox draw of site s */
    int32_t bR, bC;       /* block origin */
    uint32_t cur_bits, new_bits;  /* bit s = site (s / 4, s % 4) is +1 */
    int64_t dE;           /* exact energy change of the proposal, 1/16 units */
    double log_alpha, u_accept;
    int32_t accept;
    int32_t pad;
} orc_pass_rec;
int orc_prop_pass(int L, int8_t* v, int n_chains, const double* J, const double* Jp,
                  const double* h, const double* beta, const int32_t* chain_param,
                  const double* w, const double* logits_in, const uint32_t* thr_in,
                  uint64_t seed, uint32_t pass, int apply, orc_pass_rec* rec);

/* S(q) = |sum_r s_r e^{i q.r}|^2 / N of one configuration [Lr][Lc] at
 * q = 2 pi (nR / Lr, nC / Lc), into sq[nR][nC]. */
void orc_structure_factor(int Lr, int Lc, const int8_t* v, double* sq);
#ifdef __cplusplus
}
#endif
