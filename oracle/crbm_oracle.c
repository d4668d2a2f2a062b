/*
 * crbm_oracle.c — TEST INFRASTRUCTURE ONLY (the oracle); see crbm_oracle.h.
 *
 * Plain scalar C, double precision for every real number, int8 +-1 spins and
 * hidden units in [chain][row][col] order, no blocking, no bit packing, no
 * SIMD.  Each function names the passage of arXiv 2511.20911 it restates.
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA contraction,
 * so the table arithmetic is the plain left-to-right double evaluation).
 */
#include "crbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Philox */
/* Salmon et al., SC'11, Sec. 4: Philox-4x32 with R = 10 rounds.  One round
 * multiplies counter words 0 and 2 by the two round multipliers, forming
 * 64-bit products, and permutes/whitens:
 *     (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
 * and between rounds the key is bumped by the Weyl constants (golden ratio
 * and sqrt(3) - 1, as 32-bit fractions). */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_word(uint32_t cell, uint32_t sweep, uint32_t chain, uint32_t tag,
                            uint64_t seed, int word) {
    uint32_t ctr[4] = {cell, sweep, chain, tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------------ lattice */
/* Fig. 1(a) and Sec. II.A: the SS lattice has a 3x3 unit cell holding 8
 * nearest-neighbour (J1) bonds and 2 diagonal (J2) bonds, labelled 0..9 with
 * k in [0,7] the J1 filters and k in {8, 9} the J2 filters.  In window
 * coordinates (row, col): horizontal bonds of rows 0 and 1, vertical bonds of
 * columns 0 and 1, and the two orthogonal dimers: "\" on plaquette (0,0) and
 * "/" on plaquette (1,1).  Tiling the window with stride 2 covers every
 * square-lattice bond once and every site with exactly one diagonal. */
int orc_canonical_bonds(orc_bond out[10]) {
    static const orc_bond b[10] = {
        {0, 0, 0, 1, 0}, {0, 1, 0, 2, 0}, {1, 0, 1, 1, 0}, {1, 1, 1, 2, 0},
        {0, 0, 1, 0, 0}, {1, 0, 2, 0, 0}, {0, 1, 1, 1, 0}, {1, 1, 2, 1, 0},
        {0, 0, 1, 1, 1}, {1, 2, 2, 1, 1},
    };
    memcpy(out, b, sizeof(b));
    return 10;
}

static int n_windows(int L) { return (L + 1) / 2; }

/* A lattice of Lr rows by Lc columns with its own boundary along each axis
 * (Sec. III: the hardware also runs open boundaries along the lateral
 * direction only, for laterally confined strips).  Windows (i, j) with
 * i < (Lr+1)/2, j < (Lc+1)/2; cell index i (Lc+1)/2 + j. */
typedef struct {
    int Lr, Lc, pr, pc;
} orc_geom;

/* Appendix, "Wrapper Module": a periodic axis copies its first rows (columns)
 * past the edge; an open one inserts zeros.  A zero-padded endpoint is a null
 * site (-1) that contributes nothing. */
static int site_g(const orc_geom* g, int i, int j, int r, int c) {
    int R = 2 * i + r, C = 2 * j + c;
    if (R >= g->Lr) {
        if (!g->pr) return -1;
        R %= g->Lr;
    }
    if (C >= g->Lc) {
        if (!g->pc) return -1;
        C %= g->Lc;
    }
    return R * g->Lc + C;
}

static int check_model(int L, const orc_bond* bonds, int nb) {
    if (L < 3 || L > 4096 || nb < 1 || nb > 16) return -1;
    for (int k = 0; k < nb; ++k) {
        const orc_bond* b = &bonds[k];
        if (b->r1 < 0 || b->r1 > 2 || b->c1 < 0 || b->c1 > 2 || b->r2 < 0 || b->r2 > 2 ||
            b->c2 < 0 || b->c2 > 2 || b->cls > 1)
            return -1;
        if (b->r1 == b->r2 && b->c1 == b->c2) return -1;
    }
    return 0;
}

int orc_quantize(double x, int32_t* q) {
    if (!(x == x)) return -1;
    double v = nearbyint(16.0 * x);
    if (v < -2047.0 || v > 2047.0) return -1;
    *q = (int32_t)v;
    return 0;
}

/* ------------------------------------------------------------- weights */
/* Eqs. (4)-(7) (Carleo et al. mapping): exp(K v_i v_j) is reproduced, up to a
 * constant, by a hidden unit h = +-1 coupled with weight a to v_i and s a to
 * v_j, since sum_h exp(a h (v_i + s v_j)) = 2 cosh(a (v_i + s v_j)), whose
 * aligned/anti-aligned ratio is cosh(2a).  Hence cosh(2a) = exp(2|K|),
 * a = 1/2 arccosh(exp(2|K|)), s = sgn(K).  The Boltzmann weight of Eq. (1) is
 * exp(-beta H), so a J bond has K = -beta J (J > 0 antiferromagnetic). */
void orc_weight(double beta, double J, double* a, int* s) {
    double K = -beta * J;
    *a = 0.5 * acosh(exp(2.0 * fabs(K)));
    *s = (K >= 0.0) ? 1 : -1;
}

/* Sigmoid of Eqs. (9)-(10) as an unsigned 32-bit acceptance threshold: a unit
 * becomes +1 iff a uniform 32-bit draw u satisfies u < thr. */
uint32_t orc_threshold(double y) {
    double p = 1.0 / (1.0 + exp(-y));
    double t = nearbyint(ldexp(p, 32));
    if (t > 4294967295.0) t = 4294967295.0;
    if (t < 0.0) t = 0.0;
    return (uint32_t)t;
}

static int degrees_g(const orc_geom* g, const orc_bond* bonds, int nb, int* DJ, int* DJp) {
    if (check_model(g->Lr, bonds, nb) || check_model(g->Lc, bonds, nb)) return -1;
    int Wr = n_windows(g->Lr), Wc = n_windows(g->Lc), N = g->Lr * g->Lc;
    int* deg = (int*)calloc((size_t)2 * N, sizeof(int));
    if (!deg) return -2;
    for (int i = 0; i < Wr; ++i)
        for (int j = 0; j < Wc; ++j)
            for (int k = 0; k < nb; ++k) {
                int s1 = site_g(g, i, j, bonds[k].r1, bonds[k].c1);
                int s2 = site_g(g, i, j, bonds[k].r2, bonds[k].c2);
                if (s1 >= 0) deg[bonds[k].cls * N + s1]++;
                if (s2 >= 0) deg[bonds[k].cls * N + s2]++;
            }
    int m0 = 0, m1 = 0;
    for (int s = 0; s < N; ++s) {
        if (deg[s] > m0) m0 = deg[s];
        if (deg[N + s] > m1) m1 = deg[N + s];
    }
    free(deg);
    *DJ = m0;
    *DJp = m1;
    return 0;
}

int orc_degrees(int L, int periodic, const orc_bond* bonds, int nb, int* DJ, int* DJp) {
    orc_geom g = {L, L, periodic, periodic};
    return degrees_g(&g, bonds, nb, DJ, DJp);
}

int orc_degrees_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, int* DJ, int* DJp) {
    orc_geom g = {Lr, Lc, pr, pc};
    return degrees_g(&g, bonds, nb, DJ, DJp);
}

/* Eq. (9): P(H=1|V) = sigmoid of the forward cross-correlation; with +-1
 * hidden units the hidden conditional is sigmoid(2 a m), m = v1 + s v2.
 * Eq. (10): P(V=1|H) = sigmoid of the zero-padded reverse correlation summed
 * over the filters plus the visible bias; here sigmoid(2 x) with
 * x = beta h + a_J n_J + a_J' n_J'. */
/* Paper precision (Sec. III, "Dimension and Precision"): 10-bit weights with
 * 4 fraction bits, an accumulator 2 bits wider, a 16-bit sigmoid table. */
int32_t orc_q54(double x) {
    double v = nearbyint(16.0 * x);
    if (v > 511.0) v = 511.0;
    if (v < -511.0) v = -511.0;
    return (int32_t)v;
}

uint32_t orc_lut16(int32_t acc) {
    if (acc > 2047) acc = 2047;
    if (acc < -2047) acc = -2047;
    double p = 1.0 / (1.0 + exp(-2.0 * (double)acc / 16.0));
    double t = nearbyint(ldexp(p, 16));
    if (t > 65535.0) t = 65535.0;
    return (uint32_t)t << 16;
}

int orc_tables(int L, int periodic, const orc_bond* bonds, int nb, double J, double Jp,
               double h, double beta, uint32_t* Th, uint32_t* Tv) {
    return orc_tables_ex(L, periodic, bonds, nb, J, Jp, h, beta, ORC_PRECISION_EXACT, Th, Tv);
}

/* Visible table of one field value h (Eq. 10), exact or paper precision. */
static void visible_table(int DJ, int DJp, const double a[2], double beta, double hd, int precision,
                          uint32_t* Tv) {
    int nP = 2 * DJp + 1;
    if (precision == ORC_PRECISION_PAPER) {
        int32_t A[2] = {orc_q54(a[0]), orc_q54(a[1])}, B = orc_q54(beta * hd);
        for (int nJ = -DJ; nJ <= DJ; ++nJ)
            for (int nJp = -DJp; nJp <= DJp; ++nJp)
                Tv[(nJ + DJ) * nP + (nJp + DJp)] = orc_lut16(B + A[0] * nJ + A[1] * nJp);
        return;
    }
    for (int nJ = -DJ; nJ <= DJ; ++nJ)
        for (int nJp = -DJp; nJp <= DJp; ++nJp) {
            double x = beta * hd + a[0] * nJ + a[1] * nJp;
            Tv[(nJ + DJ) * nP + (nJp + DJp)] = orc_threshold(2.0 * x);
        }
}

/* Tables of one parameter point; Tv_odd (may be NULL) is the visible table of
 * the odd columns, whose field is h_odd (the appendix's option of separate
 * odd- and even-column visible biases). */
static int tables_g(const orc_geom* g, const orc_bond* bonds, int nb, double J, double Jp, double h,
                    double h_odd, double beta, int precision, uint32_t* Th, uint32_t* Tv, uint32_t* Tv_odd) {
    int DJ, DJp;
    if (precision != ORC_PRECISION_EXACT && precision != ORC_PRECISION_PAPER) return -1;
    if (precision == ORC_PRECISION_PAPER && nb > 10) return -1;
    if (degrees_g(g, bonds, nb, &DJ, &DJp)) return -1;
    int32_t qJ, qJp, qh, qho;
    if (orc_quantize(J, &qJ) || orc_quantize(Jp, &qJp) || orc_quantize(h, &qh) || orc_quantize(h_odd, &qho))
        return -1;
    if (!(beta >= 0.0) || beta > 1.0e6) return -1;
    double Jd = qJ / 16.0, Jpd = qJp / 16.0, hd = qh / 16.0;
    double a[2];
    int s[2];
    orc_weight(beta, Jd, &a[0], &s[0]);
    orc_weight(beta, Jpd, &a[1], &s[1]);
    if (precision == ORC_PRECISION_PAPER) {
        int32_t A[2] = {orc_q54(a[0]), orc_q54(a[1])};
        for (int cls = 0; cls < 2; ++cls)
            for (int m = -2; m <= 2; ++m) Th[cls * 5 + (m + 2)] = orc_lut16(A[cls] * m);
    } else {
        for (int cls = 0; cls < 2; ++cls)
            for (int m = -2; m <= 2; ++m) Th[cls * 5 + (m + 2)] = orc_threshold(2.0 * a[cls] * m);
    }
    visible_table(DJ, DJp, a, beta, hd, precision, Tv);
    if (Tv_odd) visible_table(DJ, DJp, a, beta, qho / 16.0, precision, Tv_odd);
    return 0;
}

int orc_tables_ex(int L, int periodic, const orc_bond* bonds, int nb, double J, double Jp,
                  double h, double beta, int precision, uint32_t* Th, uint32_t* Tv) {
    orc_geom g = {L, L, periodic, periodic};
    return tables_g(&g, bonds, nb, J, Jp, h, h, beta, precision, Th, Tv, NULL);
}

int orc_tables_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, double J, double Jp,
                    double h, double h_odd, double beta, int precision, uint32_t* Th, uint32_t* Tv,
                    uint32_t* Tv_odd) {
    orc_geom g = {Lr, Lc, pr, pc};
    return tables_g(&g, bonds, nb, J, Jp, h, h_odd, beta, precision, Th, Tv, Tv_odd);
}

/* ------------------------------------------------------ configuration */
void orc_init_rect(int Lr, int Lc, const uint32_t* chain_ids, int n_chains, uint64_t seed, int8_t* spins) {
    int Wc = n_windows(Lc);
    for (int c = 0; c < n_chains; ++c)
        for (int R = 0; R < Lr; ++R)
            for (int C = 0; C < Lc; ++C) {
                uint32_t cell = (uint32_t)((R >> 1) * Wc + (C >> 1));
                uint32_t u = philox_word(cell, 0u, chain_ids[c], ORC_TAG_INIT, seed,
                                         2 * (R & 1) + (C & 1));
                spins[(size_t)c * Lr * Lc + R * Lc + C] = (u < 0x80000000u) ? 1 : -1;
            }
}

void orc_init(int L, const uint32_t* chain_ids, int n_chains, uint64_t seed, int8_t* spins) {
    orc_init_rect(L, L, chain_ids, n_chains, seed, spins);
}

/* Eq. (1) on the bond multiset generated by the stride-2 windows. */
static void counts_g(const orc_geom* g, const orc_bond* bonds, int nb, const int8_t* v, int64_t* NJ,
                     int64_t* NJp, int64_t* M) {
    int Wr = n_windows(g->Lr), Wc = n_windows(g->Lc);
    int64_t n[2] = {0, 0}, m = 0;
    for (int i = 0; i < Wr; ++i)
        for (int j = 0; j < Wc; ++j)
            for (int k = 0; k < nb; ++k) {
                int s1 = site_g(g, i, j, bonds[k].r1, bonds[k].c1);
                int s2 = site_g(g, i, j, bonds[k].r2, bonds[k].c2);
                if (s1 < 0 || s2 < 0) continue;
                n[bonds[k].cls] += v[s1] * v[s2];
            }
    for (int s = 0; s < g->Lr * g->Lc; ++s) m += v[s];
    *NJ = n[0];
    *NJp = n[1];
    *M = m;
}

void orc_counts(int L, int periodic, const orc_bond* bonds, int nb, const int8_t* v,
                int64_t* NJ, int64_t* NJp, int64_t* M) {
    orc_geom g = {L, L, periodic, periodic};
    counts_g(&g, bonds, nb, v, NJ, NJp, M);
}

void orc_counts_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, const int8_t* v,
                     int64_t* NJ, int64_t* NJp, int64_t* M) {
    orc_geom g = {Lr, Lc, pr, pc};
    counts_g(&g, bonds, nb, v, NJ, NJp, M);
}

/* Sec. IV.B, Eq. (11): S(q) = sum_ij <s_i s_j> e^{i q.(R_i - R_j)}, reported
 * per spin: |sum_r s_r e^{i q.r}|^2 / N at q = 2 pi (nR, nC) / L. */
static void add_structure_factor(int Lr, int Lc, const int8_t* v, double* sq) {
    const double twopi = 6.283185307179586476925286766559;
    int N = Lr * Lc;
    for (int nR = 0; nR < Lr; ++nR)
        for (int nC = 0; nC < Lc; ++nC) {
            double re = 0.0, im = 0.0;
            for (int R = 0; R < Lr; ++R)
                for (int C = 0; C < Lc; ++C) {
                    double ph = twopi * ((double)(nR * R) / (double)Lr + (double)(nC * C) / (double)Lc);
                    re += v[R * Lc + C] * cos(ph);
                    im += v[R * Lc + C] * sin(ph);
                }
            sq[nR * Lc + nC] += (re * re + im * im) / (double)N;
        }
}

/* S(q) of one configuration alone (sq overwritten), the function the sampler
 * accumulates every sq_every sweeps. */
void orc_structure_factor(int Lr, int Lc, const int8_t* v, double* sq) {
    for (int i = 0; i < Lr * Lc; ++i) sq[i] = 0.0;
    add_structure_factor(Lr, Lc, v, sq);
}

/* ------------------------------------------------------------ sampling */
typedef struct {
    uint32_t Th[10];
    uint32_t* Tv;
    uint32_t* Tv_odd;  /* visible table of the odd columns */
    int s[2];
    int paper;  /* ORC_PRECISION_PAPER: 16-bit uniforms and thresholds */
    int bitplane; /* ORC_RNG_BITPLANE: uniforms from shared bit-plane words */
} orc_point;

/* The bit-plane uniform of chain `chain` at node `node` of cell `cell` (see
 * ORC_RNG_BITPLANE in crbm_oracle.h): all 32 planes of its 32-chain group,
 * bit chain % 32 of each, most significant first. */
static uint32_t bitplane_uniform(uint32_t cell, uint32_t sweep, uint32_t chain, int node, uint64_t seed) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t u = 0;
    for (int j = 0; j < 8; ++j) {
        uint32_t ctr[4] = {cell, sweep, chain / 32u, ORC_TAG_BITPLANE + 8u * (uint32_t)node + (uint32_t)j};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        for (int i = 0; i < 4; ++i) {
            const int b = 4 * j + i;
            u |= ((out[i] >> (chain % 32u)) & 1u) << (31 - b);
        }
    }
    return u;
}

/* One unit's decision.  Exact precision: word w of Philox((cell, sweep,
 * chain, tag)) against the 32-bit threshold.  Paper precision: the 16-bit
 * uniform in half `half` of that word against the threshold's upper half. */
static int draw_below(const orc_point* pt, uint32_t cell, uint32_t sweep, uint32_t chain,
                      uint32_t tag, int word, int half, uint64_t seed, uint32_t t) {
    uint32_t u = philox_word(cell, sweep, chain, tag, seed, word);
    if (!pt->paper) return u < t;
    uint32_t u16 = half ? (u >> 16) : (u & 0xffffu);
    return u16 < (t >> 16);
}

/* Sec. II.B and Fig. 1(d): one sweep = every hidden unit drawn from Eq. (9)
 * given the current spins, then every spin drawn from Eq. (10) given those
 * hidden units.  The Philox counter (cell, sweep, chain, tag) fixes every draw:
 * hidden bond k of cell (i, j) uses word k&3 of tag k>>2; the spin at
 * window offset (r, c) uses word 2r+c of tag ORC_TAG_VIS. */
static void one_sweep(const orc_geom* g, const orc_bond* bonds, int nb, const orc_point* pt,
                      int DJ, int DJp, uint32_t chain, uint32_t sweep, uint64_t seed, int8_t* v,
                      int8_t* hid, int* field) {
    int Wr = n_windows(g->Lr), Wc = n_windows(g->Lc), N = g->Lr * g->Lc;
    /* hidden | visible */
    for (int i = 0; i < Wr; ++i)
        for (int j = 0; j < Wc; ++j) {
            uint32_t cell = (uint32_t)(i * Wc + j);
            for (int k = 0; k < nb; ++k) {
                const orc_bond* b = &bonds[k];
                int s1 = site_g(g, i, j, b->r1, b->c1);
                int s2 = site_g(g, i, j, b->r2, b->c2);
                int m = (s1 >= 0 ? v[s1] : 0) + pt->s[b->cls] * (s2 >= 0 ? v[s2] : 0);
                uint32_t t = pt->Th[b->cls * 5 + (m + 2)];
                int up;
                if (pt->bitplane)
                    up = bitplane_uniform(cell, sweep, chain, k, seed) < t;
                else if (!pt->paper)
                    up = draw_below(pt, cell, sweep, chain, (uint32_t)(k >> 2), k & 3, 0, seed, t);
                else if (k < 8)
                    up = draw_below(pt, cell, sweep, chain, 0u, k >> 1, k & 1, seed, t);
                else
                    up = draw_below(pt, cell, sweep, chain, 1u, 0, k & 1, seed, t);
                hid[cell * nb + k] = up ? 1 : -1;
            }
        }
    /* visible | hidden: zero-padded reverse correlation = scatter of every
     * hidden unit onto its two endpoints with coefficients (+1, s). */
    memset(field, 0, sizeof(int) * 2 * N);
    for (int i = 0; i < Wr; ++i)
        for (int j = 0; j < Wc; ++j) {
            int cell = i * Wc + j;
            for (int k = 0; k < nb; ++k) {
                const orc_bond* b = &bonds[k];
                int s1 = site_g(g, i, j, b->r1, b->c1);
                int s2 = site_g(g, i, j, b->r2, b->c2);
                int hv = hid[cell * nb + k];
                if (s1 >= 0) field[b->cls * N + s1] += hv;
                if (s2 >= 0) field[b->cls * N + s2] += pt->s[b->cls] * hv;
            }
        }
    int nP = 2 * DJp + 1;
    for (int R = 0; R < g->Lr; ++R)
        for (int C = 0; C < g->Lc; ++C) {
            int s = R * g->Lc + C;
            uint32_t cell = (uint32_t)((R >> 1) * Wc + (C >> 1));
            int x = 2 * (R & 1) + (C & 1);
            const uint32_t* Tv = (C & 1) ? pt->Tv_odd : pt->Tv;
            uint32_t t = Tv[(field[s] + DJ) * nP + (field[N + s] + DJp)];
            int up = pt->bitplane ? bitplane_uniform(cell, sweep, chain, 10 + x, seed) < t
                     : pt->paper  ? draw_below(pt, cell, sweep, chain, 1u, 1 + (x >> 1), x & 1, seed, t)
                                  : draw_below(pt, cell, sweep, chain, ORC_TAG_VIS, x, 0, seed, t);
            v[s] = up ? 1 : -1;
        }
}

int orc_run(int L, int periodic, const orc_bond* bonds, int nb, const double* J, const double* Jp,
            const double* h, const double* beta, int n_params, const int32_t* chain_param,
            const uint32_t* chain_ids, int n_chains, uint64_t seed, int64_t sweep0,
            int64_t n_sweeps, int measure_every, int8_t* spins, int64_t* sums, int32_t* series,
            int64_t series_cap, int sq_every, double* sq) {
    return orc_run_ex(L, periodic, bonds, nb, J, Jp, h, beta, n_params, chain_param, chain_ids,
                      n_chains, seed, sweep0, n_sweeps, measure_every, spins, sums, series,
                      series_cap, sq_every, sq, ORC_PRECISION_EXACT);
}

static int run_g(const orc_geom* g, const orc_bond* bonds, int nb, const double* J, const double* Jp,
                 const double* h, const double* h_odd, const double* beta, int n_params,
                 const int32_t* chain_param, const uint32_t* chain_ids, int n_chains, uint64_t seed,
                 int64_t sweep0, int64_t n_sweeps, int measure_every, int8_t* spins, int64_t* sums,
                 int32_t* series, int64_t series_cap, int sq_every, double* sq, int precision) {
    const int bitplane = (precision & ORC_RNG_BITPLANE) != 0;
    precision &= ~ORC_RNG_BITPLANE;
    if (bitplane && (precision != ORC_PRECISION_EXACT || nb > 10)) return -1;
    int DJ, DJp;
    if (degrees_g(g, bonds, nb, &DJ, &DJp)) return -1;
    if (n_params < 1 || n_chains < 0 || n_sweeps < 0 || sweep0 < 0 ||
        sweep0 + n_sweeps > 4294967295LL || measure_every < 0 || sq_every < 0)
        return -1;
    for (int c = 0; c < n_chains; ++c)
        if (chain_param[c] < 0 || chain_param[c] >= n_params) return -1;
    int nTv = (2 * DJ + 1) * (2 * DJp + 1);
    orc_point* pts = (orc_point*)calloc((size_t)n_params, sizeof(orc_point));
    uint32_t* tv = (uint32_t*)calloc((size_t)n_params * nTv * 2, sizeof(uint32_t));
    if (!pts || !tv) {
        free(pts);
        free(tv);
        return -2;
    }
    int err = 0;
    for (int p = 0; p < n_params; ++p) {
        pts[p].Tv = tv + (size_t)p * 2 * nTv;
        pts[p].Tv_odd = pts[p].Tv + nTv;
        pts[p].paper = precision == ORC_PRECISION_PAPER;
        pts[p].bitplane = bitplane;
        if (tables_g(g, bonds, nb, J[p], Jp[p], h[p], h_odd ? h_odd[p] : h[p], beta[p], precision, pts[p].Th,
                     pts[p].Tv, pts[p].Tv_odd))
            err = -1;
        int32_t q;
        double a;
        orc_quantize(J[p], &q);
        orc_weight(beta[p], q / 16.0, &a, &pts[p].s[0]);
        orc_quantize(Jp[p], &q);
        orc_weight(beta[p], q / 16.0, &a, &pts[p].s[1]);
    }
    if (err) {
        free(pts);
        free(tv);
        return -1;
    }
    int N = g->Lr * g->Lc;
    int n_cells = n_windows(g->Lr) * n_windows(g->Lc);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < n_chains; ++c) {
        int8_t* v = spins + (size_t)c * N;
        int8_t* hid = (int8_t*)malloc((size_t)n_cells * nb);
        int* field = (int*)malloc(sizeof(int) * 2 * N);
        const orc_point* pt = &pts[chain_param[c]];
        for (int64_t t = sweep0; t < sweep0 + n_sweeps; ++t) {
            one_sweep(g, bonds, nb, pt, DJ, DJp, chain_ids[c], (uint32_t)t, seed, v, hid, field);
            if (measure_every > 0 && (t + 1) % measure_every == 0 && sums) {
                int64_t nJ, nJp, M;
                counts_g(g, bonds, nb, v, &nJ, &nJp, &M);
                int64_t* s = sums + (size_t)c * ORC_NSUM;
                if (series && s[0] < series_cap) {
                    int32_t* e = series + ((size_t)c * series_cap + s[0]) * 3;
                    e[0] = (int32_t)nJ;
                    e[1] = (int32_t)nJp;
                    e[2] = (int32_t)M;
                }
                s[0] += 1;
                s[1] += nJ;
                s[2] += nJp;
                s[3] += M;
                s[4] += M < 0 ? -M : M;
                s[5] += nJ * nJ;
                s[6] += nJp * nJp;
                s[7] += M * M;
                s[8] += nJ * nJp;
                s[9] += nJ * M;
                s[10] += nJp * M;
            }
            if (sq_every > 0 && (t + 1) % sq_every == 0 && sq)
                add_structure_factor(g->Lr, g->Lc, v, sq + (size_t)c * N);
        }
        free(hid);
        free(field);
    }
    free(pts);
    free(tv);
    return 0;
}

int orc_run_ex(int L, int periodic, const orc_bond* bonds, int nb, const double* J,
               const double* Jp, const double* h, const double* beta, int n_params,
               const int32_t* chain_param, const uint32_t* chain_ids, int n_chains, uint64_t seed,
               int64_t sweep0, int64_t n_sweeps, int measure_every, int8_t* spins, int64_t* sums,
               int32_t* series, int64_t series_cap, int sq_every, double* sq, int precision) {
    orc_geom g = {L, L, periodic, periodic};
    return run_g(&g, bonds, nb, J, Jp, h, NULL, beta, n_params, chain_param, chain_ids, n_chains, seed, sweep0,
                 n_sweeps, measure_every, spins, sums, series, series_cap, sq_every, sq, precision);
}

int orc_run_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, const double* J,
                 const double* Jp, const double* h, const double* h_odd, const double* beta, int n_params,
                 const int32_t* chain_param, const uint32_t* chain_ids, int n_chains, uint64_t seed,
                 int64_t sweep0, int64_t n_sweeps, int measure_every, int8_t* spins, int64_t* sums,
                 int32_t* series, int64_t series_cap, int sq_every, double* sq, int precision) {
    orc_geom g = {Lr, Lc, pr, pc};
    return run_g(&g, bonds, nb, J, Jp, h, h_odd, beta, n_params, chain_param, chain_ids, n_chains, seed, sweep0,
                 n_sweeps, measure_every, spins, sums, series, series_cap, sq_every, sq, precision);
}

/* ------------------------------------------------- parallel tempering */
/* Replica exchange between adjacent rungs of a temperature ladder (the
 * paper's introduction lists parallel tempering among the Monte Carlo
 * remedies for trapping); see orc_run_pt in crbm_oracle.h. */
uint32_t orc_swap_threshold(double x) {
    double t = nearbyint(ldexp(exp(x), 32));
    if (t > 4294967295.0) t = 4294967295.0;
    if (t < 0.0) t = 0.0;
    return (uint32_t)t;
}

int orc_run_pt(int L, int periodic, const orc_bond* bonds, int nb, const double* J,
               const double* Jp, const double* h, const double* beta, int n_params,
               const int32_t* chain_param, int n_chains, uint64_t seed, int64_t sweep0,
               int64_t n_sweeps, int measure_every, int swap_every, int8_t* spins,
               int32_t* slot_of_beta, int64_t* sums, int32_t* series, int64_t series_cap) {
    return orc_run_pt_ex(L, periodic, bonds, nb, J, Jp, h, beta, n_params, chain_param, n_chains,
                         seed, sweep0, n_sweeps, measure_every, swap_every, spins, slot_of_beta, sums,
                         series, series_cap, ORC_PRECISION_EXACT);
}

static int run_pt_g(const orc_geom* g, const orc_bond* bonds, int nb, const double* J,
                    const double* Jp, const double* h, const double* beta, int n_params,
                    const int32_t* chain_param, int n_chains, uint64_t seed, int64_t sweep0,
                    int64_t n_sweeps, int measure_every, int swap_every, int8_t* spins,
                    int32_t* slot_of_beta, int64_t* sums, int32_t* series, int64_t series_cap,
                    int precision) {
    if (n_chains <= 0 || n_chains % 32 || swap_every <= 0 || measure_every < 0) return -1;
    const int bitplane = (precision & ORC_RNG_BITPLANE) != 0;  /* replica r draws as chain 32 l + r */
    precision &= ~ORC_RNG_BITPLANE;
    if (bitplane && (precision != ORC_PRECISION_EXACT || nb > 10)) return -1;
    int n_lad = n_chains / 32, N = g->Lr * g->Lc;
    for (int l = 0; l < n_lad; ++l) {
        const int32_t* cp = chain_param + 32 * l;
        for (int k = 0; k < 32; ++k) {
            if (cp[k] < 0 || cp[k] >= n_params) return -1;
            if (J[cp[k]] != J[cp[0]] || Jp[cp[k]] != Jp[cp[0]] || h[cp[k]] != h[cp[0]]) return -1;
            if (k > 0 && !(beta[cp[k]] > beta[cp[k - 1]])) return -1;
        }
    }
    int DJ, DJp;
    if (degrees_g(g, bonds, nb, &DJ, &DJp)) return -1;
    int nTv = (2 * DJ + 1) * (2 * DJp + 1);
    orc_point* pts = (orc_point*)calloc((size_t)n_params, sizeof(orc_point));
    uint32_t* tv = (uint32_t*)calloc((size_t)n_params * nTv, sizeof(uint32_t));
    if (!pts || !tv) {
        free(pts);
        free(tv);
        return -2;
    }
    int err = 0;
    for (int p = 0; p < n_params; ++p) {
        pts[p].Tv = tv + (size_t)p * nTv;
        pts[p].paper = precision == ORC_PRECISION_PAPER;
        pts[p].bitplane = bitplane;
        pts[p].Tv_odd = pts[p].Tv;
        if (tables_g(g, bonds, nb, J[p], Jp[p], h[p], h[p], beta[p], precision, pts[p].Th, pts[p].Tv, NULL))
            err = 1;
        int32_t qq;
        double a;
        orc_quantize(J[p], &qq);
        orc_weight(beta[p], qq / 16.0, &a, &pts[p].s[0]);
        orc_quantize(Jp[p], &qq);
        orc_weight(beta[p], qq / 16.0, &a, &pts[p].s[1]);
    }
    if (err) {
        free(pts);
        free(tv);
        return -1;
    }
    int n_cells = n_windows(g->Lr) * n_windows(g->Lc);
#pragma omp parallel for schedule(dynamic, 1)
    for (int l = 0; l < n_lad; ++l) {
        int8_t* hid = (int8_t*)malloc((size_t)n_cells * nb);
        int* field = (int*)malloc(sizeof(int) * 2 * N);
        const int32_t* cp = chain_param + 32 * l;
        int32_t* sob = slot_of_beta + 32 * l;
        int32_t q[3];
        orc_quantize(J[cp[0]], &q[0]);
        orc_quantize(Jp[cp[0]], &q[1]);
        orc_quantize(h[cp[0]], &q[2]);
        for (int64_t t = sweep0; t < sweep0 + n_sweeps; ++t) {
            int bos[32];
            for (int k = 0; k < 32; ++k) bos[sob[k]] = k;
            for (int r = 0; r < 32; ++r)
                one_sweep(g, bonds, nb, &pts[cp[bos[r]]], DJ, DJp, (uint32_t)(32 * l + r),
                          (uint32_t)t, seed, spins + (size_t)(32 * l + r) * N, hid, field);
            int64_t nJ[32], nP[32], M[32], E[32];
            for (int r = 0; r < 32; ++r) {
                counts_g(g, bonds, nb, spins + (size_t)(32 * l + r) * N, &nJ[r], &nP[r], &M[r]);
                E[r] = (int64_t)q[0] * nJ[r] + (int64_t)q[1] * nP[r] - (int64_t)q[2] * M[r];
            }
            if (measure_every > 0 && (t + 1) % measure_every == 0 && sums) {
                for (int k = 0; k < 32; ++k) {
                    const int r = sob[k];
                    int64_t* s = sums + (size_t)(32 * l + k) * ORC_NSUM;
                    if (series && s[0] < series_cap) {
                        int32_t* e = series + ((size_t)(32 * l + k) * series_cap + s[0]) * 3;
                        e[0] = (int32_t)nJ[r];
                        e[1] = (int32_t)nP[r];
                        e[2] = (int32_t)M[r];
                    }
                    s[0] += 1;
                    s[1] += nJ[r];
                    s[2] += nP[r];
                    s[3] += M[r];
                    s[4] += M[r] < 0 ? -M[r] : M[r];
                    s[5] += nJ[r] * nJ[r];
                    s[6] += nP[r] * nP[r];
                    s[7] += M[r] * M[r];
                    s[8] += nJ[r] * nP[r];
                    s[9] += nJ[r] * M[r];
                    s[10] += nP[r] * M[r];
                }
            }
            if ((t + 1) % swap_every == 0) {
                const int64_t m = (t + 1) / swap_every - 1;
                for (int k = (int)(m & 1); k < 31; k += 2) {
                    const int64_t D = E[sob[k]] - E[sob[k + 1]];
                    int accept = D <= 0;
                    if (!accept) {
                        const double x = (beta[cp[k]] - beta[cp[k + 1]]) * (double)D / 16.0;
                        uint32_t ctr[4] = {(uint32_t)k, (uint32_t)m, (uint32_t)l, ORC_TAG_SWAP};
                        uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
                        uint32_t out[4];
                        orc_philox4x32_10(ctr, key, out);
                        accept = out[0] < orc_swap_threshold(x);
                    }
                    if (accept) {
                        const int32_t tmp = sob[k];
                        sob[k] = sob[k + 1];
                        sob[k + 1] = tmp;
                    }
                }
            }
        }
        free(hid);
        free(field);
    }
    free(pts);
    free(tv);
    return 0;
}

int orc_run_pt_ex(int L, int periodic, const orc_bond* bonds, int nb, const double* J,
                  const double* Jp, const double* h, const double* beta, int n_params,
                  const int32_t* chain_param, int n_chains, uint64_t seed, int64_t sweep0,
                  int64_t n_sweeps, int measure_every, int swap_every, int8_t* spins,
                  int32_t* slot_of_beta, int64_t* sums, int32_t* series, int64_t series_cap,
                  int precision) {
    orc_geom g = {L, L, periodic, periodic};
    return run_pt_g(&g, bonds, nb, J, Jp, h, beta, n_params, chain_param, n_chains, seed, sweep0, n_sweeps,
                    measure_every, swap_every, spins, slot_of_beta, sums, series, series_cap, precision);
}

int orc_run_pt_rect(int Lr, int Lc, int pr, int pc, const orc_bond* bonds, int nb, const double* J,
                    const double* Jp, const double* h, const double* beta, int n_params,
                    const int32_t* chain_param, int n_chains, uint64_t seed, int64_t sweep0,
                    int64_t n_sweeps, int measure_every, int swap_every, int8_t* spins,
                    int32_t* slot_of_beta, int64_t* sums, int32_t* series, int64_t series_cap,
                    int precision) {
    orc_geom g = {Lr, Lc, pr, pc};
    return run_pt_g(&g, bonds, nb, J, Jp, h, beta, n_params, chain_param, n_chains, seed, sweep0, n_sweeps,
                    measure_every, swap_every, spins, slot_of_beta, sums, series, series_cap, precision);
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------ learned block proposal */
/* bfloat16 rounding as the GPU applies it to fp32 values: x is first rounded
 * to float (exact for every float-valued x), then to the nearest bfloat16
 * (8 significant bits), ties to even; infinities and NaN pass through. */
double orc_bf16(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf / nan */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* Input planes of the (k+6)^2 patch around block (bR, bC); input[c][P]. */
int orc_patch_input(int L, const int8_t* v, int bR, int bC, int k, double beta, double h,
                    double* input) {
    int P = k + 6;
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            int R = ((bR - 3 + a) % L + L) % L, C = ((bC - 3 + b) % L + L) % L;
            int dR = ((R - bR) % L + L) % L, dC = ((C - bC) % L + L) % L;
            int inside = dR < k && dC < k;
            int x = a * P + b;
            input[0 * P * P + x] = inside ? 0.0 : (double)v[R * L + C];
            input[1 * P * P + x] = inside ? 1.0 : 0.0;
            input[2 * P * P + x] = (double)(R & 1);
            input[3 * P * P + x] = (double)(C & 1);
            input[4 * P * P + x] = beta;
            input[5 * P * P + x] = h;
        }
    return 0;
}

/* One valid 3x3 convolution: out[o][y][x] = b[o] + sum_c,ky,kx W[o][c][ky][kx]
 * in[c][y+ky][x+kx], in of side S, out of side S - 2. */
static void conv3(const double* W, const double* b, int cin, int cout, int S, const double* in,
                  double* out) {
    int T = S - 2;
    for (int o = 0; o < cout; ++o)
        for (int y = 0; y < T; ++y)
            for (int x = 0; x < T; ++x) {
                double acc = b[o];
                for (int c = 0; c < cin; ++c)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx)
                            acc += W[((o * cin + c) * 3 + ky) * 3 + kx] * in[(c * S + y + ky) * S + x + kx];
                out[(o * T + y) * T + x] = acc;
            }
}

typedef struct {
    double w[ORC_NET_PARAMS];
} orc_net;

static void net_weights(const double* w, int bf16, double* out) {
    for (int i = 0; i < ORC_NET_PARAMS; ++i) out[i] = bf16 ? orc_bf16(w[i]) : w[i];
}

/* Forward pass keeping the activations: z1, a1 [16][(k+4)^2], z2, a2 [16][(k+2)^2]. */
static void net_forward_full(int k, const double* wr, const double* input, int bf16, double* in_r,
                             double* z1, double* a1, double* z2, double* a2, double* logits) {
    int P = k + 6, S1 = k + 4, S2 = k + 2;
    const double *W1 = wr, *b1 = wr + 864, *W2 = wr + 880, *b2 = wr + 3184, *W3 = wr + 3200,
                 *b3 = wr + 3344;
    for (int i = 0; i < 6 * P * P; ++i) in_r[i] = bf16 ? orc_bf16(input[i]) : input[i];
    conv3(W1, b1, 6, 16, P, in_r, z1);
    for (int i = 0; i < 16 * S1 * S1; ++i) {
        double r = z1[i] > 0.0 ? z1[i] : 0.0;
        a1[i] = bf16 ? orc_bf16(r) : r;
    }
    conv3(W2, b2, 16, 16, S1, a1, z2);
    for (int i = 0; i < 16 * S2 * S2; ++i) {
        double r = z2[i] > 0.0 ? z2[i] : 0.0;
        a2[i] = bf16 ? orc_bf16(r) : r;
    }
    conv3(W3, b3, 16, 1, S2, a2, logits);
}

int orc_net_forward(int k, const double* w, const double* input, int bf16, double* logits) {
    if (k < 1 || k > 8) return -1;
    int P = k + 6, S1 = k + 4, S2 = k + 2;
    double* buf = (double*)malloc(sizeof(double) * (ORC_NET_PARAMS + 6 * P * P + 32 * S1 * S1 + 32 * S2 * S2));
    if (!buf) return -2;
    double* wr = buf;
    double* in_r = wr + ORC_NET_PARAMS;
    double* z1 = in_r + 6 * P * P;
    double* a1 = z1 + 16 * S1 * S1;
    double* z2 = a1 + 16 * S1 * S1;
    double* a2 = z2 + 16 * S2 * S2;
    net_weights(w, bf16, wr);
    net_forward_full(k, wr, input, bf16, in_r, z1, a1, z2, a2, logits);
    free(buf);
    return 0;
}

/* Mean binary cross-entropy of q = sigmoid(logit) against the block bits
 * (target +1 -> 1) over n examples, and its gradient with respect to the
 * parameters by back-propagation (the bf16 roundings pass gradients
 * straight through). */
int orc_net_loss_grad(int k, const double* w, const double* inputs, const int8_t* targets, int n,
                      int bf16, double* loss, double* grad) {
    if (k < 1 || k > 8 || n < 1) return -1;
    int P = k + 6, S1 = k + 4, S2 = k + 2, K2 = k * k;
    size_t need = ORC_NET_PARAMS + 6 * P * P + 64 * S1 * S1 + 64 * S2 * S2 + 2 * K2;
    double* buf = (double*)calloc(need, sizeof(double));
    if (!buf) return -2;
    double* wr = buf;
    double* in_r = wr + ORC_NET_PARAMS;
    double* z1 = in_r + 6 * P * P;
    double* a1 = z1 + 16 * S1 * S1;
    double* d1 = a1 + 16 * S1 * S1;
    double* z2 = d1 + 16 * S1 * S1;
    double* a2 = z2 + 16 * S2 * S2;
    double* d2 = a2 + 16 * S2 * S2;
    double* logit = d2 + 16 * S2 * S2;
    double* dl = logit + K2;
    net_weights(w, bf16, wr);
    const double *W2 = wr + 880, *W3 = wr + 3200;
    for (int i = 0; i < ORC_NET_PARAMS; ++i) grad[i] = 0.0;
    double L_sum = 0.0;
    for (int e = 0; e < n; ++e) {
        net_forward_full(k, wr, inputs + (size_t)e * 6 * P * P, bf16, in_r, z1, a1, z2, a2, logit);
        for (int s = 0; s < K2; ++s) {
            double y = targets[(size_t)e * K2 + s] > 0 ? 1.0 : 0.0;
            double z = logit[s];
            /* BCE(sigmoid(z), y) = softplus(z) - y z, evaluated stably */
            double sp = z > 0 ? z + log1p(exp(-z)) : log1p(exp(z));
            L_sum += sp - y * z;
            dl[s] = (1.0 / (1.0 + exp(-z)) - y) / ((double)n * K2);
        }
        /* layer 3 */
        for (int s = 0; s < K2; ++s) {
            int y = s / k, x = s % k;
            grad[3344] += dl[s];
            for (int c = 0; c < 16; ++c)
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx)
                        grad[3200 + (c * 3 + ky) * 3 + kx] += dl[s] * a2[(c * S2 + y + ky) * S2 + x + kx];
        }
        for (int i = 0; i < 16 * S2 * S2; ++i) d2[i] = 0.0;
        for (int s = 0; s < K2; ++s) {
            int y = s / k, x = s % k;
            for (int c = 0; c < 16; ++c)
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx)
                        d2[(c * S2 + y + ky) * S2 + x + kx] += dl[s] * W3[(c * 3 + ky) * 3 + kx];
        }
        for (int i = 0; i < 16 * S2 * S2; ++i)
            if (!(z2[i] > 0.0)) d2[i] = 0.0;
        /* layer 2 */
        for (int o = 0; o < 16; ++o)
            for (int y = 0; y < S2; ++y)
                for (int x = 0; x < S2; ++x) {
                    double g = d2[(o * S2 + y) * S2 + x];
                    if (g == 0.0) continue;
                    grad[3184 + o] += g;
                    for (int c = 0; c < 16; ++c)
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx)
                                grad[880 + ((o * 16 + c) * 3 + ky) * 3 + kx] += g * a1[(c * S1 + y + ky) * S1 + x + kx];
                }
        for (int i = 0; i < 16 * S1 * S1; ++i) d1[i] = 0.0;
        for (int o = 0; o < 16; ++o)
            for (int y = 0; y < S2; ++y)
                for (int x = 0; x < S2; ++x) {
                    double g = d2[(o * S2 + y) * S2 + x];
                    if (g == 0.0) continue;
                    for (int c = 0; c < 16; ++c)
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx)
                                d1[(c * S1 + y + ky) * S1 + x + kx] += g * W2[((o * 16 + c) * 3 + ky) * 3 + kx];
                }
        for (int i = 0; i < 16 * S1 * S1; ++i)
            if (!(z1[i] > 0.0)) d1[i] = 0.0;
        /* layer 1 */
        for (int o = 0; o < 16; ++o)
            for (int y = 0; y < S1; ++y)
                for (int x = 0; x < S1; ++x) {
                    double g = d1[(o * S1 + y) * S1 + x];
                    if (g == 0.0) continue;
                    grad[864 + o] += g;
                    for (int c = 0; c < 6; ++c)
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx)
                                grad[((o * 6 + c) * 3 + ky) * 3 + kx] += g * in_r[(c * P + y + ky) * P + x + kx];
                }
    }
    *loss = L_sum / ((double)n * K2);
    free(buf);
    return 0;
}

/* Exact energy difference (1/16 units) of replacing block (bR, bC) of v by
 * newblock[k*k] (+-1), canonical SS lattice (even L, periodic): bonds with at
 * least one endpoint in the block and the field term of the block sites. */
static int diag_partner(int L, int R, int C) {
    int r = R & 1, c = C & 1, R2, C2;
    if (!r && !c) { R2 = R + 1; C2 = C + 1; }        /* "\" dimer, upper end */
    else if (r && c) { R2 = R - 1; C2 = C - 1; }     /* "\" dimer, lower end */
    else if (r && !c) { R2 = R + 1; C2 = C - 1; }    /* "/" dimer, upper end */
    else { R2 = R - 1; C2 = C + 1; }                 /* "/" dimer, lower end */
    R2 = (R2 % L + L) % L;
    C2 = (C2 % L + L) % L;
    return R2 * L + C2;
}

int64_t orc_block_delta_e(int L, const int8_t* v, int bR, int bC, int k, const int8_t* newblock,
                          int32_t qJ, int32_t qJp, int32_t qh) {
    int N = L * L;
    int8_t* w = (int8_t*)malloc((size_t)N);
    memcpy(w, v, (size_t)N);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) w[((bR + a) % L) * L + (bC + b) % L] = newblock[a * k + b];
    int64_t d = 0;
    for (int s = 0; s < N; ++s) {
        int R = s / L, C = s % L;
        int nbr[3] = {R * L + (C + 1) % L, ((R + 1) % L) * L + C, -1};
        int dp = diag_partner(L, R, C);
        if (dp > s) nbr[2] = dp; /* count each dimer once */
        for (int t = 0; t < 3; ++t) {
            if (nbr[t] < 0) continue;
            int e0 = v[s] * v[nbr[t]], e1 = w[s] * w[nbr[t]];
            d += (int64_t)(t < 2 ? qJ : qJp) * (e1 - e0);
        }
        d -= (int64_t)qh * (w[s] - v[s]);
    }
    free(w);
    return d;
}

/* One Metropolis-Hastings block move from configuration v: probs[b] (b =
 * the k*k bits of the proposed block, bit a*k+b'' set = +1) is the exact
 * probability of moving to that block value; the entry of the current value
 * also holds the rejection mass. */
int orc_mh_row(int L, const int8_t* v, int bR, int bC, int k, const double* w, double J, double Jp,
               double h, double beta, int bf16, double* probs) {
    if (k < 1 || k > 4 || (L & 1)) return -1;
    int P = k + 6, K2 = k * k;
    int32_t qJ, qJp, qh;
    if (orc_quantize(J, &qJ) || orc_quantize(Jp, &qJp) || orc_quantize(h, &qh)) return -1;
    double* input = (double*)malloc(sizeof(double) * 6 * P * P);
    double logit[16];
    orc_patch_input(L, v, bR, bC, k, bf16 ? orc_bf16(beta) : beta, bf16 ? orc_bf16(h) : h, input);
    orc_net_forward(k, w, input, bf16, logit);
    free(input);
    double p[16];
    for (int s = 0; s < K2; ++s) {
        double q = 1.0 / (1.0 + exp(-logit[s]));
        double t = nearbyint(ldexp(q, 32));
        if (t < 1.0) t = 1.0;
        if (t > 4294967295.0) t = 4294967295.0;
        p[s] = ldexp(t, -32);
    }
    int cur = 0;
    for (int s = 0; s < K2; ++s)
        if (v[((bR + s / k) % L) * L + (bC + s % k) % L] > 0) cur |= 1 << s;
    double logq_cur = 0.0;
    for (int s = 0; s < K2; ++s) logq_cur += ((cur >> s) & 1) ? log(p[s]) : log1p(-p[s]);
    double stay = 1.0;
    int8_t nb[16];
    for (int b = 0; b < (1 << K2); ++b) {
        probs[b] = 0.0;
        if (b == cur) continue;
        double logq = 0.0;
        for (int s = 0; s < K2; ++s) {
            nb[s] = ((b >> s) & 1) ? 1 : -1;
            logq += ((b >> s) & 1) ? log(p[s]) : log1p(-p[s]);
        }
        int64_t dE = orc_block_delta_e(L, v, bR, bC, k, nb, qJ, qJp, qh);
        double loga = -beta * (double)dE / 16.0 + logq_cur - logq;
        double acc = loga >= 0.0 ? 1.0 : exp(loga);
        probs[b] = exp(logq) * acc;
        stay -= probs[b];
    }
    probs[cur] = stay;
    return 0;
}

/* orc_mh_row over many configurations v[n][L*L] (rows probs[n][2^(k*k)]). */
int orc_mh_rows(int L, const int8_t* v, int n, int bR, int bC, int k, const double* w, double J,
                double Jp, double h, double beta, int bf16, double* probs) {
    int err = 0;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        if (orc_mh_row(L, v + (size_t)i * L * L, bR, bC, k, w, J, Jp, h, beta, bf16,
                       probs + ((size_t)i << (k * k))))
            err = 1;
    return err ? -1 : 0;
}

/* One pass of learned block moves (no counterpart in the paper: the learned
 * proposal mixed with the block Gibbs sweeps of Sec. II.B).  The steps, in
 * order, for every block b of the pass and every chain c:
 *   1. origin: nb1 = max(1, L / 8) blocks per side at spacing L / nb1, shifted
 *      by words 0 and 1 of Philox((pass, 0, 0, ORC_TAG_PROP_OFFSET));
 *   2. logits of the net on the patch (orc_patch_input, bf16 on, beta and h
 *      rounded to bf16 as net inputs), or the given ones;
 *   3. t_s = clamp(nearbyint(2^32 sigmoid(logit_s)), 1, 2^32 - 1); site s
 *      proposes +1 iff word s % 4 of Philox((b, pass, c, ORC_TAG_PROP_BITS +
 *      s / 4)) < t_s;
 *   4. dE of the proposed block (orc_block_delta_e), log alpha = -beta dE / 16
 *      + sum_s log q(x_s) - sum_s log q(x'_s) with q(+1) = t_s / 2^32 and
 *      q(-1) = 1 - t_s / 2^32 (the exact beta, not its bf16 rounding);
 *   5. u = (word 0 of Philox((b, pass, c, ORC_TAG_PROP_ACCEPT)) >> 8) / 2^24;
 *      accept iff log alpha >= 0 or u < exp(log alpha);
 *   6. with apply != 0, accepted blocks are written into v.
 * Blocks of one pass are at least 8 sites apart, so with L >= 10 no block
 * lies in another's patch or energy halo and the order of the moves does not
 * matter.  rec[b * n_chains + c] receives the record; logits_in (NULL: run
 * the net) is [n_blocks][n_chains][16]; thr_in (NULL: step 3's thresholds)
 * [n_blocks][n_chains][16] replaces the thresholds, so that a test can feed
 * another implementation's thresholds and compare the remaining steps.
 * Returns the number of blocks, or a negative error. */
int orc_prop_pass(int L, int8_t* v, int n_chains, const double* J, const double* Jp,
                  const double* h, const double* beta, const int32_t* chain_param,
                  const double* w, const double* logits_in, const uint32_t* thr_in,
                  uint64_t seed, uint32_t pass, int apply, orc_pass_rec* rec) {
    const int k = 4, K2 = 16;
    if (L < 10 || (L & 1) || n_chains < 1) return -1;
    int nb1 = L / 8 > 1 ? L / 8 : 1;
    int spacing = L / nb1, n_blocks = nb1 * nb1;
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {pass, 0u, 0u, ORC_TAG_PROP_OFFSET}, off[4];
    orc_philox4x32_10(ctr, key, off);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < n_chains; ++c) {
        int p = chain_param[c];
        int32_t qJ, qJp, qh;
        if (orc_quantize(J[p], &qJ) || orc_quantize(Jp[p], &qJp) || orc_quantize(h[p], &qh)) {
            err = 1;
            continue;
        }
        int8_t* vc = v + (size_t)c * L * L;
        double input[6 * 10 * 10];
        for (int b = 0; b < n_blocks; ++b) {
            orc_pass_rec* r = rec + (size_t)b * n_chains + c;
            int bR = (int)((off[0] % (uint32_t)L + (uint32_t)(spacing * (b / nb1))) % (uint32_t)L);
            int bC = (int)((off[1] % (uint32_t)L + (uint32_t)(spacing * (b % nb1))) % (uint32_t)L);
            r->bR = bR;
            r->bC = bC;
            if (logits_in) {
                for (int s = 0; s < K2; ++s) r->logit[s] = logits_in[((size_t)b * n_chains + c) * K2 + s];
            } else {
                orc_patch_input(L, vc, bR, bC, k, orc_bf16(beta[p]), orc_bf16(h[p]), input);
                orc_net_forward(k, w, input, 1, r->logit);
            }
            uint32_t draws[16];
            for (int call = 0; call < 4; ++call) {
                uint32_t cc[4] = {(uint32_t)b, pass, (uint32_t)c, ORC_TAG_PROP_BITS + (uint32_t)call}, o[4];
                orc_philox4x32_10(cc, key, o);
                for (int j = 0; j < 4; ++j) draws[4 * call + j] = o[j];
            }
            uint32_t cur = 0, nw = 0;
            double logq_cur = 0.0, logq_new = 0.0;
            int8_t nb[16];
            for (int s = 0; s < K2; ++s) {
                double q = 1.0 / (1.0 + exp(-r->logit[s]));
                double t = nearbyint(ldexp(q, 32));
                if (t < 1.0) t = 1.0;
                if (t > 4294967295.0) t = 4294967295.0;
                if (thr_in) t = (double)thr_in[((size_t)b * n_chains + c) * K2 + s];
                r->thr[s] = (uint32_t)t;
                r->draw[s] = draws[s];
                double pq = ldexp(t, -32);
                int xc = vc[((bR + s / k) % L) * L + (bC + s % k) % L] > 0;
                int xn = draws[s] < (uint32_t)t;
                cur |= (uint32_t)xc << s;
                nw |= (uint32_t)xn << s;
                nb[s] = xn ? 1 : -1;
                logq_cur += xc ? log(pq) : log1p(-pq);
                logq_new += xn ? log(pq) : log1p(-pq);
            }
            r->cur_bits = cur;
            r->new_bits = nw;
            r->dE = orc_block_delta_e(L, vc, bR, bC, k, nb, qJ, qJp, qh);
            r->log_alpha = -beta[p] * (double)r->dE / 16.0 + logq_cur - logq_new;
            uint32_t ca[4] = {(uint32_t)b, pass, (uint32_t)c, ORC_TAG_PROP_ACCEPT}, oa[4];
            orc_philox4x32_10(ca, key, oa);
            r->u_accept = ldexp((double)(oa[0] >> 8), -24);
            r->accept = r->log_alpha >= 0.0 || r->u_accept < exp(r->log_alpha);
        }
        if (apply)
            for (int b = 0; b < n_blocks; ++b) {
                const orc_pass_rec* r = rec + (size_t)b * n_chains + c;
                if (!r->accept) continue;
                for (int s = 0; s < K2; ++s)
                    vc[((r->bR + s / k) % L) * L + (r->bC + s % k) % L] = ((r->new_bits >> s) & 1u) ? 1 : -1;
            }
    }
    return err ? -1 : n_blocks;
}
