// Host runtime of the CRBM sampler: model construction (Eqs. 3-8 of arXiv
// 2511.20911), threshold tables, device buffers, launches and the C ABI of
// include/crbm.h.  Compiled with -ffp-contract=off: every table entry is the
// plain left-to-right double evaluation of the formulas in crbm.h.
#include "../../include/crbm.h"
#include "crbm_internal.h"
#include "crbm_context.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace crbm;




namespace {

thread_local std::string g_create_error;

// The ten filters of the SS unit cell (Fig. 1): horizontal bonds of window
// rows 0 and 1, vertical bonds of columns 0 and 1 (class 0, J1), and the
// orthogonal dimers "\" on plaquette (0,0) and "/" on plaquette (1,1)
// (class 1, J2).  Window offsets are (row, col) in [0, 2].
const crbm_bond kSSFilters[10] = {
    {0, 0, 0, 1, 0}, {0, 1, 0, 2, 0}, {1, 0, 1, 1, 0}, {1, 1, 1, 2, 0}, {0, 0, 1, 0, 0},
    {1, 0, 2, 0, 0}, {0, 1, 1, 1, 0}, {1, 1, 2, 1, 0}, {0, 0, 1, 1, 1}, {1, 2, 2, 1, 1},
};

int fail(crbm_ctx* ctx, int code, const std::string& msg) {
    if (ctx)
        ctx->err = msg;
    else
        g_create_error = msg;
    return code;
}

int cuda_fail(crbm_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, CRBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Q.4 fixed point: nearest multiple of 1/16, |16 x| <= 2047.
bool to_q4(double x, int32_t& q) {
    if (!std::isfinite(x)) return false;
    const double r = std::nearbyint(16.0 * x);
    if (r < -2047.0 || r > 2047.0) return false;
    q = static_cast<int32_t>(r);
    return true;
}

// Eqs. (5)-(7): a = 1/2 arccosh(exp(2|K|)), K = -beta J; s = sign of K (+1 at 0).
void bond_weight(double beta, double J, double& a, int& s) {
    const double K = -beta * J;
    a = 0.5 * std::acosh(std::exp(2.0 * std::fabs(K)));
    s = (K >= 0.0) ? 1 : -1;
}

// Sigmoid of Eqs. (9)-(10) as a 32-bit acceptance threshold.
uint32_t accept_threshold(double y) {
    const double prob = 1.0 / (1.0 + std::exp(-y));
    const double r = std::nearbyint(std::ldexp(prob, 32));
    if (r >= 4294967295.0) return 0xFFFFFFFFu;
    if (r <= 0.0) return 0u;
    return static_cast<uint32_t>(r);
}

// Paper precision (Sec. III, "Dimension and Precision"): a weight or bias in
// 10-bit fixed point with 4 fraction bits, in 1/16 units (saturating).
int32_t fixed_q54(double x) {
    const double r = std::nearbyint(16.0 * x);
    return static_cast<int32_t>(r > 511.0 ? 511.0 : (r < -511.0 ? -511.0 : r));
}

// Paper precision: the 16-bit sigmoid table entry of a 12-bit accumulator
// value y (1/16 units, saturating), sigmoid(2 y / 16), placed in the upper
// half of a 32-bit threshold so that the kernels compare 16-bit uniforms
// held in the upper half of a word.
uint32_t sigmoid_lut16(int32_t y) {
    const int32_t acc = y > 2047 ? 2047 : (y < -2047 ? -2047 : y);
    const double prob = 1.0 / (1.0 + std::exp(-2.0 * static_cast<double>(acc) / 16.0));
    const double r = std::nearbyint(std::ldexp(prob, 16));
    return static_cast<uint32_t>(r > 65535.0 ? 65535.0 : r) << 16;
}

// Replica-exchange acceptance exp(x), x <= 0, as a 32-bit threshold.
uint32_t swap_threshold(double x) {
    const double r = std::nearbyint(std::ldexp(std::exp(x), 32));
    if (r >= 4294967295.0) return 0xFFFFFFFFu;
    if (r <= 0.0) return 0u;
    return static_cast<uint32_t>(r);
}

int site_index(const Geometry& g, int i, int j, int r, int c) {
    int R = 2 * i + r, C = 2 * j + c;
    if (R >= g.L) {
        if (!g.periodic) return -1;
        R %= g.L;
    }
    if (C >= g.Lc) {
        if (!g.pc) return -1;
        C %= g.Lc;
    }
    return R * g.Lc + C;
}

// Geometry, visible field ranges and the generic endpoint words.
int build_geometry(crbm_ctx* ctx, const crbm_params* p, std::vector<uint32_t>& ep) {
    Geometry& g = ctx->g;
    const crbm_bond* bonds = p->bonds ? p->bonds : kSSFilters;
    const int nb = p->bonds ? p->n_bonds : 10;
    if (nb < 1 || nb > kMaxBonds) return fail(nullptr, CRBM_EINVAL, "n_bonds must be in 1..16");
    for (int k = 0; k < nb; ++k) {
        const crbm_bond& b = bonds[k];
        if (b.r1 < 0 || b.r1 > 2 || b.c1 < 0 || b.c1 > 2 || b.r2 < 0 || b.r2 > 2 || b.c2 < 0 ||
            b.c2 > 2 || b.cls > 1 || (b.r1 == b.r2 && b.c1 == b.c2))
            return fail(nullptr, CRBM_EINVAL, "bond " + std::to_string(k) + " is not a bond of the 3x3 window");
        g.r1[k] = b.r1; g.c1[k] = b.c1; g.r2[k] = b.r2; g.c2[k] = b.c2; g.cls[k] = b.cls;
    }
    if (p->L_cols != 0 && (p->L_cols < 3 || p->L_cols > 4096))
        return fail(nullptr, CRBM_EINVAL, "L_cols must be 0 or in 3..4096");
    if (p->periodic_cols < CRBM_BC_AS_ROWS || p->periodic_cols > CRBM_BC_OPEN)
        return fail(nullptr, CRBM_EINVAL, "unknown periodic_cols");
    g.L = p->L;
    g.W = (p->L + 1) / 2;
    g.Lc = p->L_cols ? p->L_cols : p->L;
    g.Wc = (g.Lc + 1) / 2;
    g.N = g.L * g.Lc;
    g.n_cells = g.W * g.Wc;
    g.nb = nb;
    g.n_calls = (nb + 3) / 4;
    g.periodic = p->periodic ? 1 : 0;
    g.pc = p->periodic_cols == CRBM_BC_AS_ROWS ? g.periodic : (p->periodic_cols == CRBM_BC_PERIODIC ? 1 : 0);
    g.n_vis_tab = p->h_odd ? 2 : 1;
    bool same = (nb == 10);
    for (int k = 0; same && k < 10; ++k)
        same = std::memcmp(&bonds[k], &kSSFilters[k], sizeof(crbm_bond)) == 0;
    g.canonical = (same && g.periodic && g.pc && g.L % 2 == 0 && g.Lc % 2 == 0 && g.n_vis_tab == 1) ? 1 : 0;

    std::vector<int> deg(2 * static_cast<size_t>(g.N), 0);  // filters per (class, site)
    g.n_real_bonds[0] = g.n_real_bonds[1] = 0;
    for (int i = 0; i < g.W; ++i)
        for (int j = 0; j < g.Wc; ++j)
            for (int k = 0; k < nb; ++k) {
                const int s1 = site_index(g, i, j, g.r1[k], g.c1[k]);
                const int s2 = site_index(g, i, j, g.r2[k], g.c2[k]);
                const int cls = g.cls[k];
                if (s1 >= 0) deg[cls * g.N + s1]++;
                if (s2 >= 0) deg[cls * g.N + s2]++;
                if (s1 >= 0 && s2 >= 0) g.n_real_bonds[cls]++;
            }
    g.DJ = g.DJp = 0;
    for (int s = 0; s < g.N; ++s) {
        g.DJ = std::max(g.DJ, deg[s]);
        g.DJp = std::max(g.DJp, deg[g.N + s]);
    }
    g.nTv = (2 * g.DJ + 1) * (2 * g.DJp + 1);
    g.nTab = 10 + g.n_vis_tab * g.nTv;
    if (g.canonical && (g.DJ != 4 || g.DJp != 1))
        return fail(nullptr, CRBM_EINVAL, "internal: SS filters must give 4 J and 1 J' filter per spin");
    // endpoint words of the generic measurement, [n_cells][nb]: per endpoint
    // 15 bits of site and a real-site flag (a padded one is 0); generic
    // contexts are SMEM-resident (L <= CRBM_SMEM_MAX_L), so sites fit
    auto endpoint = [&](int s) { return s >= 0 ? (static_cast<uint32_t>(s) | 0x8000u) : 0u; };
    ep.clear();
    if (!g.canonical && g.N <= 0x7FFF) {
        for (int i = 0; i < g.W; ++i)
            for (int j = 0; j < g.Wc; ++j)
                for (int k = 0; k < nb; ++k)
                    ep.push_back(endpoint(site_index(g, i, j, g.r1[k], g.c1[k])) |
                                 (endpoint(site_index(g, i, j, g.r2[k], g.c2[k])) << 16));
    }
    return CRBM_OK;
}

// Visible rows of one field value: Tv[nJ+DJ][nJ'+DJ'] = thr(2 (beta h + a_J nJ + a_J' nJ')), or the
// 16-bit table of paper precision.
void visible_rows(const Geometry& g, double beta, const double a[2], int32_t qh, uint32_t* out) {
    const int nP = 2 * g.DJp + 1;
    if (g.paper) {
        const int32_t A[2] = {fixed_q54(a[0]), fixed_q54(a[1])}, B = fixed_q54(beta * (qh / 16.0));
        for (int nJ = -g.DJ; nJ <= g.DJ; ++nJ)
            for (int nJp = -g.DJp; nJp <= g.DJp; ++nJp)
                out[(nJ + g.DJ) * nP + (nJp + g.DJp)] = sigmoid_lut16(B + A[0] * nJ + A[1] * nJp);
        return;
    }
    const double hd = qh / 16.0;
    for (int nJ = -g.DJ; nJ <= g.DJ; ++nJ)
        for (int nJp = -g.DJp; nJp <= g.DJp; ++nJp) {
            const double x = beta * hd + a[0] * nJ + a[1] * nJp;
            out[(nJ + g.DJ) * nP + (nJp + g.DJp)] = accept_threshold(2.0 * x);
        }
}

// Th[cls][m+2] = thr(2 a_cls m), then the visible rows of field h and, with
// an odd-column field, those of h_odd (qho).
void point_tables(const Geometry& g, double beta, int32_t qJ, int32_t qJp, int32_t qh, int32_t qho,
                  uint32_t* out, int sgn[2]) {
    double a[2];
    bond_weight(beta, qJ / 16.0, a[0], sgn[0]);
    bond_weight(beta, qJp / 16.0, a[1], sgn[1]);
    if (g.paper) {
        const int32_t A[2] = {fixed_q54(a[0]), fixed_q54(a[1])};
        for (int cls = 0; cls < 2; ++cls)
            for (int m = -2; m <= 2; ++m) out[cls * 5 + m + 2] = sigmoid_lut16(A[cls] * m);
    } else {
        for (int cls = 0; cls < 2; ++cls)
            for (int m = -2; m <= 2; ++m) out[cls * 5 + m + 2] = accept_threshold(2.0 * a[cls] * m);
    }
    visible_rows(g, beta, a, qh, out + 10);
    if (g.n_vis_tab == 2) visible_rows(g, beta, a, qho, out + 10 + g.nTv);
}

template <typename T>
int dalloc(crbm_ctx* ctx, T*& ptr, size_t count) {
    if (count == 0) count = 1;
    const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&ptr), count * sizeof(T));
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();  // clear the (non-sticky) allocation error so later launch checks do not see it
        return fail(ctx, CRBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return CRBM_OK;
}

void free_device(DeviceState& d) {
    void* ptrs[] = {d.v, d.tab, d.ctab, d.crec, d.sneg, d.gep, d.sums, d.series, d.corr,
                    d.seg, d.segmask, d.spins8, d.h, d.cnt, d.sob, d.swap_tab, d.swap_off,
                    d.swap_len, d.wq, d.chain_bh, d.chain_q, d.sched, d.hit, d.hit_q, d.flag};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    d = DeviceState{};
}

int default_warps(const Geometry& g) {
    if (const char* env = std::getenv("CRBM_WARPS")) {
        const int w = std::atoi(env);
        if (w >= 1 && w <= kMaxSweepWarps) return w;
    }
    // about six cells per warp, up to 16 warps per CTA
    return std::max(1, std::min(std::min(16, kMaxSweepWarps), (g.n_cells + 5) / 6));
}

}  // namespace

namespace crbm {
bool host_to_q4(double x, int32_t& q) { return to_q4(x, q); }
void host_point_tables(const Geometry& g, double beta, int32_t qJ, int32_t qJp, int32_t qh,
                       uint32_t* out, int sgn[2]) {
    point_tables(g, beta, qJ, qJp, qh, qh, out, sgn);
}
}  // namespace crbm

namespace crbm {
SweepArgs fill_sweep_args(const crbm_ctx* ctx, int chunk) {
    SweepArgs a{};
    a.g = ctx->g;
    a.v = ctx->d.v;
    a.tab = ctx->d.tab;
    a.ctab = ctx->d.ctab;
    a.crec = ctx->d.crec;
    a.sneg = ctx->d.sneg;
    a.gep = ctx->d.gep;
    a.hit = ctx->d.hit;
    a.hit_q = ctx->d.hit_q;
    a.sums = ctx->d.sums;
    a.series = ctx->d.series;
    a.h = ctx->d.h;
    a.cnt = ctx->d.cnt;
    a.sob = ctx->d.sob;
    a.swap_tab = ctx->d.swap_tab;
    a.swap_off = ctx->d.swap_off;
    a.swap_len = ctx->d.swap_len;
    a.wq = ctx->d.wq;
    a.swap_every = ctx->swap_every;
    a.n_bands = 1;
    a.corr = ctx->d.corr;
    a.seg = ctx->d.seg;
    a.segmask = ctx->d.segmask;
    a.n_words = ctx->n_words;
    a.n_chains_padded = ctx->n_words * 32;
    a.n_chains = ctx->n_chains;
    a.key0 = static_cast<uint32_t>(ctx->seed);
    a.key1 = static_cast<uint32_t>(ctx->seed >> 32);
    for (int r = 0; r < 10; ++r) {  // Philox key schedule (Weyl increments)
        a.rk[2 * r] = a.key0 + static_cast<uint32_t>(r) * 0x9E3779B9u;
        a.rk[2 * r + 1] = a.key1 + static_cast<uint32_t>(r) * 0xBB67AE85u;
    }
    a.t0 = static_cast<uint32_t>(ctx->sweeps);
    a.n_sweeps = chunk;
    a.measure_every = ctx->measure_every;
    a.meas0 = ctx->meas;
    a.series_len = ctx->series_len;
    a.sq_every = ctx->sq_every;
    return a;
}
}  // namespace crbm

extern "C" {

int crbm_create(crbm_ctx** out, const crbm_params* p) {
    if (!out || !p) return fail(nullptr, CRBM_EINVAL, "null argument");
    *out = nullptr;
    if (p->L < 3 || p->L > 4096) return fail(nullptr, CRBM_EINVAL, "L must be in 3..4096");
    if (p->n_params < 1 || !p->J || !p->Jp || !p->h || !p->beta)
        return fail(nullptr, CRBM_EINVAL, "need n_params >= 1 and J, Jp, h, beta arrays");
    if (p->n_chains < 1 || p->n_chains > (1 << 30)) return fail(nullptr, CRBM_EINVAL, "n_chains must be in 1..2^30");
    if (p->measure_every < 0 || p->series_len < 0 || p->sq_every < 0)
        return fail(nullptr, CRBM_EINVAL, "measure_every, series_len and sq_every must be >= 0");
    if (p->layout < CRBM_LAYOUT_AUTO || p->layout > CRBM_LAYOUT_STREAM)
        return fail(nullptr, CRBM_EINVAL, "unknown layout");
    crbm_ctx* ctx = new (std::nothrow) crbm_ctx();
    if (!ctx) return fail(nullptr, CRBM_ENOMEM, "host allocation failed");
    std::vector<uint32_t> gep;
    int rc = build_geometry(ctx, p, gep);
    if (rc) {
        delete ctx;
        return rc;
    }
    Geometry& g = ctx->g;
    if (p->precision != CRBM_PRECISION_EXACT && p->precision != CRBM_PRECISION_PAPER) {
        delete ctx;
        return fail(nullptr, CRBM_EINVAL, "unknown precision");
    }
    g.paper = p->precision == CRBM_PRECISION_PAPER ? 1 : 0;
    if (p->rng != CRBM_RNG_LANE && p->rng != CRBM_RNG_BITPLANE) {
        delete ctx;
        return fail(nullptr, CRBM_EINVAL, "unknown rng");
    }
    g.bitplane = p->rng == CRBM_RNG_BITPLANE ? 1 : 0;
    if (g.bitplane && (!g.canonical || g.paper || p->sq_every > 0)) {
        delete ctx;
        return fail(nullptr, CRBM_EUNSUPPORTED,
                    "bit-plane uniforms need the ten SS filters on an even periodic lattice, exact precision and "
                    "no correlations");
    }
    // AUTO: shared memory when the lattice, its hidden words and the tables fit
    // in one CTA's 227 KB, else the streamed layout (SS filters, even periodic L)
    ctx->layout = p->layout;
    if (ctx->layout == CRBM_LAYOUT_AUTO) {
        const size_t need = g.bitplane    ? smem_bytes_bitplane(g, false)
                            : g.canonical ? smem_bytes_canon(g)
                                          : smem_bytes_generic(g);
        ctx->layout = (p->L <= CRBM_SMEM_MAX_L && g.Lc <= CRBM_SMEM_MAX_L && need <= 227 * 1024)
                          ? CRBM_LAYOUT_SMEM
                          : CRBM_LAYOUT_STREAM;
    }
    if (ctx->layout == CRBM_LAYOUT_SMEM && (p->L > CRBM_SMEM_MAX_L || g.Lc > CRBM_SMEM_MAX_L)) {
        delete ctx;
        return fail(nullptr, CRBM_EINVAL, "SMEM layout needs L, L_cols <= CRBM_SMEM_MAX_L");
    }
    if (g.paper && g.nb > 10) {
        delete ctx;
        return fail(nullptr, CRBM_EUNSUPPORTED, "paper precision draws 16-bit uniforms for at most ten filters");
    }
    if (ctx->layout == CRBM_LAYOUT_STREAM && !g.canonical) {
        delete ctx;
        return fail(nullptr, CRBM_EUNSUPPORTED,
                    "the streamed layout serves the ten SS filters on an even, periodic lattice");
    }
    if (ctx->layout == CRBM_LAYOUT_STREAM && g.bitplane && p->swap_every > 0) {
        delete ctx;
        return fail(nullptr, CRBM_EUNSUPPORTED, "bit-plane uniforms take replica exchange in the SMEM layout only");
    }
    if (ctx->layout == CRBM_LAYOUT_STREAM && p->sq_every > 0) {
        delete ctx;
        return fail(nullptr, CRBM_EUNSUPPORTED, "spin correlations are accumulated in the SMEM layout only");
    }
    g.vil = ctx->layout == CRBM_LAYOUT_STREAM ? 1 : 0;
    if (ctx->layout == CRBM_LAYOUT_SMEM &&
        (g.bitplane ? smem_bytes_bitplane(g, false) : g.canonical ? smem_bytes_canon(g) : smem_bytes_generic(g)) >
            227 * 1024) {
        delete ctx;
        return fail(nullptr, CRBM_EUNSUPPORTED,
                    "lattice, hidden layer and threshold columns exceed 227 KB of shared memory");
    }
    if (p->sq_every > 0 && (!g.periodic || !g.pc || g.Lc != g.L)) {
        delete ctx;
        return fail(nullptr, CRBM_EINVAL, "spin correlations need a square lattice, periodic along both axes");
    }
    ctx->n_chains = p->n_chains;
    // the streamed layout stores 64-chain words: an even number of 32-chain halves
    ctx->n_words = ctx->layout == CRBM_LAYOUT_STREAM ? 2 * ((p->n_chains + 63) / 64) : (p->n_chains + 31) / 32;
    ctx->n_params = p->n_params;
    ctx->seed = p->seed;
    ctx->measure_every = p->measure_every;
    ctx->series_len = p->series_len;
    ctx->sq_every = p->sq_every;
    ctx->stream = static_cast<cudaStream_t>(p->stream);
    ctx->warps = default_warps(g);
    for (int k = 0; k < 3; ++k) ctx->q[k].resize(p->n_params);
    ctx->q_odd.resize(p->n_params);
    ctx->beta.assign(p->beta, p->beta + p->n_params);
    for (int i = 0; i < p->n_params; ++i) {
        if (!to_q4(p->J[i], ctx->q[0][i]) || !to_q4(p->Jp[i], ctx->q[1][i]) ||
            !to_q4(p->h[i], ctx->q[2][i]) || !to_q4(p->h_odd ? p->h_odd[i] : p->h[i], ctx->q_odd[i])) {
            delete ctx;
            return fail(nullptr, CRBM_EINVAL, "parameter point " + std::to_string(i) +
                                                  ": J, J', h, h_odd must be finite with |16 x| <= 2047");
        }
        if (!(p->beta[i] >= 0.0) || !(p->beta[i] <= 1.0e6)) {
            delete ctx;
            return fail(nullptr, CRBM_EINVAL, "parameter point " + std::to_string(i) + ": beta must be in [0, 1e6]");
        }
    }
    ctx->chain_param.resize(p->n_chains);
    for (int c = 0; c < p->n_chains; ++c) {
        const int32_t pp = p->chain_param
                               ? p->chain_param[c]
                               : static_cast<int32_t>(static_cast<int64_t>(c) * p->n_params / p->n_chains);
        if (pp < 0 || pp >= p->n_params) {
            delete ctx;
            return fail(nullptr, CRBM_EINVAL, "chain_param[" + std::to_string(c) + "] out of range");
        }
        ctx->chain_param[c] = pp;
    }
    // Replica-exchange ladders: 32-chain words of equal couplings and
    // strictly increasing beta; per pair a threshold table over the energy
    // difference dE = 1 .. len-1 (1/16 units), len = the first dE whose
    // threshold is 0 (or past the largest possible |dE|).
    ctx->swap_every = p->swap_every;
    std::vector<uint32_t> swap_tab;
    std::vector<int32_t> swap_off, swap_len, wq;
    if (p->swap_every < 0) {
        delete ctx;
        return fail(nullptr, CRBM_EINVAL, "swap_every must be >= 0");
    }
    if (p->swap_every > 0) {
        if (g.n_vis_tab == 2) {
            delete ctx;
            return fail(nullptr, CRBM_EUNSUPPORTED, "replica exchange needs one field on every column (no h_odd)");
        }
        if (p->n_chains % 32 != 0) {
            delete ctx;
            return fail(nullptr, CRBM_EINVAL, "replica exchange needs n_chains % 32 == 0");
        }
        const int nwl = p->n_chains / 32;
        const int64_t e_max = 2 * (2047LL * g.n_real_bonds[0] + 2047LL * g.n_real_bonds[1] + 2047LL * g.N);
        swap_off.assign(32 * static_cast<size_t>(nwl), 0);
        swap_len.assign(32 * static_cast<size_t>(nwl), 0);
        wq.assign(3 * static_cast<size_t>(nwl), 0);
        for (int w = 0; w < nwl; ++w) {
            const int32_t* cpw = &ctx->chain_param[32 * w];
            for (int k = 0; k < 32; ++k) {
                const int pk = cpw[k], p0 = cpw[0];
                if (ctx->q[0][pk] != ctx->q[0][p0] || ctx->q[1][pk] != ctx->q[1][p0] ||
                    ctx->q[2][pk] != ctx->q[2][p0] || (k > 0 && !(ctx->beta[pk] > ctx->beta[cpw[k - 1]]))) {
                    delete ctx;
                    return fail(nullptr, CRBM_EINVAL,
                                "ladder " + std::to_string(w) +
                                    ": rungs need equal J, J', h and strictly increasing beta");
                }
            }
            wq[3 * w] = ctx->q[0][cpw[0]];
            wq[3 * w + 1] = ctx->q[1][cpw[0]];
            wq[3 * w + 2] = ctx->q[2][cpw[0]];
            const int64_t emax_w = 2 * (std::abs(static_cast<int64_t>(wq[3 * w])) * g.n_real_bonds[0] +
                                        std::abs(static_cast<int64_t>(wq[3 * w + 1])) * g.n_real_bonds[1] +
                                        std::abs(static_cast<int64_t>(wq[3 * w + 2])) * g.N);
            (void)e_max;
            for (int k = 0; k < 31; ++k) {
                const double db = ctx->beta[cpw[k]] - ctx->beta[cpw[k + 1]];
                swap_off[32 * w + k] = static_cast<int32_t>(swap_tab.size());
                int64_t len = 1;
                swap_tab.push_back(0u);  // dE = 0 is accepted before any lookup
                while (len <= emax_w) {
                    const uint32_t thr = swap_threshold(db * static_cast<double>(len) / 16.0);
                    if (thr == 0u) break;
                    swap_tab.push_back(thr);
                    ++len;
                    if (swap_tab.size() > (1u << 26)) {
                        delete ctx;
                        return fail(nullptr, CRBM_EUNSUPPORTED,
                                    "adjacent rungs too close in beta for the swap tables");
                    }
                }
                swap_len[32 * w + k] = static_cast<int32_t>(len);
            }
        }
    }
    // Per-point tables and signs, then lane-expanded per word.
    ctx->tables.resize(static_cast<size_t>(p->n_params) * g.nTab);
    std::vector<int> sgn(2 * static_cast<size_t>(p->n_params));
    for (int i = 0; i < p->n_params; ++i)
        point_tables(g, ctx->beta[i], ctx->q[0][i], ctx->q[1][i], ctx->q[2][i], ctx->q_odd[i],
                     &ctx->tables[static_cast<size_t>(i) * g.nTab], &sgn[2 * i]);
    const int nw = ctx->n_words, npad = nw * 32;
    // generic lane-expanded tables (layout in crbm_internal.h); canonical contexts use ctab
    const int nTg = g.canonical ? 0 : kGenHid + g.n_vis_tab * g.nTv;
    std::vector<uint32_t> tab(static_cast<size_t>(nw) * nTg * 32);
    std::vector<uint32_t> sneg(2 * static_cast<size_t>(nw), 0u);
    std::vector<int32_t> seg(33 * static_cast<size_t>(nw), 0);
    std::vector<uint32_t> segmask(32 * static_cast<size_t>(nw), 0u);
    for (int w = 0; w < nw; ++w) {
        int nseg = 0;
        for (int l = 0; l < 32; ++l) {
            const int c = w * 32 + l;
            const bool real = c < p->n_chains;
            const int pp = real ? ctx->chain_param[c] : ctx->chain_param[0];
            if (nTg > 0) {
                const uint32_t* T = &ctx->tables[static_cast<size_t>(pp) * g.nTab];
                uint32_t* out = &tab[static_cast<size_t>(w) * nTg * 32 + l];
                for (int cls = 0; cls < 2; ++cls)
                    for (int pad = 0; pad < 4; ++pad)
                        for (int idx = 0; idx < 4; ++idx) {
                            const int e1 = idx & 1, e2 = idx >> 1;
                            const int m = ((pad & 1) ? 0 : 2 * e1 - 1) + ((pad & 2) ? 0 : sgn[2 * pp + cls] * (2 * e2 - 1));
                            out[((cls * 4 + pad) * 4 + idx) * 32] = T[cls * 5 + m + 2];
                        }
                for (int e = 0; e < g.n_vis_tab * g.nTv; ++e) out[(kGenHid + e) * 32] = T[10 + e];
            }
            if (sgn[2 * pp] < 0) sneg[2 * w] |= 1u << l;
            if (sgn[2 * pp + 1] < 0) sneg[2 * w + 1] |= 1u << l;
            if (!real) continue;
            int sidx = -1;
            for (int s = 0; s < nseg; ++s)
                if ((seg[33 * w + 1 + s] >> 8) == pp) sidx = s;
            if (sidx < 0) {
                sidx = nseg++;
                seg[33 * w + 1 + sidx] = (pp << 8) | l;
            }
            segmask[32 * w + sidx] |= 1u << l;
        }
        seg[33 * w] = nseg;
    }
    // Canonical fast-path tables (crbm_canon.cu): per word and lane, the
    // hidden table indexed by the raw endpoint bits (e1 + 2 e2) and the
    // visible tables indexed by the five raw filter bits of each spin
    // position; the coefficient signs and the field sums are folded in.
    std::vector<uint32_t> ctab;
    if (g.bitplane) {  // threshold planes of each word (layout at kBpTab)
        ctab.assign(static_cast<size_t>(nw) * kCanonTab, 0u);
        for (int w = 0; w < nw; ++w)
            for (int l = 0; l < 32; ++l) {
                const int c = w * 32 + l;
                const int pp = c < p->n_chains ? ctx->chain_param[c] : ctx->chain_param[0];
                const uint32_t* T = &ctx->tables[static_cast<size_t>(pp) * g.nTab];
                uint32_t* out = &ctab[static_cast<size_t>(w) * kCanonTab];
                auto put = [&](int row, uint32_t t) {
                    for (int b = 0; b < 32; ++b) out[row * 32 + b] |= ((t >> (31 - b)) & 1u) << l;
                };
                for (int cls = 0; cls < 2; ++cls)
                    for (int mi = 0; mi < 3; ++mi) put(kBpHidPlanes / 32 + cls * 3 + mi, T[cls * 5 + 2 * mi]);
                if (T[2] != 0x80000000u || T[7] != 0x80000000u) {  // the sweep takes m = 0 as exactly 1/2
                    delete ctx;
                    return fail(nullptr, CRBM_EINVAL, "internal: bit-plane sweep needs thr(0) = 2^31");
                }
                for (int cnt = 0; cnt <= 4; ++cnt)
                    for (int j = 0; j < 2; ++j)
                        put(kBpVisPlanes / 32 + cnt * 2 + j, T[10 + (2 * cnt) * (2 * g.DJp + 1) + 2 * j]);
                for (int cls = 0; cls < 2; ++cls)
                    if (sgn[2 * pp + cls] < 0) out[kBpFlip + cls] |= 1u << l;
            }
    } else if (g.canonical) {
        ctab.assign(static_cast<size_t>(nw) * kCanonTab, 0u);
        for (int w = 0; w < nw; ++w)
            for (int l = 0; l < 32; ++l) {
                const int c = w * 32 + l;
                const int pp = c < p->n_chains ? ctx->chain_param[c] : ctx->chain_param[0];
                const uint32_t* T = &ctx->tables[static_cast<size_t>(pp) * g.nTab];
                uint32_t* out = &ctab[static_cast<size_t>(w) * kCanonTab];
                for (int cls = 0; cls < 2; ++cls)
                    for (int idx = 0; idx < 4; ++idx) {
                        const int e1 = idx & 1, e2 = idx >> 1;
                        const int m = (2 * e1 - 1) + sgn[2 * pp + cls] * (2 * e2 - 1);
                        out[(cls * 4 + idx) * 32 + l] = T[cls * 5 + m + 2];
                    }
                for (int sc = 0; sc < 4; ++sc)
                    for (int idx = 0; idx < 32; ++idx) {
                        int n[2] = {0, 0};
                        for (int slot = 0; slot < 5; ++slot) {
                            const int cls = kCanonSlot[sc][slot][0];
                            const int coef = kCanonSlot[sc][slot][1] ? sgn[2 * pp + cls] : 1;
                            n[cls] += coef * (2 * ((idx >> slot) & 1) - 1);
                        }
                        out[kCanonTh + (sc * 32 + idx) * 32 + l] =
                            T[10 + (n[0] + g.DJ) * (2 * g.DJp + 1) + (n[1] + g.DJp)];
                    }
            }
    }
    // Per-cell records of the canonical SMEM sweep (layout in crbm_internal.h).
    std::vector<uint32_t> crec;
    if (g.bitplane && ctx->layout == CRBM_LAYOUT_SMEM) {
        // hidden node cell*10 + k: its endpoint sites (s1 | s2 << 16); then per
        // spin: its four J incidences and its J' incidence (hidden node | 0x8000
        // when the spin is the second endpoint), its cell and window offset
        // ([0] = J0 | J1 << 16, [1] = J2 | J3 << 16, [2] = J' | cell << 16 | x << 28)
        const size_t nh = static_cast<size_t>(g.n_cells) * 10;
        crec.assign((nh + 3 * static_cast<size_t>(g.N) + 3) & ~static_cast<size_t>(3), 0u);
        std::vector<std::vector<uint32_t>> inc(2 * static_cast<size_t>(g.N));
        for (int c = 0; c < g.n_cells; ++c)
            for (int k = 0; k < 10; ++k) {
                const int i = c / g.Wc, j = c % g.Wc;
                const int s1 = site_index(g, i, j, g.r1[k], g.c1[k]), s2 = site_index(g, i, j, g.r2[k], g.c2[k]);
                crec[static_cast<size_t>(c) * 10 + k] = static_cast<uint32_t>(s1) | (static_cast<uint32_t>(s2) << 16);
                inc[static_cast<size_t>(g.cls[k]) * g.N + s1].push_back(static_cast<uint32_t>(c * 10 + k));
                inc[static_cast<size_t>(g.cls[k]) * g.N + s2].push_back(static_cast<uint32_t>(c * 10 + k) | 0x8000u);
            }
        for (int s = 0; s < g.N; ++s) {
            const std::vector<uint32_t>& a = inc[s];
            const std::vector<uint32_t>& b = inc[static_cast<size_t>(g.N) + s];
            if (a.size() != 4 || b.size() != 1) {
                delete ctx;
                return fail(nullptr, CRBM_EINVAL, "internal: bit-plane records need 4 J and 1 J' incidence per spin");
            }
            const int R = s / g.Lc, C = s % g.Lc;
            const uint32_t cell = static_cast<uint32_t>((R >> 1) * g.Wc + (C >> 1));
            const uint32_t x = static_cast<uint32_t>(2 * (R & 1) + (C & 1));
            uint32_t* o = &crec[nh + 3 * static_cast<size_t>(s)];
            o[0] = a[0] | (a[1] << 16);
            o[1] = a[2] | (a[3] << 16);
            o[2] = b[0] | (cell << 16) | (x << 28);
        }
    } else if (g.canonical && ctx->layout == CRBM_LAYOUT_SMEM) {
        const int L = g.L, W = g.W, Lc = g.Lc, Wc = g.Wc;
        const uint32_t key0 = static_cast<uint32_t>(ctx->seed), key1 = static_cast<uint32_t>(ctx->seed >> 32);
        const uint32_t rk2 = key0 + 0x9E3779B9u, rk4 = key0 + 2u * 0x9E3779B9u;  // round keys 1, 2 (word 0)
        const uint32_t vb = 4u * kCanonSmemV, wb = 4u * static_cast<uint32_t>(kCanonSmemV + g.N);
        auto site = [&](int R, int C) { return vb + 4u * static_cast<uint32_t>((R % L) * Lc + C % Lc); };
        auto hrow = [&](int i, int j) { return wb + 128u * static_cast<uint32_t>(i * Wc + j); };
        crec.assign(static_cast<size_t>(g.n_cells) * kCellRec * 4, 0u);
        for (int i = 0; i < W; ++i)
            for (int j = 0; j < Wc; ++j) {
                uint32_t* o = &crec[static_cast<size_t>(i * Wc + j) * kCellRec * 4];
                const uint64_t m = 0xD2511F53ull * static_cast<uint32_t>(i * Wc + j);
                const uint32_t lo = static_cast<uint32_t>(m), hi = static_cast<uint32_t>(m >> 32) ^ key1;
                uint32_t qh[4], ql[4];  // round-1 products of the calls with tags 0, 1, 2, visible
                const uint32_t tags[4] = {0u, 1u, 2u, kTagVis};
                for (int t = 0; t < 4; ++t) {
                    const uint64_t p = 0xCD9E8D57ull * (hi ^ tags[t]);
                    qh[t] = static_cast<uint32_t>(p >> 32) ^ rk2;
                    ql[t] = static_cast<uint32_t>(p) ^ rk4;
                }
                const int R = 2 * i, C = 2 * j;
                const uint32_t rec[kCellRec * 4] = {
                    site(R, C),     site(R + 1, C), site(R + 2, C),        site(R, C + 2),
                    site(R + 1, C + 2), hrow(i, j), lo,                    qh[2],
                    qh[0],          ql[0],          qh[1],                 ql[1],
                    site(R, C),     site(R + 1, C), hrow(i, j),            hrow((i + W - 1) % W, j),
                    hrow(i, (j + Wc - 1) % Wc), lo, qh[3],                 ql[3],
                    ql[2],          0u,             0u,                    0u};
                std::copy(rec, rec + kCellRec * 4, o);
                if (g.paper) {  // the cell's row of visible draws replaces Q2.hi and Qv.hi
                    const uint32_t pw = 4u * static_cast<uint32_t>(canon_smem_pw_offset(g)) +
                                        256u * static_cast<uint32_t>(i * Wc + j);
                    o[7] = pw;
                    o[18] = pw;
                }
            }
    }
    // Per-cell records of the generic SMEM sweep (layout in crbm_internal.h).
    if (!g.canonical && ctx->layout == CRBM_LAYOUT_SMEM) {
        const GenericSmem gs = generic_smem(g);
        const int Wr = g.W, Wc = g.Wc, nb = g.nb, nP = 2 * g.DJp + 1;
        const size_t nh = static_cast<size_t>(g.n_cells) * nb;
        crec.assign((nh + static_cast<size_t>(g.n_cells) * kGenVisRec) * 4, 0u);
        auto site_off = [&](int s) { return 4u * static_cast<uint32_t>(s >= 0 ? gs.v + s : gs.zero); };
        for (int c = 0; c < g.n_cells; ++c)
            for (int k = 0; k < nb; ++k) {
                const int i = c / Wc, j = c % Wc;
                const int s1 = site_index(g, i, j, g.r1[k], g.c1[k]), s2 = site_index(g, i, j, g.r2[k], g.c2[k]);
                const int pad = (s1 < 0 ? 1 : 0) | (s2 < 0 ? 2 : 0);
                uint32_t* o = &crec[(static_cast<size_t>(c) * nb + k) * 4];
                o[0] = site_off(s1);
                o[1] = site_off(s2);
                o[2] = 4u * static_cast<uint32_t>(gs.tab + static_cast<size_t>((g.cls[k] * 4 + pad) * 4) * 32);
            }
        // incidences (cell, filter, endpoint) of every spin
        std::vector<std::vector<int>> incid(g.N);
        for (int c = 0; c < g.n_cells; ++c)
            for (int k = 0; k < nb; ++k) {
                const int i = c / Wc, j = c % Wc;
                const int s1 = site_index(g, i, j, g.r1[k], g.c1[k]), s2 = site_index(g, i, j, g.r2[k], g.c2[k]);
                if (s1 >= 0) incid[s1].push_back((c * kMaxBonds + k) * 2);
                if (s2 >= 0) incid[s2].push_back((c * kMaxBonds + k) * 2 + 1);
            }
        for (int c = 0; c < g.n_cells; ++c) {
            const int i = c / Wc, j = c % Wc;
            const int iu = i > 0 ? i - 1 : (g.periodic ? Wr - 1 : -1);
            const int jl = j > 0 ? j - 1 : (g.pc ? Wc - 1 : -1);
            const int src[4] = {c, iu >= 0 ? iu * Wc + j : -1, jl >= 0 ? i * Wc + jl : -1,
                                iu >= 0 && jl >= 0 ? iu * Wc + jl : -1};
            uint32_t* o = &crec[(nh + static_cast<size_t>(c) * kGenVisRec) * 4];
            for (int q = 0; q < 4; ++q)
                o[q] = 4u * static_cast<uint32_t>(src[q] >= 0 ? gs.hw + static_cast<size_t>(src[q]) * 16 : gs.zrow);
            for (int x = 0; x < 4; ++x) {
                const int R = 2 * i + (x >> 1), C = 2 * j + (x & 1);
                uint32_t* mj = o + 4 * (1 + 2 * x);
                uint32_t* mp = o + 4 * (2 + 2 * x);
                int deg[2] = {0, 0};
                if (R < g.L && C < g.Lc) {
                    const int s = R * g.Lc + C;
                    for (const int e : incid[s]) {
                        const int cc = e / (2 * kMaxBonds), k = (e / 2) % kMaxBonds, second = e & 1;
                        int q = 0;
                        while (q < 4 && src[q] != cc) ++q;
                        if (q == 4) {
                            delete ctx;
                            return fail(nullptr, CRBM_EINVAL, "internal: incidence outside the cell's windows");
                        }
                        const int cls = g.cls[k];
                        (cls ? mp : mj)[q] |= 1u << (k + 16 * second);
                        ++deg[cls];
                    }
                    o[4 * 10 + x] = site_off(s);
                } else {
                    o[4 * 10 + x] = 4u * static_cast<uint32_t>(gs.zero + 1);
                }
                const int odd_table = (g.n_vis_tab == 2 && (C & 1)) ? g.nTv : 0;  // odd column: second table
                o[4 * 9 + x] = 4u * static_cast<uint32_t>(
                    gs.tab + static_cast<size_t>(kGenHid + odd_table + (g.DJ - deg[0]) * nP + (g.DJp - deg[1])) * 32);
            }
        }
    }
    // Device state.
    cudaGetDevice(&ctx->device);
    DeviceState& d = ctx->d;
    const size_t N = static_cast<size_t>(g.N);
    if ((rc = dalloc(ctx, d.v, nw * N)) || (rc = dalloc(ctx, d.tab, tab.size())) ||
        (rc = dalloc(ctx, d.ctab, ctab.size())) || (rc = dalloc(ctx, d.crec, crec.size() / 4)) ||
        (rc = dalloc(ctx, d.sneg, sneg.size())) || (rc = dalloc(ctx, d.gep, gep.size())) ||
        (rc = dalloc(ctx, d.sums, static_cast<size_t>(npad) * kNSum)) ||
        (rc = dalloc(ctx, d.series, static_cast<size_t>(p->series_len) * npad * 3)) ||
        (rc = dalloc(ctx, d.corr, p->sq_every > 0 ? static_cast<size_t>(p->n_params) * N : 1)) ||
        (rc = dalloc(ctx, d.seg, seg.size())) || (rc = dalloc(ctx, d.segmask, segmask.size())) ||
        (rc = dalloc(ctx, d.spins8, static_cast<size_t>(npad) * N)) ||
        (rc = dalloc(ctx, d.sob, static_cast<size_t>(npad))) || (rc = dalloc(ctx, d.flag, 1)) ||
        (rc = dalloc(ctx, d.sched, 4 + static_cast<size_t>(nw))) ||
        (rc = dalloc(ctx, d.swap_tab, swap_tab.size())) || (rc = dalloc(ctx, d.swap_off, swap_off.size())) ||
        (rc = dalloc(ctx, d.swap_len, swap_len.size())) || (rc = dalloc(ctx, d.wq, wq.size())) ||
        (g.vil && (rc = dalloc(ctx, d.h, static_cast<size_t>(nw) * g.n_cells * 32))) ||
        (g.vil && (rc = dalloc(ctx, d.cnt, static_cast<size_t>(npad) * 3)))) {
        g_create_error = ctx->err;
        free_device(d);
        delete ctx;
        return rc;
    }
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    auto h2d = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    h2d(d.tab, tab.data(), tab.size() * 4);
    h2d(d.ctab, ctab.data(), ctab.size() * 4);
    h2d(d.crec, crec.data(), crec.size() * 4);
    h2d(d.sneg, sneg.data(), sneg.size() * 4);
    h2d(d.gep, gep.data(), gep.size() * 4);
    h2d(d.seg, seg.data(), seg.size() * 4);
    h2d(d.segmask, segmask.data(), segmask.size() * 4);
    h2d(d.swap_tab, swap_tab.data(), swap_tab.size() * 4);
    h2d(d.swap_off, swap_off.data(), swap_off.size() * 4);
    h2d(d.swap_len, swap_len.data(), swap_len.size() * 4);
    h2d(d.wq, wq.data(), wq.size() * 4);
    std::vector<int32_t> ident(static_cast<size_t>(npad));
    for (int c = 0; c < npad; ++c) ident[c] = c & 31;
    h2d(d.sob, ident.data(), ident.size() * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.sums, 0, static_cast<size_t>(npad) * kNSum * 8, st);
    if (e == cudaSuccess && p->series_len)
        e = cudaMemsetAsync(d.series, 0, static_cast<size_t>(p->series_len) * npad * 12, st);
    if (e == cudaSuccess && p->sq_every)
        e = cudaMemsetAsync(d.corr, 0, static_cast<size_t>(p->n_params) * N * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.spins8, 1, static_cast<size_t>(npad) * N, st);
    if (e == cudaSuccess && d.cnt) e = cudaMemsetAsync(d.cnt, 0, static_cast<size_t>(npad) * 12, st);
    if (e == cudaSuccess)
        e = launch_init(g, d.v, nw, static_cast<uint32_t>(ctx->seed),
                        static_cast<uint32_t>(ctx->seed >> 32), st);
    // The staged host vectors go out of scope: finish the copies first.
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        g_create_error = std::string("crbm_create: ") + cudaGetErrorString(e);
        free_device(d);
        delete ctx;
        return CRBM_ECUDA;
    }
    ctx->launches = 1;
    if (!std::getenv("CRBM_WARPS") && ctx->layout == CRBM_LAYOUT_SMEM)
        if (const int w = autotune_lookup(ctx)) ctx->warps = w;  // shape tuned earlier on this GPU
    *out = ctx;
    return CRBM_OK;
}

void crbm_destroy(crbm_ctx* ctx) {
    if (!ctx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != ctx->device) cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_device(ctx->d);
    if (cur != ctx->device) cudaSetDevice(cur);
    delete ctx;
}

int crbm_sweep(crbm_ctx* ctx, int64_t n_sweeps) {
    if (!ctx) return CRBM_EINVAL;
    if (n_sweeps < 0) return fail(ctx, CRBM_EINVAL, "n_sweeps must be >= 0");
    if (ctx->sweeps + n_sweeps > 4294967295LL)
        return fail(ctx, CRBM_EINVAL, "the 32-bit sweep counter of the Philox key would overflow");
    int64_t left = n_sweeps;
    while (left > 0) {
        // Chunks keep one launch within a few seconds on large grids.
        const int chunk = static_cast<int>(std::min<int64_t>(left, 1 << 20));
        const SweepArgs a = fill_sweep_args(ctx, chunk);
        cudaError_t e;
        if (ctx->layout == CRBM_LAYOUT_STREAM) {
            e = launch_sweep_stream(a, ctx->stream, &ctx->launches);
        } else {
            // canonical: persistent grid over (word, chunk) items, chunks of about
            // 1/CRBM_CHUNKS_PER_WORD of the launch (at least 8 sweeps): short
            // enough that the last round leaves few SMs idle, long enough that
            // reloading a word's tables and state stays cheap
            const int chunk = std::max(8, (a.n_sweeps + CRBM_CHUNKS_PER_WORD - 1) / CRBM_CHUNKS_PER_WORD);
            e = ctx->g.bitplane    ? launch_sweep_bitplane(a, ctx->warps, chunk, ctx->d.sched, ctx->stream)
                : ctx->g.canonical ? launch_sweep_canon_persistent(a, ctx->warps, chunk, ctx->d.sched, ctx->stream)
                                   : launch_sweep_generic(a, ctx->warps, ctx->stream);
            ++ctx->launches;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sweep launch");
        const int64_t t0 = ctx->sweeps, t1 = ctx->sweeps + chunk;
        if (ctx->measure_every > 0) ctx->meas += t1 / ctx->measure_every - t0 / ctx->measure_every;
        if (ctx->sq_every > 0) ctx->sq_meas += t1 / ctx->sq_every - t0 / ctx->sq_every;
        ctx->sweeps = t1;
        left -= chunk;
    }
    return CRBM_OK;
}

int64_t crbm_sweep_count(const crbm_ctx* ctx) { return ctx ? ctx->sweeps : -1; }

int64_t crbm_launch_count(const crbm_ctx* ctx) { return ctx ? ctx->launches : -1; }

int crbm_layout(const crbm_ctx* ctx) { return ctx ? ctx->layout : CRBM_EINVAL; }


int crbm_observables(crbm_ctx* ctx, int64_t* out, size_t n_out) {
    if (!ctx || !out) return CRBM_EINVAL;
    const size_t need = static_cast<size_t>(ctx->n_chains) * kNSum;
    if (n_out < need) return fail(ctx, CRBM_EINVAL, "output buffer too small");
    cudaError_t e = cudaMemcpyAsync(out, ctx->d.sums, need * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? CRBM_OK : cuda_fail(ctx, e, "crbm_observables");
}

int crbm_series(crbm_ctx* ctx, int32_t* out, size_t n_out) {
    if (!ctx || !out) return CRBM_EINVAL;
    const size_t per = static_cast<size_t>(ctx->n_chains) * 3;
    if (n_out < per * ctx->series_len) return fail(ctx, CRBM_EINVAL, "output buffer too small");
    cudaError_t e = cudaSuccess;
    const size_t pitch = static_cast<size_t>(ctx->n_words) * 32 * 3 * 4;
    if (ctx->series_len > 0)
        e = cudaMemcpy2DAsync(out, per * 4, ctx->d.series, pitch, per * 4, ctx->series_len,
                              cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? CRBM_OK : cuda_fail(ctx, e, "crbm_series");
}

int crbm_correlations(crbm_ctx* ctx, int64_t* out, size_t n_out, int64_t* n_samples) {
    if (!ctx || !out) return CRBM_EINVAL;
    if (ctx->sq_every <= 0) return fail(ctx, CRBM_EINVAL, "context created with sq_every = 0");
    const size_t need = static_cast<size_t>(ctx->n_params) * ctx->g.N;
    if (n_out < need) return fail(ctx, CRBM_EINVAL, "output buffer too small");
    cudaError_t e = cudaMemcpyAsync(out, ctx->d.corr, need * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crbm_correlations");
    if (n_samples) {
        std::vector<int64_t> per(ctx->n_params, 0);
        for (int c = 0; c < ctx->n_chains; ++c) per[ctx->chain_param[c]]++;
        for (int i = 0; i < ctx->n_params; ++i) n_samples[i] = per[i] * ctx->sq_meas;
    }
    return CRBM_OK;
}

int crbm_structure_factor(crbm_ctx* ctx, double* out, size_t n_out) {
    if (!ctx || !out) return CRBM_EINVAL;
    const int L = ctx->g.L, N = ctx->g.N;
    const size_t need = static_cast<size_t>(ctx->n_params) * N;
    if (n_out < need) return fail(ctx, CRBM_EINVAL, "output buffer too small");
    std::vector<int64_t> corr(need), ns(ctx->n_params);
    const int rc = crbm_correlations(ctx, corr.data(), need, ns.data());
    if (rc) return rc;
    // S(q) = (1/N) sum_d <C(d)> cos(q.d): C(d) = C(-d), so the sine part cancels.
    std::vector<double> cosk(L);
    for (int k = 0; k < L; ++k) cosk[k] = std::cos(6.283185307179586476925286766559 * k / L);
    for (int p = 0; p < ctx->n_params; ++p) {
        const int64_t* c = &corr[static_cast<size_t>(p) * N];
        for (int nR = 0; nR < L; ++nR)
            for (int nC = 0; nC < L; ++nC) {
                double s = 0.0;
                for (int dR = 0; dR < L; ++dR)
                    for (int dC = 0; dC < L; ++dC)
                        s += static_cast<double>(c[dR * L + dC]) * cosk[(nR * dR + nC * dC) % L];
                out[static_cast<size_t>(p) * N + nR * L + nC] = ns[p] > 0 ? s / (static_cast<double>(ns[p]) * N) : 0.0;
            }
    }
    return CRBM_OK;
}

int crbm_reset_observables(crbm_ctx* ctx) {
    if (!ctx) return CRBM_EINVAL;
    const size_t npad = static_cast<size_t>(ctx->n_words) * 32;
    cudaError_t e = cudaMemsetAsync(ctx->d.sums, 0, npad * kNSum * 8, ctx->stream);
    if (e == cudaSuccess && ctx->series_len)
        e = cudaMemsetAsync(ctx->d.series, 0, static_cast<size_t>(ctx->series_len) * npad * 12, ctx->stream);
    if (e == cudaSuccess && ctx->sq_every)
        e = cudaMemsetAsync(ctx->d.corr, 0, static_cast<size_t>(ctx->n_params) * ctx->g.N * 8, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crbm_reset_observables");
    ctx->meas = 0;
    ctx->sq_meas = 0;
    return CRBM_OK;
}

int crbm_get_spins(crbm_ctx* ctx, int8_t* out, size_t n_out) {
    if (!ctx || !out) return CRBM_EINVAL;
    const size_t need = static_cast<size_t>(ctx->n_chains) * ctx->g.N;
    if (n_out < need) return fail(ctx, CRBM_EINVAL, "output buffer too small");
    cudaError_t e = launch_unpack(ctx->g, ctx->d.v, ctx->d.spins8, ctx->n_words, ctx->stream);
    ++ctx->launches;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, ctx->d.spins8, need, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? CRBM_OK : cuda_fail(ctx, e, "crbm_get_spins");
}

int crbm_set_spins(crbm_ctx* ctx, const int8_t* in, size_t n_in) {
    if (!ctx || !in) return CRBM_EINVAL;
    const size_t need = static_cast<size_t>(ctx->n_chains) * ctx->g.N;
    if (n_in < need) return fail(ctx, CRBM_EINVAL, "input buffer too small");
    // the values are checked on the device, and the spins packed only when all are +-1
    int bad = 0;
    cudaError_t e = cudaMemcpyAsync(ctx->d.spins8, in, need, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_check_spins(ctx->d.spins8, need, ctx->d.flag, ctx->stream);
    if (e == cudaSuccess)
        e = launch_pack(ctx->g, ctx->d.spins8, ctx->d.v, ctx->n_words, ctx->d.flag, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, ctx->d.flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    ctx->launches += 2;
    // the caller may free `in` on return
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crbm_set_spins");
    return bad ? fail(ctx, CRBM_EINVAL, "spins must be +1 or -1") : CRBM_OK;
}

int crbm_get_permutation(crbm_ctx* ctx, int32_t* out, size_t n_out) {
    if (!ctx || !out) return CRBM_EINVAL;
    if (n_out < static_cast<size_t>(ctx->n_chains)) return fail(ctx, CRBM_EINVAL, "output buffer too small");
    cudaError_t e = cudaMemcpyAsync(out, ctx->d.sob, static_cast<size_t>(ctx->n_chains) * 4,
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? CRBM_OK : cuda_fail(ctx, e, "crbm_get_permutation");
}

int crbm_set_targets(crbm_ctx* ctx, const int64_t* e_target, int32_t n) {
    if (!ctx || !e_target || n != ctx->n_params) return fail(ctx, CRBM_EINVAL, "need one target per parameter point");
    const size_t np = static_cast<size_t>(ctx->n_words) * 32;
    DeviceState& d = ctx->d;
    int rc = CRBM_OK;
    // the sweeps record first hits only where both buffers exist and hold targets: a failed
    // call leaves neither behind
    auto drop = [&]() {
        cudaFree(d.hit);
        cudaFree(d.hit_q);
        d.hit = nullptr;
        d.hit_q = nullptr;
    };
    if (!d.hit) {
        if ((rc = dalloc(ctx, d.hit, 2 * np))) return rc;
        if ((rc = dalloc(ctx, d.hit_q, 4 * np))) {
            drop();
            return rc;
        }
    }
    std::vector<int64_t> ht(2 * np);
    std::vector<int32_t> hq(4 * np, 0);
    for (size_t c = 0; c < np; ++c) {
        const bool real = c < static_cast<size_t>(ctx->n_chains);
        const int pp = real ? ctx->chain_param[c] : 0;
        ht[2 * c] = real ? e_target[pp] : INT64_MIN;  // padding chains never count
        ht[2 * c + 1] = -1;
        hq[4 * c] = ctx->q[0][pp];
        hq[4 * c + 1] = ctx->q[1][pp];
        hq[4 * c + 2] = ctx->q[2][pp];
    }
    cudaError_t e = cudaMemcpyAsync(d.hit, ht.data(), ht.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.hit_q, hq.data(), hq.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        drop();
        return cuda_fail(ctx, e, "crbm_set_targets");
    }
    return CRBM_OK;
}

int crbm_first_hits(crbm_ctx* ctx, int64_t* out, size_t n_out) {
    if (!ctx || !out) return CRBM_EINVAL;
    if (!ctx->d.hit) return fail(ctx, CRBM_EINVAL, "no targets set (crbm_set_targets)");
    if (n_out < static_cast<size_t>(ctx->n_chains)) return fail(ctx, CRBM_EINVAL, "output buffer too small");
    std::vector<int64_t> ht(2 * static_cast<size_t>(ctx->n_chains));
    cudaError_t e = cudaMemcpyAsync(ht.data(), ctx->d.hit, ht.size() * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crbm_first_hits");
    for (int c = 0; c < ctx->n_chains; ++c) out[c] = ht[2 * static_cast<size_t>(c) + 1];
    return CRBM_OK;
}

int crbm_get_tables(crbm_ctx* ctx, uint32_t* out, size_t n_out, int32_t* dims) {
    if (!ctx) return CRBM_EINVAL;
    if (dims) {
        dims[0] = ctx->g.DJ;
        dims[1] = ctx->g.DJp;
    }
    if (!out) return CRBM_OK;
    if (n_out < ctx->tables.size()) return fail(ctx, CRBM_EINVAL, "output buffer too small");
    std::memcpy(out, ctx->tables.data(), ctx->tables.size() * 4);
    return CRBM_OK;
}

// Checkpoint layout: header of 16 int64, then packed spins [n_words][N] u32,
// sums [n_words*32][11] i64, series [series_len][n_words*32][3] i32,
// correlations [n_params][N] i64 (when sq_every > 0).
int crbm_save(crbm_ctx* ctx, void* buf, size_t* n) {
    if (!ctx || !n) return CRBM_EINVAL;
    const size_t npad = static_cast<size_t>(ctx->n_words) * 32, N = ctx->g.N;
    const size_t b_v = ctx->n_words * N * 4, b_s = npad * kNSum * 8,
                 b_t = static_cast<size_t>(ctx->series_len) * npad * 12,
                 b_c = ctx->sq_every ? static_cast<size_t>(ctx->n_params) * N * 8 : 0;
    const size_t b_p = npad * 4;
    const size_t total = 16 * 8 + b_v + b_s + b_t + b_c + b_p;
    if (!buf) {
        *n = total;
        return CRBM_OK;
    }
    if (*n < total) return fail(ctx, CRBM_EINVAL, "checkpoint buffer too small");
    int64_t hdr[16] = {0x4d425243 /* "CRBM" */, 1, ctx->g.L, ctx->n_chains, ctx->n_params,
                       static_cast<int64_t>(ctx->seed), ctx->sweeps, ctx->meas, ctx->sq_meas,
                       ctx->series_len, ctx->sq_every, ctx->measure_every, ctx->g.nb,
                       ctx->g.periodic | (ctx->g.pc << 1) | (static_cast<int64_t>(ctx->g.Lc) << 2), ctx->swap_every,
                       ctx->g.paper | (ctx->g.bitplane << 1)};
    char* p = static_cast<char*>(buf);
    std::memcpy(p, hdr, sizeof(hdr));
    cudaError_t e = cudaMemcpyAsync(p + 128, ctx->d.v, b_v, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + 128 + b_v, ctx->d.sums, b_s, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && b_t)
        e = cudaMemcpyAsync(p + 128 + b_v + b_s, ctx->d.series, b_t, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && b_c)
        e = cudaMemcpyAsync(p + 128 + b_v + b_s + b_t, ctx->d.corr, b_c, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p + 128 + b_v + b_s + b_t + b_c, ctx->d.sob, b_p, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crbm_save");
    *n = total;
    return CRBM_OK;
}

int crbm_load(crbm_ctx* ctx, const void* buf, size_t n) {
    if (!ctx || !buf) return CRBM_EINVAL;
    size_t need = 0;
    crbm_save(ctx, nullptr, &need);
    if (n < need) return fail(ctx, CRBM_EINVAL, "checkpoint too small for this context");
    int64_t hdr[16];
    std::memcpy(hdr, buf, sizeof(hdr));
    if (hdr[0] != 0x4d425243 || hdr[1] != 1 || hdr[2] != ctx->g.L || hdr[3] != ctx->n_chains ||
        hdr[4] != ctx->n_params || hdr[5] != static_cast<int64_t>(ctx->seed) ||
        hdr[9] != ctx->series_len || hdr[10] != ctx->sq_every || hdr[11] != ctx->measure_every ||
        hdr[12] != ctx->g.nb ||
        hdr[13] != (ctx->g.periodic | (ctx->g.pc << 1) | (static_cast<int64_t>(ctx->g.Lc) << 2)) ||
        hdr[14] != ctx->swap_every ||
        hdr[15] != (ctx->g.paper | (ctx->g.bitplane << 1)))
        return fail(ctx, CRBM_EINVAL, "checkpoint does not match this context");
    const size_t npad = static_cast<size_t>(ctx->n_words) * 32, N = ctx->g.N;
    const size_t b_v = ctx->n_words * N * 4, b_s = npad * kNSum * 8,
                 b_t = static_cast<size_t>(ctx->series_len) * npad * 12,
                 b_c = ctx->sq_every ? static_cast<size_t>(ctx->n_params) * N * 8 : 0;
    const char* p = static_cast<const char*>(buf);
    cudaError_t e = cudaMemcpyAsync(ctx->d.v, p + 128, b_v, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d.sums, p + 128 + b_v, b_s, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && b_t)
        e = cudaMemcpyAsync(ctx->d.series, p + 128 + b_v + b_s, b_t, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && b_c)
        e = cudaMemcpyAsync(ctx->d.corr, p + 128 + b_v + b_s + b_t, b_c, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d.sob, p + 128 + b_v + b_s + b_t + b_c, npad * 4, cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "crbm_load");
    ctx->sweeps = hdr[6];
    ctx->meas = hdr[7];
    ctx->sq_meas = hdr[8];
    return CRBM_OK;
}

int crbm_philox(const uint32_t* in, uint32_t* out, size_t n) {
    if (!in || !out || n > (1u << 26)) return fail(nullptr, CRBM_EINVAL, "crbm_philox: bad arguments");
    if (n == 0) return CRBM_OK;
    uint32_t *din = nullptr, *dout = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&din), n * 24) != cudaSuccess)
        return fail(nullptr, CRBM_ENOMEM, "crbm_philox: cudaMalloc");
    if (cudaMalloc(reinterpret_cast<void**>(&dout), n * 16) != cudaSuccess) {
        cudaFree(din);
        return fail(nullptr, CRBM_ENOMEM, "crbm_philox: cudaMalloc");
    }
    cudaError_t e = cudaMemcpy(din, in, n * 24, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox(din, dout, static_cast<int>(n), nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
    return e == cudaSuccess ? CRBM_OK : cuda_fail(nullptr, e, "crbm_philox");
}

int crbm_philox_stream(uint32_t* sink, int32_t n_blocks, int32_t threads, int32_t calls, uint64_t seed,
                       void* stream) {
    if (!sink || n_blocks < 1 || n_blocks > (1 << 20) || threads < 32 || threads > 1024 || threads % 32 ||
        calls < 0 || static_cast<int64_t>(n_blocks) * threads > (1LL << 31))
        return fail(nullptr, CRBM_EINVAL, "crbm_philox_stream: bad arguments");
    const cudaError_t e = launch_philox_stream(sink, n_blocks, threads, calls, static_cast<uint32_t>(seed),
                                               static_cast<uint32_t>(seed >> 32), static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CRBM_OK : cuda_fail(nullptr, e, "crbm_philox_stream");
}

const char* crbm_last_error(const crbm_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
