// crbm_sweep_stream_noalloc: the streamed two-phase sweep without any
// allocation, for callers that cannot call cudaMalloc -- for example code
// that runs inside another framework's memory pool or allocator hooks, or a
// service whose device memory is budgeted and fixed at start-up.
//
// The caller passes the spins (device memory it owns); everything else the
// sweep needs beyond its inputs and outputs -- the lane-expanded threshold
// tables and the hidden words written by the first phase and read by the
// second -- lives in g_noalloc_scratch, one fixed array in this library's
// device image.  Every GPU that loads the library holds the array until the
// process exits.
#include <mutex>

#include "../../include/crbm.h"
#include "crbm_internal.h"

namespace {

using namespace crbm;

constexpr size_t kScratchWords = CRBM_NOALLOC_SCRATCH_BYTES / sizeof(uint32_t);

// Scratch of the no-allocation sweep: per 32-chain word, kCanonTab table
// words, then the lanes' hidden words of every word ([n_words][n_cells][32]).
__device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
// Device address of g_noalloc_scratch per device, stored only once the
// lookup has succeeded (a failed lookup is retried by the next call).
std::mutex g_setup_mutex;
uint32_t* g_scratch_addr[kMaxDevices];
// Failures report only their code (no message string: that would allocate).
int noalloc_fail(int code, const char*) { return code; }

}  // namespace

extern "C" int crbm_sweep_stream_noalloc(const crbm_params* p, uint32_t* v, int64_t sweep0,
                                         int64_t n_sweeps) {
    if (!p || !v) return noalloc_fail(CRBM_EINVAL, "null argument");
    if (p->L < 4 || p->L > 4096 || (p->L & 1) || !p->periodic || p->bonds)
        return noalloc_fail(CRBM_EINVAL,
                            "needs an even L in 4..4096, periodic, and the ten SS filters (bonds = NULL)");
    if ((p->L_cols != 0 && p->L_cols != p->L) ||
        (p->periodic_cols != CRBM_BC_AS_ROWS && p->periodic_cols != CRBM_BC_PERIODIC) || p->h_odd ||
        (p->precision != CRBM_PRECISION_EXACT && p->precision != CRBM_PRECISION_PAPER) || p->rng != CRBM_RNG_LANE)
        return noalloc_fail(CRBM_EINVAL,
                            "needs a square periodic lattice, one field, a known precision and lane uniforms");
    if (p->n_params < 1 || !p->J || !p->Jp || !p->h || !p->beta || p->n_chains < 1 || p->n_chains > (1 << 30))
        return noalloc_fail(CRBM_EINVAL, "need n_params >= 1, the four parameter arrays and 1 <= n_chains <= 2^30");
    if (sweep0 < 0 || n_sweeps < 0 || n_sweeps > 2147483647LL || sweep0 + n_sweeps > 4294967295LL)
        return noalloc_fail(CRBM_EINVAL, "sweep range outside the 32-bit Philox sweep counter");
    const int L = p->L, W = L / 2, N = L * L, n_cells = W * W;
    const int n_words = 2 * ((p->n_chains + 63) / 64);
    const size_t need = static_cast<size_t>(n_words) * kCanonTab + static_cast<size_t>(n_words) * n_cells * 32;
    if (need > kScratchWords)
        return noalloc_fail(CRBM_EUNSUPPORTED,
                            "lattice and chain count need more than CRBM_NOALLOC_SCRATCH_BYTES of scratch "
                            "(4 bytes x n_words x (4352 + 32 (L/2)^2), n_words = 2 ceil(n_chains/64))");
    for (int c = 0; p->chain_param && c < p->n_chains; ++c)
        if (p->chain_param[c] < 0 || p->chain_param[c] >= p->n_params)
            return noalloc_fail(CRBM_EINVAL, "chain_param out of range");
    for (int i = 0; i < p->n_params; ++i) {
        int32_t q;
        if (!host_to_q4(p->J[i], q) || !host_to_q4(p->Jp[i], q) || !host_to_q4(p->h[i], q) ||
            !(p->beta[i] >= 0.0) || !(p->beta[i] <= 1.0e6))
            return noalloc_fail(CRBM_EINVAL, "J, J', h must be finite with |16 x| <= 2047, beta in [0, 1e6]");
    }

    // One-time set-up per device, with that device current: the host-side
    // name of g_noalloc_scratch is not a device address, so fetch it.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(CRBM_ECUDA, "cudaGetDevice failed or device index too large");
    uint32_t* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) == cudaSuccess)
                g_scratch_addr[dev] = static_cast<uint32_t*>(ptr);
        }
        scratch = g_scratch_addr[dev];
    }
    if (!scratch) return noalloc_fail(CRBM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    cudaStream_t st = static_cast<cudaStream_t>(p->stream);

    Geometry g{};
    g.L = L;
    g.W = W;
    g.Lc = L;
    g.Wc = W;
    g.pc = 1;
    g.n_vis_tab = 1;
    g.N = N;
    g.n_cells = n_cells;
    g.nb = 10;
    g.n_calls = 3;
    g.periodic = 1;
    g.canonical = 1;
    g.DJ = 4;
    g.DJp = 1;
    g.nTv = 27;
    g.nTab = 37;
    g.n_real_bonds[0] = 2 * N;
    g.n_real_bonds[1] = N / 2;
    g.vil = 1;
    g.paper = p->precision == CRBM_PRECISION_PAPER ? 1 : 0;

    // Lane tables, one word at a time from a stack buffer (a pageable copy
    // has been staged when cudaMemcpyAsync returns, so the buffer is reused).
    uint32_t buf[kCanonTab];
    uint32_t T[37];
    int sgn[2];
    for (int w = 0; w < n_words && e == cudaSuccess; ++w) {
        for (int l = 0; l < 32; ++l) {
            const int c = w * 32 + l;
            const int cc = c < p->n_chains ? c : 0;
            const int pp = p->chain_param
                               ? p->chain_param[cc]
                               : static_cast<int>(static_cast<int64_t>(cc) * p->n_params / p->n_chains);
            int32_t qJ = 0, qJp = 0, qh = 0;
            host_to_q4(p->J[pp], qJ);
            host_to_q4(p->Jp[pp], qJp);
            host_to_q4(p->h[pp], qh);
            host_point_tables(g, p->beta[pp], qJ, qJp, qh, T, sgn);
            for (int cls = 0; cls < 2; ++cls)
                for (int idx = 0; idx < 4; ++idx) {
                    const int m = (2 * (idx & 1) - 1) + sgn[cls] * (2 * (idx >> 1) - 1);
                    buf[(cls * 4 + idx) * 32 + l] = T[cls * 5 + m + 2];
                }
            for (int sc = 0; sc < 4; ++sc)
                for (int idx = 0; idx < 32; ++idx) {
                    int n[2] = {0, 0};
                    for (int slot = 0; slot < 5; ++slot) {
                        const int cls = kCanonSlot[sc][slot][0];
                        const int coef = kCanonSlot[sc][slot][1] ? sgn[cls] : 1;
                        n[cls] += coef * (2 * ((idx >> slot) & 1) - 1);
                    }
                    buf[kCanonTh + (sc * 32 + idx) * 32 + l] = T[10 + (n[0] + 4) * 3 + (n[1] + 1)];
                }
        }
        e = cudaMemcpyAsync(scratch + static_cast<size_t>(w) * kCanonTab, buf, sizeof(buf),
                            cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return noalloc_fail(CRBM_ECUDA, "table upload failed");

    SweepArgs a{};
    a.g = g;
    a.v = v;
    a.ctab = scratch;
    a.h = scratch + static_cast<size_t>(n_words) * kCanonTab;
    a.n_words = n_words;
    a.n_chains_padded = n_words * 32;
    a.key0 = static_cast<uint32_t>(p->seed);
    a.key1 = static_cast<uint32_t>(p->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.rk[2 * r] = a.key0 + static_cast<uint32_t>(r) * 0x9E3779B9u;
        a.rk[2 * r + 1] = a.key1 + static_cast<uint32_t>(r) * 0xBB67AE85u;
    }
    a.t0 = static_cast<uint32_t>(sweep0);
    a.n_sweeps = static_cast<int>(n_sweeps);
    a.measure_every = 0;  // spins only: no observables are accumulated
    int64_t launches = 0;
    e = launch_sweep_stream(a, st, &launches);
    if (e != cudaSuccess) return noalloc_fail(CRBM_ECUDA, cudaGetErrorString(e));
    return CRBM_OK;
}
