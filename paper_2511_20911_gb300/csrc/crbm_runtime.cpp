// Native runtime around the sweep kernels: the autotuner (CTA shape per
// lattice shape, timed on scratch copies of a context's state and cached per
// GPU in a text file) and batched launches (several contexts, mixed lattice
// sizes and tempering ladders, in one kernel launch captured in a CUDA graph).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "crbm_context.h"

using namespace crbm;

namespace {

// ----------------------------------------------------------------- cache
// One line per tuned shape: "<key> <warps>"; the key names the GPU, the
// lattice, the filter set and the number of packed words.
std::mutex g_cache_mutex;

std::string cache_path() {
    if (const char* p = std::getenv("CRBM_AUTOTUNE_CACHE")) return p;
    const char* home = std::getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/crbm_autotune.txt";
}

std::string shape_key(const crbm_ctx* ctx) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, ctx->device);
    std::ostringstream k;
    k << prop.name << "|sm" << prop.multiProcessorCount << "|L" << ctx->g.L << "|p" << ctx->g.periodic << "|c"
      << ctx->g.canonical << "|nb" << ctx->g.nb << "|w" << ctx->n_words << "|x" << (ctx->swap_every > 0)
      << "|q" << ctx->g.paper << "|bp" << ctx->g.bitplane << "|Lc" << ctx->g.Lc << "|pc" << ctx->g.pc << "|v" << ctx->g.n_vis_tab;
    std::string s = k.str();
    std::replace(s.begin(), s.end(), ' ', '_');
    return s;
}

// Shared memory of a batch member's body (bit-plane records from global memory).
size_t member_smem(const crbm_ctx* ctx) {
    return ctx->g.bitplane ? smem_bytes_bitplane(ctx->g, false)
           : ctx->g.canonical ? smem_bytes_canon(ctx->g)
                              : smem_bytes_generic(ctx->g);
}

int smem_ok(const crbm_ctx* ctx) { return member_smem(ctx) <= 227 * 1024; }

cudaError_t launch_one(const SweepArgs& a, const crbm_ctx* ctx, int warps) {
    if (!ctx->g.canonical) return launch_sweep_generic(a, warps, ctx->stream);
    const int chunk = std::max(8, (a.n_sweeps + CRBM_CHUNKS_PER_WORD - 1) / CRBM_CHUNKS_PER_WORD);  // as crbm_sweep does
    if (ctx->g.bitplane) return launch_sweep_bitplane(a, warps, chunk, ctx->d.sched, ctx->stream);
    return launch_sweep_canon_persistent(a, warps, chunk, ctx->d.sched, ctx->stream);
}

}  // namespace

namespace crbm {
int autotune_lookup(const crbm_ctx* ctx) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    std::ifstream f(cache_path());
    if (!f) return 0;
    const std::string key = shape_key(ctx);
    std::string k;
    int w = 0, found = 0;
    while (f >> k >> w)
        if (k == key && w >= 1 && w <= kMaxSweepWarps) found = w;  // last entry wins
    return found;
}
}  // namespace crbm

extern "C" {

int crbm_autotune(crbm_ctx* ctx, int64_t probe_sweeps, int32_t* best_warps) {
    if (!ctx) return CRBM_EINVAL;
    if (ctx->layout != CRBM_LAYOUT_SMEM) {
        ctx->err = "the autotuner chooses CTA shapes of the SMEM layout";
        return CRBM_EUNSUPPORTED;
    }
    if (probe_sweeps < 1 || probe_sweeps > 100000) {
        ctx->err = "probe_sweeps must be in 1..100000";
        return CRBM_EINVAL;
    }
    const size_t npad = static_cast<size_t>(ctx->n_words) * 32, N = ctx->g.N;
    uint32_t* v2 = nullptr;
    int64_t* s2 = nullptr;
    int32_t* p2 = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&v2), ctx->n_words * N * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s2), npad * kNSum * 8);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p2), npad * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best = ctx->warps;
    float best_ms = 1e30f;
    // (in-between counts such as 9, 11, 13, 18 and 26, which divide some half-steps' node groups
    // evenly, measured no faster on the L=18 grid lines)
    const int cand[] = {2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32};
    for (int w : cand) {
        if (e != cudaSuccess) break;
        // the generic kernel is built for CTAs of at most 512 threads
        if (w > std::max(1, ctx->g.n_cells) || w > (ctx->g.canonical ? kMaxSweepWarps : 16)) continue;
        // scratch copies: the tuning sweeps never touch the context's chains
        e = cudaMemcpyAsync(v2, ctx->d.v, ctx->n_words * N * 4, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s2, 0, npad * kNSum * 8, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p2, ctx->d.sob, npad * 4, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) break;
        SweepArgs a = fill_sweep_args(ctx, static_cast<int>(probe_sweeps));
        a.v = v2;
        a.sums = s2;
        a.sob = p2;
        a.series_len = 0;
        a.sq_every = 0;
        a.clock = nullptr;
        a.hit = nullptr;  // the probes record no time to solution
        a.n_sweeps = static_cast<int>(std::max<int64_t>(1, probe_sweeps / 4));
        e = launch_one(a, ctx, w);  // warm-up
        a.n_sweeps = static_cast<int>(probe_sweeps);
        if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
        if (e == cudaSuccess) e = launch_one(a, ctx, w);
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = w;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(v2);
    cudaFree(s2);
    cudaFree(p2);
    if (e != cudaSuccess) {
        ctx->err = std::string("crbm_autotune: ") + cudaGetErrorString(e);
        return CRBM_ECUDA;
    }
    ctx->warps = best;
    if (best_warps) *best_warps = best;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    const std::string path = cache_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // best effort
    if (FILE* f = std::fopen(path.c_str(), "a")) {
        std::fprintf(f, "%s %d\n", shape_key(ctx).c_str(), best);
        std::fclose(f);
    }
    return CRBM_OK;
}

int crbm_warps(const crbm_ctx* ctx) { return ctx ? ctx->warps : CRBM_EINVAL; }

}  // extern "C"

// ----------------------------------------------------------------- batches
struct crbm_batch {
    std::vector<crbm_ctx*> ctx;
    cudaStream_t stream = nullptr;     // the contexts' common stream
    cudaStream_t capture = nullptr;    // private stream the graph is captured on
    int4* items = nullptr;             // per CTA: (member or -1, word, band, bands)
    int n_items = 0;
    int64_t* clock = nullptr;          // device [n][2]
    int* every = nullptr;              // device [n]
    std::vector<int64_t> mirror;       // host view of clock
    std::vector<int64_t> staged;       // pinned-free staging for clock uploads
    int threads = 0;
    size_t smem = 0;
    int smem_rec = 0;                  // canonical members stage their records in shared memory
    int modes = 0;                     // kBatchPaper | kBatchBitplane: member kinds present
    int cluster = 1;                   // CTAs per item (thread-block cluster)
    std::vector<int> bands;            // per member: CTAs its words are split over
    cudaGraphExec_t exec = nullptr;
    int64_t graph_n = -1;
    std::vector<const int64_t*> hit_seen;  // per member: first-hit records the graph was captured with
    std::string err;
};

namespace {
thread_local std::string g_batch_create_error;

void batch_free(crbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->items);
    cudaFree(b->clock);
    cudaFree(b->every);
    delete b;
}
}  // namespace

extern "C" {

int crbm_batch_create(crbm_batch** out, crbm_ctx* const* ctxs, int32_t n_ctx) {
    if (!out || !ctxs || n_ctx < 1 || n_ctx > kMaxBatch) {
        g_batch_create_error = "need 1..CRBM_BATCH_MAX contexts";
        return CRBM_EINVAL;
    }
    *out = nullptr;
    crbm_batch* b = new (std::nothrow) crbm_batch();
    if (!b) return CRBM_ENOMEM;
    int warps = 1;
    for (int c = 0; c < n_ctx; ++c) {
        crbm_ctx* x = ctxs[c];
        if (!x || x->layout != CRBM_LAYOUT_SMEM || !smem_ok(x) || x->stream != ctxs[0]->stream ||
            x->device != ctxs[0]->device || std::count(ctxs, ctxs + c, x)) {
            g_batch_create_error = "batch members must be distinct SMEM-layout contexts on one device and stream";
            delete b;
            return CRBM_EINVAL;
        }
        b->ctx.push_back(x);
        warps = std::max(warps, x->warps);
        b->smem = std::max(b->smem, member_smem(x));
        if (x->g.paper) b->modes |= kBatchPaper;
        if (x->g.bitplane) b->modes |= kBatchBitplane;
    }
    // stage the canonical members' per-cell records in shared memory when all of them fit
    size_t with_rec = b->smem;
    for (auto* x : b->ctx)
        if (x->g.canonical && !x->g.bitplane)
            with_rec = std::max(with_rec, sizeof(uint32_t) * canon_smem_rec_offset(x->g) +
                                              sizeof(uint4) * static_cast<size_t>(x->g.n_cells) * kCellRec);
    if (with_rec <= 227 * 1024) {
        b->smem = with_rec;
        b->smem_rec = 1;
    }
    b->threads = 32 * warps;
    // Thread-block clusters of `cluster` CTAs (CRBM_BATCH_CLUSTER, default 8,
    // a power of two; 1 = none).  A canonical exact-precision, lane-uniform
    // member without correlations is
    // split into B bands of cell rows per word, B the smallest power of two
    // (at most the cluster size and W) that brings its cells per CTA down to
    // the heaviest member's when split over a whole cluster (at least 16);
    // its words then share clusters, cluster/B words per cluster, padded with
    // ranks of the same member that only keep the barriers.  Other words are
    // packed one per CTA.  Falls back to no clusters when none can be resident.
    int cluster = 8;
    if (const char* env = std::getenv("CRBM_BATCH_CLUSTER")) cluster = std::max(1, std::min(8, std::atoi(env)));
    while (cluster & (cluster - 1)) --cluster;  // a power of two
    if (cluster > 1 && batch_max_active_clusters(cluster, b->threads, b->smem, b->modes) < 1) cluster = 1;
    auto splittable = [&](const crbm_ctx* x) {
        return cluster > 1 && x->g.canonical && !x->g.paper && !x->g.bitplane && x->sq_every == 0;
    };
    int target = 16;
    for (auto* x : b->ctx)
        if (splittable(x)) target = std::max(target, x->g.n_cells / std::min(cluster, x->g.W));
    for (auto* x : b->ctx) {
        int nb = 1;
        if (splittable(x))
            while (nb < cluster && 2 * nb <= x->g.W && x->g.n_cells / nb > target) nb *= 2;
        b->bands.push_back(nb);
    }
    if (*std::max_element(b->bands.begin(), b->bands.end()) == 1) cluster = 1;  // nothing to split
    // tasks: split words cluster by cluster (heaviest member first), then
    // whole words one per CTA (heaviest first), padded to whole clusters
    std::vector<int> order(n_ctx);
    for (int c = 0; c < n_ctx; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
        return b->ctx[p]->g.n_cells / b->bands[p] > b->ctx[q]->g.n_cells / b->bands[q];
    });
    std::vector<int4> items;
    std::vector<std::pair<int64_t, int4>> whole;
    for (int c : order) {
        const crbm_ctx* x = b->ctx[c];
        const int nb = b->bands[c];
        if (nb == 1) {
            const int64_t cost = static_cast<int64_t>(x->g.n_cells) * (x->g.canonical ? 2 : 3);
            for (int w = 0; w < x->n_words; ++w) whole.push_back({cost, make_int4(c, w, 0, 1)});
            continue;
        }
        const int per = cluster / nb;  // words per cluster
        for (int w0 = 0; w0 < x->n_words; w0 += per)
            for (int k = 0; k < per; ++k)
                for (int r = 0; r < nb; ++r)
                    items.push_back(w0 + k < x->n_words ? make_int4(c, w0 + k, r, nb) : make_int4(c, 0, nb, nb));
    }
    std::stable_sort(whole.begin(), whole.end(),
                     [](const std::pair<int64_t, int4>& p, const std::pair<int64_t, int4>& q) { return p.first > q.first; });
    for (auto& p : whole) items.push_back(p.second);
    while (items.size() % static_cast<size_t>(cluster)) items.push_back(make_int4(-1, 0, 0, 1));
    b->cluster = cluster;
    std::vector<int> every;
    for (auto* x : b->ctx) every.push_back(x->measure_every);
    b->stream = ctxs[0]->stream;
    b->n_items = static_cast<int>(items.size());
    b->mirror.assign(2 * n_ctx, -1);
    b->hit_seen.assign(n_ctx, nullptr);
    b->staged.assign(2 * n_ctx, 0);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->items), items.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->clock), 2 * n_ctx * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->every), n_ctx * sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpy(b->items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->every, every.data(), every.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        g_batch_create_error = std::string("crbm_batch_create: ") + cudaGetErrorString(e);
        batch_free(b);
        return CRBM_ECUDA;
    }
    *out = b;
    return CRBM_OK;
}

int crbm_batch_sweep(crbm_batch* b, int64_t n_sweeps) {
    if (!b) return CRBM_EINVAL;
    if (n_sweeps < 0 || n_sweeps > (1 << 20)) {
        b->err = "n_sweeps must be in 0..2^20 per batched launch";
        return CRBM_EINVAL;
    }
    if (n_sweeps == 0) return CRBM_OK;
    const int n = static_cast<int>(b->ctx.size());
    for (auto* x : b->ctx)
        if (x->sweeps + n_sweeps > 4294967295LL) {
            b->err = "the 32-bit sweep counter of a member would overflow";
            return CRBM_EINVAL;
        }
    // upload the members' counters when they moved outside this batch
    bool stale = false;
    for (int c = 0; c < n; ++c)
        if (b->mirror[2 * c] != b->ctx[c]->sweeps || b->mirror[2 * c + 1] != b->ctx[c]->meas) stale = true;
    cudaError_t e = cudaSuccess;
    if (stale) {
        for (int c = 0; c < n; ++c) {
            b->staged[2 * c] = b->ctx[c]->sweeps;
            b->staged[2 * c + 1] = b->ctx[c]->meas;
        }
        // pageable source: staged by the time the call returns
        e = cudaMemcpyAsync(b->clock, b->staged.data(), 2 * n * sizeof(int64_t), cudaMemcpyHostToDevice, b->stream);
        b->mirror = b->staged;
    }
    // re-capture for another sweep count, or when a member's first-hit records
    // appeared (crbm_set_targets allocates them) after the graph was captured
    bool recapture = !b->exec || b->graph_n != n_sweeps;
    for (int c = 0; c < n; ++c)
        if (b->hit_seen[c] != b->ctx[c]->d.hit) recapture = true;
    if (e == cudaSuccess && recapture) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        BatchArgs args{};
        args.items = b->items;
        args.n_desc = n;
        args.smem_rec = b->smem_rec;
        for (int c = 0; c < n; ++c) {
            args.d[c] = fill_sweep_args(b->ctx[c], static_cast<int>(n_sweeps));
            args.d[c].clock = b->clock + 2 * c;
            args.d[c].n_bands = b->bands[c];
            b->hit_seen[c] = b->ctx[c]->d.hit;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 =
                launch_sweep_batch(args, b->n_items, b->cluster, b->threads, b->smem, b->modes, b->capture);
            cudaError_t e2 = launch_batch_advance(b->clock, b->every, n, n_sweeps, b->capture);
            e = cudaStreamEndCapture(b->capture, &graph);
            if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        b->graph_n = n_sweeps;
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) {
        b->err = std::string("crbm_batch_sweep: ") + cudaGetErrorString(e);
        return CRBM_ECUDA;
    }
    for (int c = 0; c < n; ++c) {  // host mirrors of the device clocks
        crbm_ctx* x = b->ctx[c];
        const int64_t t0 = x->sweeps, t1 = t0 + n_sweeps;
        if (x->measure_every > 0) x->meas += t1 / x->measure_every - t0 / x->measure_every;
        if (x->sq_every > 0) x->sq_meas += t1 / x->sq_every - t0 / x->sq_every;
        x->sweeps = t1;
        x->launches += 1;
        b->mirror[2 * c] = x->sweeps;
        b->mirror[2 * c + 1] = x->meas;
    }
    return CRBM_OK;
}

int crbm_batch_threads(const crbm_batch* b) { return b ? b->threads : CRBM_EINVAL; }

int crbm_batch_autotune(crbm_batch* b, int64_t probe_sweeps, int32_t* best_threads) {
    if (!b) return CRBM_EINVAL;
    if (probe_sweeps < 1 || probe_sweeps > 100000) {
        b->err = "probe_sweeps must be in 1..100000";
        return CRBM_EINVAL;
    }
    const int n = static_cast<int>(b->ctx.size());
    for (auto* x : b->ctx)
        if (x->sweeps + 3 * probe_sweeps > 4294967295LL) {
            b->err = "the 32-bit sweep counter of a member would overflow during the probes";
            return CRBM_EINVAL;
        }
    // Every member's state as a checkpoint (spins, sums, series, correlations,
    // replica permutation, counters) plus its first-hit records and launch
    // count, put back after each probe.
    std::vector<std::vector<char>> ck(n);
    std::vector<std::vector<int64_t>> hits(n);
    std::vector<int64_t> launches(n);
    for (int c = 0; c < n; ++c) {
        crbm_ctx* x = b->ctx[c];
        size_t sz = 0;
        int rc = crbm_save(x, nullptr, &sz);
        ck[c].resize(sz);
        if (rc == CRBM_OK) rc = crbm_save(x, ck[c].data(), &sz);
        if (rc == CRBM_OK && x->d.hit) {
            hits[c].resize(2 * static_cast<size_t>(x->n_words) * 32);
            if (cudaMemcpy(hits[c].data(), x->d.hit, hits[c].size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = CRBM_ECUDA;
        }
        if (rc != CRBM_OK) {
            b->err = "crbm_batch_autotune: checkpointing a member failed";
            return rc;
        }
        launches[c] = x->launches;
    }
    auto restore = [&]() {
        for (int c = 0; c < n; ++c) {
            crbm_ctx* x = b->ctx[c];
            int rc = crbm_load(x, ck[c].data(), ck[c].size());
            if (rc == CRBM_OK && x->d.hit &&
                cudaMemcpy(x->d.hit, hits[c].data(), hits[c].size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
                rc = CRBM_ECUDA;
            if (rc != CRBM_OK) return rc;
            x->launches = launches[c];
        }
        return static_cast<int>(CRBM_OK);
    };
    auto drop_graph = [&]() {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        b->graph_n = -1;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int threads0 = b->threads;
    int best = threads0, rc = CRBM_OK;
    float best_ms = 1e30f;
    // (measured on the mixed-size tempering batch with clusters of 8: 16 warps 6.8 % faster than 32)
    const int cand[] = {8, 12, 16, 20, 24, 28, 32};
    for (int w : cand) {
        if (e != cudaSuccess || rc != CRBM_OK) break;
        if (w > kMaxSweepWarps) continue;
        if (b->cluster > 1 && batch_max_active_clusters(b->cluster, 32 * w, b->smem, b->modes) < 1) continue;
        b->threads = 32 * w;
        drop_graph();
        rc = crbm_batch_sweep(b, std::max<int64_t>(1, probe_sweeps / 4));  // warm-up (and the graph)
        drop_graph();
        if (rc == CRBM_OK) rc = crbm_batch_sweep(b, probe_sweeps);       // instantiates the graph
        if (rc == CRBM_OK) e = cudaEventRecord(e0, b->stream);
        if (rc == CRBM_OK && e == cudaSuccess) rc = crbm_batch_sweep(b, probe_sweeps);
        if (rc == CRBM_OK && e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (rc == CRBM_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (rc == CRBM_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rc == CRBM_OK && e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = 32 * w;
        }
        if (rc == CRBM_OK && e == cudaSuccess) rc = restore();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->threads = (rc == CRBM_OK && e == cudaSuccess) ? best : threads0;
    drop_graph();
    if (rc != CRBM_OK || e != cudaSuccess) {
        const int rr = restore();  // best effort: the members as they were
        b->err = std::string("crbm_batch_autotune: ") +
                 (e != cudaSuccess ? cudaGetErrorString(e) : "a probe sweep failed") +
                 (rr != CRBM_OK ? " (restoring the members failed too)" : "");
        return e != cudaSuccess ? CRBM_ECUDA : rc;
    }
    if (best_threads) *best_threads = best;
    return CRBM_OK;
}

int crbm_batch_cluster(const crbm_batch* b) { return b ? b->cluster : CRBM_EINVAL; }

const char* crbm_batch_last_error(const crbm_batch* b) {
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

void crbm_batch_destroy(crbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

}  // extern "C"
