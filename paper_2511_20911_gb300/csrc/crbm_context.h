// Definition of the opaque context of include/crbm.h, shared by the host
// runtime files (crbm_host.cpp, crbm_runtime.cpp).
#pragma once

#include <string>
#include <vector>

#include "../../include/crbm.h"
#include "crbm_internal.h"

struct crbm_ctx {
    crbm::Geometry g{};
    int n_chains = 0, n_words = 0, n_params = 0;
    int layout = CRBM_LAYOUT_SMEM;
    int warps = 8;
    uint64_t seed = 0;
    int measure_every = 0, series_len = 0, sq_every = 0, swap_every = 0;
    int64_t sweeps = 0;     // global sweep counter
    int64_t meas = 0;       // measurements since the last reset
    int64_t sq_meas = 0;    // correlation samples since the last reset
    int64_t launches = 0;
    int64_t passes = 0;     // block-proposal passes (Philox sweep slot of the moves)
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<int32_t> chain_param;
    std::vector<int32_t> q[3];     // quantised J, J', h per point
    std::vector<int32_t> q_odd;    // quantised odd-column field per point (h when none is given)
    std::vector<double> beta;
    std::vector<uint32_t> tables;  // [n_params][nTab]
    crbm::DeviceState d;
    std::string err;
};

namespace crbm {
// Kernel arguments of one sweep launch of ctx (n sweeps from its counters).
SweepArgs fill_sweep_args(const crbm_ctx* ctx, int n_sweeps);
// Autotuner cache: the CTA warp count stored for ctx's shape, or 0.
int autotune_lookup(const crbm_ctx* ctx);
}  // namespace crbm
