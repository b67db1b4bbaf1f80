// vs_api_internal.h -- host-side state behind the opaque handles of vs.h.
#pragma once

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/vs.h"
#include "vs_internal.h"

namespace vs {
struct Serve;
}

struct vs_ctx {
    vs_options opt;
    std::chrono::steady_clock::time_point t0;
    vs::Serve *serve = nullptr;      // owned; released by serve_shutdown
    std::mutex serve_init_mu;
};

struct vs_field {
    vs_ctx *ctx = nullptr;
    vs::Geo g{};
    int prec = VS_FP64;
    int nc = 18;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool loaded = false;
    void *U = nullptr;
    int8_t *ref = nullptr;
    int8_t *cur = nullptr;
    void *G = nullptr;              // random gauge transformation (18 reals per site)
    bool gauge_on = false;          // links are in the random gauge G
    double *partials = nullptr;
    double *d_result = nullptr;
    unsigned long long *d_counts = nullptr;
    unsigned long long *d_sweep = nullptr;  // kSweepSlots counters of vs_subsweep and served jobs
    int *defer_idx = nullptr;       // FP32: positions left by a class launch to k_redecide [kDeferCap]
    unsigned *defer_n = nullptr;    // [0] entries appended, [1] k_redecide blocks done
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    void *flowS = nullptr;          // Runge-Kutta exponent H_S, 9 reals per link
    size_t flowS_bytes = 0;
    unsigned long long *sweep_counts = nullptr;
    double *sweep_actions = nullptr;
    int sweep_cap = 0;
    int last_action_every = 0;
    long long sweeps_done = 0;      // sweeps since the last load (re-unitarisation phase)
    bool profiling = false;
    double prof_ms = 0;
    int64_t prof_launches = 0;
    std::vector<cudaEvent_t> events;
};

namespace vs {

// NVTX range for tools such as Nsight Systems (header-only NVTX v3: a no-op
// unless a tool is attached to the process).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

vs_status fail(vs_status st, const char *fmt, ...);
vs_status cuda_fail(cudaError_t e, const char *what);
void *dev_alloc(vs_ctx *c, size_t bytes);
void dev_free(vs_ctx *c, void *p);
uint64_t field_footprint(const int32_t dims[4], int32_t precision, int32_t storage);
bool valid_dims(const int32_t dims[4]);

// Enqueue n_sweeps on the field's stream.  want_stats: per-sweep counters and
// actions into the field's stats buffers.  fixed_counters (optional): every
// sweep adds its counts into this one block of kSweepSlots instead.
vs_status smooth_enqueue(vs_field *f, int32_t n_sweeps, double rho, double eps, double u0,
                         const vs_anneal *sched, int32_t vp, bool want_stats,
                         unsigned long long *fixed_counters = nullptr);

// Reset n blocks of kSweepSlots counters (stride kSweepSlots): counts to 0, the
// margin slot to kMarginInit.
cudaError_t init_sweep_counters(unsigned long long *c, int n, cudaStream_t st);

void serve_shutdown(vs_ctx *c);

}  // namespace vs
