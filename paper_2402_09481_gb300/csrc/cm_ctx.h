// The context object behind the opaque cm_ctx handle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cm.h"
#include "cm_internal.h"
#include "ntt_device.cuh"

struct cm_server;  // continuous-batching request loop (cm_server.cu)

struct cm_ctx {
    int device = 0;
    int nsm = 0;
    uint64_t budget = 0;         // scratch bytes one call may take
    cm::PlanOptions popt;        // planner options of the single calls
    cm::Tuning tune{};           // cm_calibrate's figures (popt.tune points here once taken)
    cudaMemPool_t pool = nullptr;
    uint64_t *d_tables = nullptr;
    uint32_t *d_status = nullptr;
    cm::RootTables rt{};
    uint32_t *d_tables30 = nullptr;
    cm::RootTables30 rt30{};
    uint32_t *d_tables25 = nullptr;
    cm::RootTables25 rt25{};
    cm_server *server = nullptr;
    // one-launch cluster kernel per length 2^14 .. 2^17: -1 not yet checked, 0 no, 1 yes
    std::atomic<int> cluster25[4] = {-1, -1, -1, -1};

    // per-kernel tracing (cm_profile_*): events around each launch when on
    struct ProfRec {
        const char *name;
        cudaEvent_t a, b;
    };
    bool prof_on = false;
    std::mutex prof_mu;
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    std::map<std::string, std::pair<uint64_t, double>> prof_acc;
};

namespace cm {
// Brackets one kernel launch with profiling events when tracing is on.
struct ProfScope {
    cm_ctx *c;
    const char *name;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(cm_ctx *c_, const char *name_, cudaStream_t st_);
    ~ProfScope();
};
}  // namespace cm

// Frees what optional subsystems attached to the context (server, caches).
void cm_ctx_release_extras(cm_ctx *c);
