// The context object behind the opaque cm_ctx handle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm.h"
#include "ntt_device.cuh"

struct cm_server;  // continuous-batching request loop (cm_server.cu)

struct cm_ctx {
    int device = 0;
    int nsm = 0;
    uint64_t budget = 0;         // scratch bytes one call may take
    cudaMemPool_t pool = nullptr;
    uint64_t *d_tables = nullptr;
    uint32_t *d_status = nullptr;
    cm::RootTables rt{};
    cm_server *server = nullptr;
};

// Frees what optional subsystems attached to the context (server, caches).
void cm_ctx_release_extras(cm_ctx *c);
