// Batched extraction: one persistent kernel walking a work list.
//
// Every instance of a batch is planned like a single call (middle-product form,
// transform length L = 2^lg).  Instances with L <= 2^13 are one work item (the
// whole extraction on one CTA).  Instances with 2^13 < L <= 2^25 are split into
// phases: forward column-pass tiles of both operands (phase 0, bits unpacked on
// the fly), fused middle rows (phase 1), inverse column-pass tiles with parity
// (phase 2) and pack chunks (phase 3).  Dodis et al. instances add a
// precondition item to phase 0.  The list is ordered phase by phase, so an item
// only ever waits for items that were dequeued before it by CTAs that are
// running (the grid is sized to be fully resident); each wait is bounded and
// gives up with CM_FLAG_TIMEOUT.  Instances with L > 2^25 (two column passes)
// run through the per-call kernels after the work-list kernel.
//
// A batch is planned once (cm_batch_create: scratch, work list, optional
// autotuning of the pass tile, CUDA-graph capture) and replayed with
// cm_batch_launch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "cm.h"
#include "cm_ctx.h"
#include "cm_internal.h"
#include "cm_batch_internal.h"
#include "ntt_generic.cuh"

namespace cm {

cm_status enqueue_extract(cm_ctx *ctx, const Plan &p, const uint64_t *x, const uint64_t *y,
                          uint64_t *z, void *scratch, cudaStream_t st);

namespace {

constexpr uint64_t kSpinLimit = 1ull << 22;  // polls of 64 ns-ish each before giving up

// ctrl layout (uint32): [0] next item, [1] abort, [2..] done[inst * 4 + phase]
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <class F>
__device__ void do_small(const BatchInst &I, const typename F::T *tw, typename F::T *sA, typename F::T *sB,
                         uint32_t *status) {
    using T = typename F::T;
    const int lg = I.lg, L = 1 << lg;
    int any1 = 0, any0 = 0;
    for (int i = threadIdx.x; i < L; i += kThreads) {
        sA[sp(i)] = (T)I.amap.get(i);
        sB[sp(i)] = (T)I.bmap.get(i);
    }
    if (I.kind == CM_DODIS) {
        for (uint64_t i = threadIdx.x; i < I.nx; i += kThreads) {
            const uint64_t b = (__ldg(I.amap.src + (i >> 6)) >> (i & 63)) & 1ull;
            any1 |= (int)b;
            any0 |= (int)(b ^ 1);
        }
    }
    any1 = __syncthreads_or(any1);
    any0 = __syncthreads_or(any0);
    const bool bad = I.kind == CM_DODIS && !(any1 && any0);
    if (bad && threadIdx.x == 0) atomicOr(status, kFlagPrecond);
    if (I.pre && threadIdx.x == 0) {
        I.pre[0] = any1 ? 1u : 0u;
        I.pre[1] = any0 ? 1u : 0u;
    }
    ntt_fwd_rt<F>(sA, sB, 2, lg, 0, tw);
    const T linv = (T)I.linv;
    for (int i = threadIdx.x; i < L; i += kThreads) sA[sp(i)] = F::prod(sA[sp(i)], sB[sp(i)], linv);
    __syncthreads();
    ntt_inv_rt<F>(sA, sA, 1, lg, 0, tw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nwords = (I.m + 63) >> 6;
    for (uint64_t w = warp; w < nwords; w += kThreads / 32) {
        const uint64_t p0 = (w << 6) + lane, p1 = p0 + 32;
        const uint32_t b0 = (p0 < I.m) ? (uint32_t)(F::canon(sA[sp((int)(I.lo + p0))]) & 1u) : 0u;
        const uint32_t b1 = (p1 < I.m) ? (uint32_t)(F::canon(sA[sp((int)(I.lo + p1))]) & 1u) : 0u;
        const uint32_t w0 = __ballot_sync(0xffffffffu, b0);
        const uint32_t w1 = __ballot_sync(0xffffffffu, b1);
        if (lane == 0) I.z[w] = bad ? 0ull : ((uint64_t)w1 << 32 | w0);
    }
}

// Column-pass tile (the single pass of a 2^14 .. 2^25 transform: N = L).
template <class F, bool INV>
__device__ void do_pass(const BatchInst &I, int operand, uint32_t tile, const typename F::T *tw,
                        typename F::T *s, const RootTablesT<typename F::T> &rt) {
    using T = typename F::T;
    const int logr = I.logr, lg = I.lg, ncol_lg = I.tile_lg - logr;
    const int lgS = lg - logr, cmask = (1 << ncol_lg) - 1, n = 1 << I.tile_lg;
    const uint64_t col0 = (uint64_t)tile << ncol_lg;
    const int esh = F::kAdicity - lg;
    T *data = static_cast<T *>(operand ? I.B : I.A);
    const BitMap &map = operand ? I.bmap : I.amap;
    for (int e = threadIdx.x; e < n; e += kThreads) {
        const int i = e >> ncol_lg, c = e & cmask;
        const uint64_t g = col0 + ((uint64_t)i << lgS) + c;
        T v;
        if (INV) {
            v = F::red(__ldcg(data + g));  // lazy fields: below 2q before a product by a root below 2q
            const uint64_t k = pos_to_freq_rt(i, logr);
            const uint32_t E = (uint32_t)(((col0 + c) * k) << esh);
            if (E) v = F::twmul(v, big_root_f<F>(rt.big_lo_inv, rt.big_hi_inv, E));
        } else {
            v = (T)map.get(g);
        }
        s[sp(e)] = v;
    }
    __syncthreads();
    if (INV)
        ntt_inv_rt<F>(s, s, 1, logr, ncol_lg, tw);
    else
        ntt_fwd_rt<F>(s, s, 1, logr, ncol_lg, tw);
    for (int e = threadIdx.x; e < n; e += kThreads) {
        const int i = e >> ncol_lg, c = e & cmask;
        T v = s[sp(e)];
        const uint64_t g = col0 + ((uint64_t)i << lgS) + c;
        if (INV) {
            const uint64_t p = g - I.lo;
            if (g >= I.lo && p < I.m) I.par[p] = (uint8_t)(F::canon(v) & 1u);
        } else {
            const uint64_t k = pos_to_freq_rt(i, logr);
            const uint32_t E = (uint32_t)(((col0 + c) * k) << esh);
            if (E) v = F::twmul(v, big_root_f<F>(rt.big_lo_fwd, rt.big_hi_fwd, E));
            data[g] = v;
        }
    }
}

template <class F>
__device__ void do_middle(const BatchInst &I, uint32_t r, const typename F::T *tw, typename F::T *sA,
                          typename F::T *sB) {
    using T = typename F::T;
    constexpr int LG = kMidLgMax, Bn = 1 << LG;
    constexpr int PER = 16 / sizeof(T);
    const uint64_t row = (uint64_t)r << LG;
    const uint4 *a4 = reinterpret_cast<const uint4 *>(static_cast<const T *>(I.A) + row);
    const uint4 *b4 = reinterpret_cast<const uint4 *>(static_cast<const T *>(I.B) + row);
    for (int i = threadIdx.x; i < Bn / PER; i += kThreads) {
        T pa[PER], pb[PER];
        unpack16(__ldcg(a4 + i), pa);
        unpack16(__ldcg(b4 + i), pb);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            sA[sp(PER * i + j)] = pa[j];
            sB[sp(PER * i + j)] = pb[j];
        }
    }
    __syncthreads();
    middle_row_13_f<F>(sA, sB, tw, (T)I.linv);
    uint4 *o4 = reinterpret_cast<uint4 *>(static_cast<T *>(I.A) + row);
    for (int i = threadIdx.x; i < Bn / PER; i += kThreads) {
        T pv[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) pv[j] = sA[sp(PER * i + j)];
        o4[i] = pack16(pv);
    }
}

__device__ void do_pack(const BatchInst &I, uint32_t chunk, uint32_t *status) {
    const bool bad = I.pre && (__ldcg(I.pre) == 0u || __ldcg(I.pre + 1) == 0u);
    if (bad && chunk == 0 && threadIdx.x == 0) atomicOr(status, kFlagPrecond);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nwords = (I.m + 63) >> 6;
    const uint64_t w0 = (uint64_t)chunk * kPackWordsPerItem;
    const uint64_t w1 = min(nwords, w0 + kPackWordsPerItem);
    for (uint64_t w = w0 + warp; w < w1; w += kThreads / 32) {
        const uint64_t p0 = (w << 6) + lane, p1 = p0 + 32;
        const uint32_t b0 = (p0 < I.m) ? __ldcg(I.par + p0) : 0u;
        const uint32_t b1 = (p1 < I.m) ? __ldcg(I.par + p1) : 0u;
        const uint32_t x0 = __ballot_sync(0xffffffffu, b0);
        const uint32_t x1 = __ballot_sync(0xffffffffu, b1);
        if (lane == 0) I.z[w] = bad ? 0ull : ((uint64_t)x1 << 32 | x0);
    }
}

__device__ void do_check(const BatchInst &I) {
    int any1 = 0, any0 = 0;
    const uint64_t nw = (I.nx + 63) >> 6;
    for (uint64_t w = threadIdx.x; w < nw; w += kThreads) {
        uint64_t mask = ~0ull;
        if (w == nw - 1 && (I.nx & 63)) mask = (1ull << (I.nx & 63)) - 1;
        const uint64_t v = __ldg(I.amap.src + w);
        any1 |= (v & mask) != 0;
        any0 |= (~v & mask) != 0;
    }
    any1 = __syncthreads_or(any1);
    any0 = __syncthreads_or(any0);
    if (threadIdx.x == 0) {
        I.pre[0] = any1 ? 1u : 0u;
        I.pre[1] = any0 ? 1u : 0u;
    }
}

template <class F>
__global__ void __launch_bounds__(kThreads, sizeof(typename F::T) == 4 ? 2 : 1)
k_batch(const BatchInst *__restrict__ insts, const WorkItem *__restrict__ items, uint32_t nitems,
        uint32_t *ctrl, uint32_t *status, RootTablesT<typename F::T> rt) {
    using T = typename F::T;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    T *tw = reinterpret_cast<T *>(smem_raw);  // omega_8192^e
    T *sA = tw + 8192;                        // also the pass tile (2^14 elements)
    T *sB = sA + sp_size(1 << kMidLgMax);
    __shared__ uint32_t s_item, s_skip;
    for (int e = threadIdx.x; e < 8192; e += kThreads) tw[tw_swz(e)] = __ldg(rt.small + e);
    uint32_t *next = ctrl, *abort_flag = ctrl + 1, *done = ctrl + 2;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = (ld_acquire(abort_flag) != 0u) ? nitems : atomicAdd(next, 1u);
            s_skip = 0;
        }
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= nitems) break;
        const WorkItem w = items[it];
        const BatchInst &I = insts[w.inst];
        if (threadIdx.x == 0 && w.phase > 0 && w.type != kItSmall) {
            const uint32_t need = I.need[w.phase - 1];
            const uint32_t *cnt = done + 4 * w.inst + (w.phase - 1);
            uint64_t spins = 0;
            while (ld_acquire(cnt) < need) {
                if (++spins > kSpinLimit || ld_acquire(abort_flag)) {
                    atomicOr(status, kFlagTimeout);
                    atomicExch(abort_flag, 1u);
                    s_skip = 1;
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
        }
        __syncthreads();
        if (!s_skip) {
            switch (w.type) {
                case kItSmall: do_small<F>(I, tw, sA, sB, status); break;
                case kItFwdA: do_pass<F, false>(I, 0, w.idx, tw, sA, rt); break;
                case kItFwdB: do_pass<F, false>(I, 1, w.idx, tw, sA, rt); break;
                case kItMiddle: do_middle<F>(I, w.idx, tw, sA, sB); break;
                case kItInv: do_pass<F, true>(I, 0, w.idx, tw, sA, rt); break;
                case kItPack: do_pack(I, w.idx, status); break;
                case kItCheck: do_check(I); break;
                default: break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + 4 * w.inst + w.phase, 1u);
        }
    }
}

}  // namespace

static size_t round256(size_t v) { return (v + 255) & ~size_t(255); }
// The work list runs every instance (L <= 2^25) over the lazily reduced field
// of 5 * 2^25 + 1 (exact: every count is at most K <= L <= 2^25 < q).
using BatchField = FieldF25;
using BatchT = BatchField::T;
static const size_t kBatchSmem = (8192 + 2 * (size_t)sp_size(1 << kMidLgMax)) * sizeof(BatchT);

size_t worklist_scratch_bytes(const Plan &p) {
    return p.npass == 1 ? round256(2 * sizeof(BatchT) * p.L) + round256(p.m) : 0;
}

size_t worklist_seed_bytes(const Plan &p) { return sizeof(BatchT) * p.L; }

size_t batch_smem_bytes() { return kBatchSmem; }

int batch_grid(int nsm) {
    auto kern = k_batch<BatchField>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) != cudaSuccess)
        return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, kBatchSmem) != cudaSuccess)
        return 0;
    return nsm * occ;
}

cudaError_t launch_k_batch(const BatchInst *insts, const WorkItem *items, uint32_t nitems, uint32_t *ctrl,
                           uint32_t *status, const RootTables25 &rt, int grid, cudaStream_t st) {
    k_batch<BatchField><<<grid, kThreads, kBatchSmem, st>>>(insts, items, nitems, ctrl, status, rt);
    return cudaGetLastError();
}

void build_worklist(const cm_desc *descs, const Plan *plans, const uint32_t *idx, uint32_t n,
                    uint8_t *scratch, const size_t *off, int tile_lg, uint32_t *pre,
                    std::vector<BatchInst> &insts, std::vector<WorkItem> &items, void *const *bext,
                    const uint8_t *bready, bool test_stall) {
    bool stalled = false;
    insts.assign(n, BatchInst());
    std::vector<WorkItem> phase[4];
    std::vector<WorkItem> smalls;
    std::vector<uint32_t> order(n);
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t c) { return plans[idx[a]].L > plans[idx[c]].L; });
    for (uint32_t oi = 0; oi < n; ++oi) {
        const uint32_t k = order[oi];
        const uint32_t di = idx[k];
        const Plan &p = plans[di];
        const cm_desc &d = descs[di];
        BatchInst &I = insts[k];
        memset(&I, 0, sizeof(I));
        I.amap.src = d.x; I.amap.mode = p.amode; I.amap.len = p.alen; I.amap.srclen = p.asrclen; I.amap.off = p.aoff;
        I.bmap.src = d.y; I.bmap.mode = p.bmode; I.bmap.len = p.blen; I.bmap.srclen = p.bsrclen; I.bmap.off = p.boff;
        I.z = d.z;
        I.lo = p.lo;
        I.m = p.m;
        I.linv = f25_linv_mont2(p.L);
        I.nx = p.n;
        I.lg = p.lg;
        I.kind = p.kind;
        if (p.kind == CM_DODIS && pre) I.pre = pre + 2 * k;
        if (p.npass == 0) {
            smalls.push_back({k, kItSmall, 0, 0, 0});
            continue;
        }
        I.logr = p.pass_lg[0];
        I.tile_lg = std::max(tile_lg, I.logr);  // at least one column per tile
        uint8_t *base = scratch + off[di];
        I.A = base;
        I.B = base + sizeof(BatchT) * p.L;
        I.par = base + 2 * sizeof(BatchT) * p.L;
        const bool have_b = bext && bext[k] && bready && bready[k];
        if (bext && bext[k]) I.B = bext[k];
        const uint32_t tiles = (uint32_t)(p.L >> I.tile_lg);
        const uint32_t rows = (uint32_t)(p.L >> kMidLgMax);
        const uint32_t packs = (uint32_t)((((p.m + 63) >> 6) + kPackWordsPerItem - 1) / kPackWordsPerItem);
        I.need[0] = (have_b ? 1 : 2) * tiles + (I.pre ? 1 : 0);
        if (test_stall && !stalled) {
            I.need[0] += 1;  // a count nothing will ever reach
            stalled = true;
        }
        I.need[1] = rows;
        I.need[2] = tiles;
        I.need[3] = packs;
        if (I.pre) phase[0].push_back({k, kItCheck, 0, 0, 0});
        for (uint32_t t = 0; t < tiles; ++t) {
            phase[0].push_back({k, kItFwdA, 0, t, 0});
            if (!have_b) phase[0].push_back({k, kItFwdB, 0, t, 0});
        }
        for (uint32_t r = 0; r < rows; ++r) phase[1].push_back({k, kItMiddle, 1, r, 0});
        for (uint32_t t = 0; t < tiles; ++t) phase[2].push_back({k, kItInv, 2, t, 0});
        for (uint32_t c = 0; c < packs; ++c) phase[3].push_back({k, kItPack, 3, c, 0});
    }
    items.clear();
    items.reserve(phase[0].size() + smalls.size() + phase[1].size() + phase[2].size() + phase[3].size());
    std::stable_sort(smalls.begin(), smalls.end(),
                     [&](const WorkItem &a, const WorkItem &c) { return insts[a.inst].lg > insts[c.inst].lg; });
    for (auto &w : phase[0]) items.push_back(w);
    for (auto &w : smalls) items.push_back(w);
    for (int ph = 1; ph < 4; ++ph)
        for (auto &w : phase[ph]) items.push_back(w);
}

}  // namespace cm

using namespace cm;

struct cm_batch {
    cm_ctx *ctx = nullptr;
    std::vector<cm_desc> descs;
    std::vector<Plan> plans;
    std::vector<uint32_t> wl;       // instances on the work list
    std::vector<uint32_t> solo;     // instances with L > 2^21 (single-call kernels)
    std::vector<size_t> off_scratch;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    uint32_t *d_pre = nullptr;      // Dodis et al. precondition flags, 2 per instance
    BatchInst *d_insts = nullptr;
    WorkItem *d_items = nullptr;
    uint32_t nitems = 0;
    uint32_t *d_ctrl = nullptr;
    size_t ctrl_words = 0;
    int tile_lg = kTileLg;
    int grid = 0;
    uint64_t kernel_launches = 0;
    bool test_stall = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// Build instance descriptors and the work list for the current tile size.
static cm_status batch_build(cm_batch *b) {
    const uint32_t n = (uint32_t)b->wl.size();
    std::vector<BatchInst> insts;
    std::vector<WorkItem> items;
    build_worklist(b->descs.data(), b->plans.data(), b->wl.data(), n, static_cast<uint8_t *>(b->scratch),
                   b->off_scratch.data(), b->tile_lg, b->d_pre, insts, items, nullptr, nullptr, b->test_stall);
    if (b->d_insts) cudaFree(b->d_insts);
    if (b->d_items) cudaFree(b->d_items);
    b->d_insts = nullptr;
    b->d_items = nullptr;
    b->nitems = (uint32_t)items.size();
    if (n && cudaMalloc(&b->d_insts, n * sizeof(BatchInst)) != cudaSuccess) return CM_ENOMEM;
    if (!items.empty() && cudaMalloc(&b->d_items, items.size() * sizeof(WorkItem)) != cudaSuccess)
        return CM_ENOMEM;
    if (n && cudaMemcpy(b->d_insts, insts.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice) != cudaSuccess)
        return CM_EDEVICE;
    if (!items.empty() &&
        cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) != cudaSuccess)
        return CM_EDEVICE;
    b->ctrl_words = 2 + 4 * (size_t)n;
    if (!b->d_ctrl && cudaMalloc(&b->d_ctrl, b->ctrl_words * sizeof(uint32_t)) != cudaSuccess) return CM_ENOMEM;
    return CM_OK;
}

// Enqueue one execution of the batch on st.
static cm_status batch_enqueue(cm_batch *b, cudaStream_t st) {
    cm_ctx *ctx = b->ctx;
    b->kernel_launches = 0;
    if (b->nitems) {
        if (cudaMemsetAsync(b->d_ctrl, 0, b->ctrl_words * sizeof(uint32_t), st) != cudaSuccess) return CM_EDEVICE;
        ProfScope ps(ctx, "k_batch", st);
        k_batch<BatchField><<<b->grid, kThreads, kBatchSmem, st>>>(b->d_insts, b->d_items, b->nitems, b->d_ctrl,
                                                         ctx->d_status, ctx->rt25);
        if (cudaGetLastError() != cudaSuccess) return CM_EDEVICE;
        b->kernel_launches += 1;
    }
    uint8_t *sc = static_cast<uint8_t *>(b->scratch);
    for (uint32_t di : b->solo) {
        const cm_desc &d = b->descs[di];
        cm_status s = enqueue_extract(ctx, b->plans[di], d.x, d.y, d.z, sc + b->off_scratch[di], st);
        if (s != CM_OK) return s;
        b->kernel_launches += b->plans[di].launches;
    }
    return CM_OK;
}

static void batch_free(cm_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_insts) cudaFree(b->d_insts);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_ctrl) cudaFree(b->d_ctrl);
    if (b->scratch) cudaFree(b->scratch);
    delete b;
}

static double time_once(cm_batch *b, cudaStream_t st) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    batch_enqueue(b, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

extern "C" cm_status cm_batch_create(cm_ctx *ctx, const cm_desc *descs, uint32_t count, uint32_t flags,
                                     cm_batch **out) {
    if (!ctx || !out || (count && !descs)) return CM_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    cm_batch *b = new cm_batch();
    b->ctx = ctx;
    b->test_stall = (flags & CM_BATCH_TEST_STALL) != 0;
    if (b->test_stall) flags = (flags & ~CM_BATCH_AUTOTUNE) | CM_BATCH_NO_GRAPH;
    b->descs.assign(descs, descs + count);
    b->plans.resize(count);
    b->off_scratch.assign(count, 0);
    size_t total = 0;
    for (uint32_t i = 0; i < count; ++i) {
        const cm_desc &d = descs[i];
        if (!d.x || !d.y || !d.z || !make_plan(d.kind, d.n, d.m, &b->plans[i], worklist_fields(ctx->popt))) {
            delete b;
            return CM_EINVAL;
        }
        b->off_scratch[i] = total;
        if (on_worklist(b->plans[i])) {
            b->wl.push_back(i);
            total += worklist_scratch_bytes(b->plans[i]);
        } else {
            // the single-call kernels, over the context's field set
            make_plan(d.kind, d.n, d.m, &b->plans[i], ctx->popt.fields, ctx->popt.tune);
            b->solo.push_back(i);
            total += round256(b->plans[i].scratch_bytes);
        }
    }
    if (total > ctx->budget) {
        delete b;
        return CM_ENOMEM;
    }
    const size_t pre_off = total;  // precondition flags, 2 words per work-list instance
    total += round256(8 * b->wl.size() + 8);
    b->scratch_bytes = total;
    if (total && cudaMalloc(&b->scratch, total) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return CM_ENOMEM;
    }
    b->d_pre = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(b->scratch) + pre_off);
    b->grid = batch_grid(ctx->nsm);  // every CTA resident
    if (b->grid < 1) {
        batch_free(b);
        return CM_EDEVICE;
    }
    cm_status s = batch_build(b);
    if (s != CM_OK) {
        batch_free(b);
        return s;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        batch_free(b);
        return CM_EDEVICE;
    }
    if ((flags & CM_BATCH_AUTOTUNE) && !b->wl.empty()) {
        // autotuner: pass tile of 2^13 or 2^14 elements (columns per tile vs
        // tiles in flight), timed on this batch; keep the faster
        double best = 1e30;
        int best_tile = kTileLg;
        for (int tl : {kTileLg, kTileLg - 1}) {
            b->tile_lg = tl;
            if ((s = batch_build(b)) != CM_OK) break;
            time_once(b, st);  // warm-up
            const double ms = time_once(b, st);
            if (ms < best) {
                best = ms;
                best_tile = tl;
            }
        }
        b->tile_lg = best_tile;
        if (s == CM_OK) s = batch_build(b);
    }
    if (s == CM_OK && !(flags & CM_BATCH_NO_GRAPH)) {
        cudaStreamSynchronize(st);
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            s = CM_EDEVICE;
        } else {
            const bool prof = ctx->prof_on;
            ctx->prof_on = false;  // no tracing events inside the graph
            cm_status es = batch_enqueue(b, st);
            ctx->prof_on = prof;
            cudaError_t ce = cudaStreamEndCapture(st, &b->graph);
            if (es != CM_OK || ce != cudaSuccess ||
                cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
                s = CM_EDEVICE;
        }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (s != CM_OK) {
        batch_free(b);
        return s;
    }
    *out = b;
    return CM_OK;
}

extern "C" cm_status cm_batch_launch(cm_batch *b, cm_stream stream) {
    if (!b) return CM_EINVAL;
    if (cudaSetDevice(b->ctx->device) != cudaSuccess) return CM_EDEVICE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b->exec && !b->ctx->prof_on) {
        if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return CM_EDEVICE;
        return CM_OK;
    }
    return batch_enqueue(b, st);
}

extern "C" void cm_batch_destroy(cm_batch *b) {
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    batch_free(b);
}

extern "C" cm_status cm_batch_info(const cm_batch *b, cm_batch_stats *st) {
    if (!b || !st) return CM_EINVAL;
    memset(st, 0, sizeof(*st));
    st->instances = (uint32_t)b->descs.size();
    st->work_items = b->nitems;
    st->solo_instances = (uint32_t)b->solo.size();
    st->tile_lg = (uint32_t)b->tile_lg;
    st->grid = (uint32_t)b->grid;
    st->scratch_bytes = b->scratch_bytes;
    st->kernel_launches = b->kernel_launches;
    st->graph = b->exec ? 1u : 0u;
    for (uint32_t i = 0; i < b->descs.size(); ++i) {
        st->output_bits += b->plans[i].m;
        st->transform_elements += b->plans[i].L;
    }
    return CM_OK;
}

extern "C" cm_status cm_batch_extract(cm_ctx *ctx, const cm_desc *descs, uint32_t count, cm_stream stream) {
    cm_batch *b = nullptr;
    cm_status s = cm_batch_create(ctx, descs, count, CM_BATCH_NO_GRAPH, &b);
    if (s != CM_OK) return s;
    s = batch_enqueue(b, static_cast<cudaStream_t>(stream));
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && s == CM_OK) s = CM_EDEVICE;
    cm_batch_destroy(b);
    return s;
}

extern "C" cm_status cm_batch_toeplitz(cm_ctx *ctx, const cm_desc *descs, uint32_t count, cm_stream stream) {
    for (uint32_t i = 0; i < count; ++i)
        if (!descs || descs[i].kind != CM_TOEPLITZ) return CM_EINVAL;
    return cm_batch_extract(ctx, descs, count, stream);
}
