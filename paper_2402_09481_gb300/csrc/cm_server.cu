// Continuous-batching request server (cm_submit / cm_poll).
//
// Clients submit single extractions of any kind and size; a worker thread
// keeps a FIFO of pending requests and a few "slots" (two per CUDA stream: a
// wave waits on the stream behind the running one, so that the stream never
// idles between waves).  Whenever
// a slot is free it admits, in queue order, the requests whose scratch fits in
// the HBM budget still unclaimed by requests on the device; a request that
// does not fit yet is passed over by at most a fixed number of waves, after
// which nothing behind it starts until it fits.  A wave runs as one work-list
// kernel on the slot's stream (requests with transforms longer than 2^21
// follow on the same stream through the single-call kernels).  Waves on
// different slots run concurrently, so requests that arrive while others are
// on the GPU start as soon as a slot and memory free up.  Admission holds the
// server lock; planning, upload and launch run outside it, so submissions
// and polls never wait for them.  Scratch comes from the context's
// stream-ordered pool and returns to it at the end of the wave.  Each
// request's result (its own status, including the Dodis et al.
// precondition, and submit / admit / completion times) is collected with
// cm_poll.  The root tables stay resident in the context.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cm.h"
#include "cm_batch_internal.h"
#include "cm_ctx.h"
#include "cm_internal.h"

namespace cm {
cm_status enqueue_blocks(cm_ctx *ctx, const std::vector<Block> &bl, const uint64_t *x, const uint64_t *y,
                         uint64_t *z, uint8_t *scratch, uint64_t tmp_off, uint64_t pre_off, cudaStream_t st);
}

using namespace cm;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t r256(size_t v) { return (v + 255) & ~size_t(255); }

struct Req {
    cm_desc d;
    Plan p;                     // one-transform plan (the work list takes L <= 2^21)
    std::vector<Block> blocks;  // longer requests: the single-call planner's products
    uint64_t tmp_off = 0, pre_off = 0;
    uint32_t flags = 0;
    uint64_t seed_id = 0;
    size_t foot = 0;  // scratch bytes while on the device
    uint32_t passed = 0;  // waves admitted past it while it did not fit
    uint64_t t_submit = 0, t_admit = 0, t_done = 0, wave = 0;
    int status = CM_OK;
    bool done = false;
};

// Grow-only device / pinned host buffer.
struct Buf {
    void *dev = nullptr, *host = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes) {
        if (bytes <= cap) return true;
        size_t c = cap ? cap : 4096;
        while (c < bytes) c *= 2;
        if (dev) cudaFree(dev);
        if (host) cudaFreeHost(host);
        dev = host = nullptr;
        cap = 0;
        if (cudaMalloc(&dev, c) != cudaSuccess || cudaMallocHost(&host, c) != cudaSuccess) return false;
        cap = c;
        return true;
    }
    void release() {
        if (dev) cudaFree(dev);
        if (host) cudaFreeHost(host);
        dev = host = nullptr;
        cap = 0;
    }
};

// Resident transform of a seed operand, keyed by (seed_id, kind, n, m).
struct SeedKey {
    uint64_t id, n, m;
    int kind;
    bool operator==(const SeedKey &o) const { return id == o.id && n == o.n && m == o.m && kind == o.kind; }
};
struct SeedKeyHash {
    size_t operator()(const SeedKey &k) const {
        return std::hash<uint64_t>()(k.id * 0x9E3779B97F4A7C15ull ^ k.n * 31 ^ k.m * 131 ^ (uint64_t)k.kind);
    }
};
struct SeedEntry {
    void *buf = nullptr;
    size_t bytes = 0;
    bool ready = false;  // holds the transform (its creating wave finished)
    int refs = 0;        // in-flight waves using it
    uint64_t last = 0;   // LRU clock
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    bool express = false;  // high-priority stream; takes work-list requests only
    bool borrowed = false;  // the stream belongs to another slot (the wave runs after that slot's)
    std::vector<uint64_t> tickets;
    std::vector<int> pre_index;  // per ticket: flag pair index, or -1
    size_t foot = 0;
    uint64_t wave = 0;
    Buf insts, items, ctrl, flags;  // flags: [0] status word, then 2 words per request
    std::vector<std::pair<SeedKey, bool>> seeds;  // cache entries used (true: created by this wave)
};

}  // namespace

struct cm_server {
    cm_ctx *ctx = nullptr;
    cm_server_options opt{};
    size_t budget = 0;
    int grid = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_ticket = 1, waves = 0;
    std::vector<Slot> slots;
    uint32_t express = 0;  // express slots (the last ones)
    size_t inflight = 0, max_inflight = 0;
    uint64_t submitted = 0, completed = 0, rejected = 0;
    bool stop = false;
    std::unordered_map<SeedKey, SeedEntry, SeedKeyHash> seeds;
    size_t seed_bytes = 0, seed_limit = 0;
    uint64_t seed_hits = 0, seed_misses = 0, lru = 0;
};

namespace {

// Drop the slot's references to seed transforms.  An entry this wave created
// becomes ready when the wave succeeded and holds a buffer; otherwise it is
// freed once no wave uses it.
void release_seeds(cm_server *S, Slot &sl, bool ok) {
    for (auto &kc : sl.seeds) {
        auto it = S->seeds.find(kc.first);
        if (it == S->seeds.end()) continue;
        SeedEntry &e = it->second;
        e.refs -= 1;
        if (!kc.second) continue;
        if (ok && e.buf) {
            e.ready = true;
        } else if (e.refs == 0) {
            if (e.buf) cudaFreeAsync(e.buf, sl.st);
            S->seed_bytes -= e.bytes;
            S->seeds.erase(it);
        }
    }
    sl.seeds.clear();
}

// Free the slot; its scratch claim returns to the budget.
void vacate_slot(cm_server *S, Slot &sl) {
    S->inflight -= sl.foot;
    sl.foot = 0;
    sl.tickets.clear();
    sl.pre_index.clear();
    sl.busy = false;
}

// Complete every request of the slot's wave with `status` (a launch that
// failed, or a device error reported by the wave's event).
void fail_wave(cm_server *S, Slot &sl, int status) {
    const uint64_t t = now_ns();
    for (uint64_t tk : sl.tickets) {
        auto it = S->reqs.find(tk);
        if (it == S->reqs.end()) continue;
        it->second.status = status;
        it->second.done = true;
        it->second.t_done = t;
        ++S->completed;
    }
    release_seeds(S, sl, false);
    vacate_slot(S, sl);
}

// Finish a completed wave: per-request status from the copied-back flags.
void finish_slot(cm_server *S, Slot &sl) {
    const uint32_t *f = static_cast<const uint32_t *>(sl.flags.host);
    const uint32_t st_word = f[0];
    const uint64_t t = now_ns();
    for (size_t i = 0; i < sl.tickets.size(); ++i) {
        auto it = S->reqs.find(sl.tickets[i]);
        if (it == S->reqs.end()) continue;
        Req &r = it->second;
        int status = CM_OK;
        if (st_word & CM_FLAG_TIMEOUT) status = CM_ETIMEDOUT;
        const int pi = sl.pre_index[i];
        if (pi >= 0 && (f[2 + 2 * pi] == 0u || f[3 + 2 * pi] == 0u)) status = CM_EPRECOND;
        r.status = status;
        r.t_done = t;
        r.done = true;
        ++S->completed;
    }
    release_seeds(S, sl, !(st_word & CM_FLAG_TIMEOUT));
    vacate_slot(S, sl);
}

// Drop the least recently used seed transform that no wave uses; false if
// there is none.
bool seed_evict_one(cm_server *S, cudaStream_t st) {
    auto victim = S->seeds.end();
    for (auto it = S->seeds.begin(); it != S->seeds.end(); ++it)
        if (it->second.refs == 0 && it->second.ready &&
            (victim == S->seeds.end() || it->second.last < victim->second.last))
            victim = it;
    if (victim == S->seeds.end()) return false;
    cudaFreeAsync(victim->second.buf, st);
    S->seed_bytes -= victim->second.bytes;
    S->seeds.erase(victim);
    return true;
}

// Make room for `bytes` of seed transforms within the cache limit.
bool seed_make_room(cm_server *S, size_t bytes, cudaStream_t st) {
    while (S->seed_bytes + bytes > S->seed_limit)
        if (!seed_evict_one(S, st)) return false;
    return true;
}

// What launching a wave needs, copied out of the request table under the lock
// (the table changes while clients submit and poll).
struct WaveReq {
    cm_desc d;
    Plan p;
    std::vector<Block> blocks;
    uint64_t tmp_off = 0, pre_off = 0;
    bool solo = false;  // runs the single-call kernels (blocks) even where the work list could take it
};
struct Wave {
    std::vector<WaveReq> r;
    std::vector<void *> bext;       // per request: its resident seed transform, else null
    std::vector<uint8_t> bready;    // it already holds the transform
    std::vector<SeedEntry *> make;  // per request: a new entry whose buffer the launch allocates
};

// Waves that may pass a queued request whose scratch does not fit; after
// that, nothing behind it is admitted until it fits.
constexpr uint32_t kMaxPassed = 16;

// Admit a wave for the free slot sl (under the lock).  The queue is taken in
// order; a request whose scratch does not fit in the budget left is passed
// over (at most kMaxPassed times), so small requests need not wait behind a
// large one.  With nothing in flight, unused seed transforms give way to a
// request that does not fit.  Marks the slot busy and copies what the launch
// needs into w; false if nothing was admitted.
bool admit_wave(cm_server *S, Slot &sl, Wave &w) {
    std::vector<uint64_t> wave, passed, other;
    std::vector<size_t> passed_at, other_at;
    size_t foot = 0;
    const size_t scan = std::max<size_t>(64, 4 * (size_t)S->opt.max_wave);
    // what the slot takes: an express slot work-list requests only; a slot
    // whose wave would wait behind another on its stream, while express slots
    // exist, the longer requests only (a short one waits for a stream of its
    // own or the express lane, not behind a long wave); any other slot all
    const bool longs_only = sl.borrowed && S->express > 0;
    for (size_t seen = 0; seen < scan && !S->pending.empty() && wave.size() < S->opt.max_wave; ++seen) {
        const uint64_t tk = S->pending.front();
        const Req &r = S->reqs[tk];
        if (sl.express ? !on_worklist(r.p) : longs_only && on_worklist(r.p)) {
            // not for this lane: stays queued for another slot (not a pass)
            other.push_back(tk);
            other_at.push_back(passed.size());
            S->pending.pop_front();
            continue;
        }
        auto fits = [&] { return S->inflight + foot + r.foot + S->seed_bytes <= S->budget; };
        if (!fits() && S->inflight + foot == 0)
            while (!fits() && seed_evict_one(S, sl.st)) {
            }
        if (!fits()) {
            if (r.passed >= kMaxPassed) break;  // stays at the head of what is left
            passed.push_back(tk);
            passed_at.push_back(wave.size());
            S->pending.pop_front();
            continue;
        }
        foot += r.foot;
        wave.push_back(tk);
        S->pending.pop_front();
    }
    // put the skipped requests back at the front in their queue order: the
    // passed ones (counted when a later request went first) and the ones this
    // slot does not take
    std::vector<uint64_t> back;
    back.reserve(passed.size() + other.size());
    for (size_t i = 0, j = 0; i < passed.size() || j < other.size();) {
        if (j < other.size() && (i >= passed.size() || other_at[j] <= i)) {
            back.push_back(other[j++]);
        } else {
            if (passed_at[i] < wave.size() && !sl.express) S->reqs[passed[i]].passed += 1;  // a later one went first
            back.push_back(passed[i++]);
        }
    }
    for (size_t j = back.size(); j-- > 0;) S->pending.push_front(back[j]);
    if (wave.empty()) return false;
    const uint64_t t = now_ns(), wid = ++S->waves;
    const uint32_t n = (uint32_t)wave.size();
    w.r.resize(n);
    w.bext.assign(n, nullptr);
    w.bready.assign(n, 0);
    w.make.assign(n, nullptr);
    sl.seeds.clear();
    for (uint32_t i = 0; i < n; ++i) {
        Req &r = S->reqs[wave[i]];
        r.t_admit = t;
        r.wave = wid;
        w.r[i].d = r.d;
        w.r[i].p = r.p;
        w.r[i].blocks = r.blocks;
        w.r[i].tmp_off = r.tmp_off;
        w.r[i].pre_off = r.pre_off;
        w.r[i].solo = !on_worklist(r.p);
        if (n == 1 && on_worklist(r.p) && !(r.flags & CM_REQ_SEED_CACHE)) {
            // a wave of one: the single call's kernels (one to a few launches)
            // instead of building and uploading a work list, within the same
            // footprint
            PlanOptions po = S->ctx->popt;
            po.budget = S->budget;
            std::vector<Block> bl;
            uint64_t to = 0, pf = 0;
            if (make_blocks(r.d.kind, r.d.n, r.d.m, po, &bl) && r256(blocks_scratch(bl, &to, &pf)) + 256 <= r.foot) {
                w.r[i].blocks.swap(bl);
                w.r[i].tmp_off = to;
                w.r[i].pre_off = pf;
                w.r[i].solo = true;
            }
        }
        // resident seed transforms (work-list requests with one column pass)
        if (!(r.flags & CM_REQ_SEED_CACHE) || !on_worklist(r.p) || r.p.npass != 1) continue;
        const SeedKey key{r.seed_id, r.p.n, r.p.m, r.p.kind};
        auto it = S->seeds.find(key);
        if (it != S->seeds.end()) {
            if (!it->second.ready) continue;  // still being made by a wave in flight
            it->second.refs += 1;
            it->second.last = ++S->lru;
            w.bext[i] = it->second.buf;
            w.bready[i] = 1;
            sl.seeds.push_back({key, false});
            ++S->seed_hits;
            continue;
        }
        const size_t bytes = worklist_seed_bytes(r.p);
        if (!seed_make_room(S, bytes, sl.st)) continue;
        SeedEntry e;
        e.bytes = bytes;
        e.refs = 1;
        e.last = ++S->lru;
        w.make[i] = &S->seeds.emplace(key, e).first->second;  // node addresses survive rehashing
        S->seed_bytes += bytes;
        sl.seeds.push_back({key, true});
        ++S->seed_misses;
    }
    sl.tickets = wave;
    sl.foot = foot;
    sl.wave = wid;
    sl.busy = true;
    S->inflight += foot;
    if (S->inflight > S->max_inflight) S->max_inflight = S->inflight;
    return true;
}

// Plan, upload and launch an admitted wave on slot sl (without the lock: it
// touches only the slot, the wave's copies and the seed entries it created,
// which no other thread reads).
cm_status enqueue_wave(cm_server *S, Slot &sl, Wave &w, uint8_t *scratch, const std::vector<size_t> &off,
                       const std::vector<uint32_t> &wl, const std::vector<uint32_t> &solo) {
    cm_ctx *ctx = S->ctx;
    const uint32_t n = (uint32_t)w.r.size();
    std::vector<cm_desc> descs(n);
    std::vector<Plan> plans(n);
    for (uint32_t i = 0; i < n; ++i) {
        descs[i] = w.r[i].d;
        plans[i] = w.r[i].p;
    }
    // flags: status word, pad, then a pair per work-list instance (index k) and
    // one per single-call request (index wl.size() + i)
    const size_t flag_words = 2 + 2 * ((size_t)n + n);
    if (!sl.flags.ensure(flag_words * 4)) return CM_ENOMEM;
    uint32_t *dflags = static_cast<uint32_t *>(sl.flags.dev);
    std::vector<void *> bext(wl.size(), nullptr);
    std::vector<uint8_t> bready(wl.size(), 0);
    for (uint32_t k = 0; k < wl.size(); ++k) {
        const uint32_t i = wl[k];
        if (SeedEntry *e = w.make[i]) {
            if (cudaMallocFromPoolAsync(&e->buf, e->bytes, ctx->pool, sl.st) != cudaSuccess) {
                cudaGetLastError();
                e->buf = nullptr;  // no resident transform: the wave computes it in scratch
            }
            w.bext[i] = e->buf;
        }
        bext[k] = w.bext[i];
        bready[k] = w.bready[i];
    }
    std::vector<BatchInst> insts;
    std::vector<WorkItem> items;
    build_worklist(descs.data(), plans.data(), wl.data(), (uint32_t)wl.size(), scratch, off.data(), kTileLg,
                   dflags + 2, insts, items, bext.data(), bready.data());
    sl.pre_index.assign(n, -1);
    for (uint32_t k = 0; k < wl.size(); ++k)
        if (plans[wl[k]].kind == CM_DODIS) sl.pre_index[wl[k]] = (int)k;
    if (cudaMemsetAsync(dflags, 0xff, flag_words * 4, sl.st) != cudaSuccess) return CM_EDEVICE;  // pairs "ok"
    if (cudaMemsetAsync(dflags, 0, 4, sl.st) != cudaSuccess) return CM_EDEVICE;                 // status word
    if (!wl.empty() && !items.empty()) {
        const size_t ib = insts.size() * sizeof(BatchInst), wb = items.size() * sizeof(WorkItem);
        const size_t cb = (2 + 4 * insts.size()) * sizeof(uint32_t);
        if (!sl.insts.ensure(ib) || !sl.items.ensure(wb) || !sl.ctrl.ensure(cb)) return CM_ENOMEM;
        memcpy(sl.insts.host, insts.data(), ib);
        memcpy(sl.items.host, items.data(), wb);
        if (cudaMemcpyAsync(sl.insts.dev, sl.insts.host, ib, cudaMemcpyHostToDevice, sl.st) != cudaSuccess ||
            cudaMemcpyAsync(sl.items.dev, sl.items.host, wb, cudaMemcpyHostToDevice, sl.st) != cudaSuccess ||
            cudaMemsetAsync(sl.ctrl.dev, 0, cb, sl.st) != cudaSuccess)
            return CM_EDEVICE;
        ProfScope ps(ctx, "k_batch", sl.st);
        if (launch_k_batch(static_cast<BatchInst *>(sl.insts.dev), static_cast<WorkItem *>(sl.items.dev),
                           (uint32_t)items.size(), static_cast<uint32_t *>(sl.ctrl.dev), dflags, ctx->rt25, S->grid,
                           sl.st) != cudaSuccess)
            return CM_EDEVICE;
    }
    for (uint32_t i : solo) {
        const WaveReq &r = w.r[i];
        uint8_t *sc = scratch + off[i];
        cm_status s = enqueue_blocks(ctx, r.blocks, r.d.x, r.d.y, r.d.z, sc, r.tmp_off, r.pre_off, sl.st);
        if (s != CM_OK) return s;
        if (r.p.kind == CM_DODIS) {
            // the single-call path keeps its flag pair at pre_off of its scratch
            const uint8_t *pf = sc + r.pre_off;
            sl.pre_index[i] = (int)(wl.size() + i);
            if (cudaMemcpyAsync(dflags + 2 + 2 * (wl.size() + i), pf, 8, cudaMemcpyDeviceToDevice, sl.st) !=
                cudaSuccess)
                return CM_EDEVICE;
        }
    }
    if (cudaMemcpyAsync(sl.flags.host, dflags, flag_words * 4, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
        return CM_EDEVICE;
    return CM_OK;
}

// Scratch layout, allocation and launch of an admitted wave; the scratch goes
// back to the pool (stream-ordered) whatever happens.
cm_status launch_wave(cm_server *S, Slot &sl, Wave &w) {
    const uint32_t n = (uint32_t)w.r.size();
    std::vector<size_t> off(n, 0);
    std::vector<uint32_t> wl, solo;
    size_t total = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const WaveReq &r = w.r[i];
        off[i] = total;
        if (!r.solo) {
            wl.push_back(i);
            total += worklist_scratch_bytes(r.p);
        } else {
            solo.push_back(i);
            uint64_t t0, t1;
            total += r256(blocks_scratch(r.blocks, &t0, &t1));
        }
    }
    void *scratch = nullptr;
    if (total && cudaMallocFromPoolAsync(&scratch, total, S->ctx->pool, sl.st) != cudaSuccess) {
        cudaGetLastError();
        return CM_ENOMEM;
    }
    cm_status s = enqueue_wave(S, sl, w, static_cast<uint8_t *>(scratch), off, wl, solo);
    if (scratch) cudaFreeAsync(scratch, sl.st);
    if (s == CM_OK && cudaEventRecord(sl.ev, sl.st) != cudaSuccess) s = CM_EDEVICE;
    return s;
}

void worker_main(cm_server *S) {
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progress = false;
        bool any_busy = false;
        for (Slot &sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaSuccess) {
                finish_slot(S, sl);
                progress = true;
            } else if (q != cudaErrorNotReady) {
                fail_wave(S, sl, CM_EDEVICE);
                progress = true;
            } else {
                any_busy = true;
            }
        }
        if (progress) S->cv_done.notify_all();
        if (S->stop && S->pending.empty() && !any_busy) break;
        for (Slot &sl : S->slots) {
            if (sl.busy || S->pending.empty()) continue;
            Wave w;
            if (!admit_wave(S, sl, w)) continue;  // another slot may take what this one does not
            // submissions and polls proceed while the wave is planned and launched
            lk.unlock();
            cm_status s = launch_wave(S, sl, w);
            if (s != CM_OK) cudaStreamSynchronize(sl.st);
            lk.lock();
            if (s != CM_OK) {
                fail_wave(S, sl, s);
                S->cv_done.notify_all();
            }
            progress = true;
        }
        if (!progress) S->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

void server_release(cm_server *S) {
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->seeds) cudaFree(kv.second.buf);  // pool memory; device is idle here
    S->seeds.clear();
    for (Slot &sl : S->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        sl.insts.release();
        sl.items.release();
        sl.ctrl.release();
        sl.flags.release();
        if (sl.ev) cudaEventDestroy(sl.ev);
    }
    for (Slot &sl : S->slots)
        if (sl.st && !sl.borrowed) cudaStreamDestroy(sl.st);
    delete S;
}

}  // namespace

void cm_ctx_release_extras(cm_ctx *c) {
    if (c->server) {
        server_release(c->server);
        c->server = nullptr;
    }
}

extern "C" cm_status cm_server_start(cm_ctx *ctx, const cm_server_options *opt) {
    if (!ctx) return CM_EINVAL;
    if (ctx->server) return CM_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    cm_server *S = new cm_server();
    S->ctx = ctx;
    if (opt) S->opt = *opt;
    if (!S->opt.slots) S->opt.slots = 3;
    if (!S->opt.max_queue) S->opt.max_queue = 1u << 20;
    if (!S->opt.max_wave) S->opt.max_wave = 512;
    S->budget = S->opt.hbm_budget_bytes ? S->opt.hbm_budget_bytes : ctx->budget / 2;
    if (S->budget > ctx->budget) S->budget = ctx->budget;
    S->seed_limit = S->opt.seed_cache_bytes ? S->opt.seed_cache_bytes : S->budget / 4;
    S->grid = batch_grid(ctx->nsm);
    if (S->grid < 1) {
        delete S;
        return CM_EDEVICE;
    }
    const uint32_t express = S->opt.express_slots == CM_SERVER_NO_EXPRESS ? 0u
                             : S->opt.express_slots ? S->opt.express_slots : 1u;
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        delete S;
        return CM_EDEVICE;
    }
    // Each regular stream carries two slots: the worker plans and enqueues a
    // wave behind the one running there, so the stream does not idle while it
    // notices a completion and launches the next wave.  Express slots have a
    // stream each.
    const uint32_t R = S->opt.slots;
    S->express = express;
    S->slots.resize(2 * (size_t)R + express);
    for (size_t i = 0; i < S->slots.size(); ++i) {
        Slot &sl = S->slots[i];
        sl.express = i >= 2 * (size_t)R;
        sl.borrowed = i >= R && !sl.express;
        cudaError_t e = sl.borrowed ? cudaSuccess
                                    : cudaStreamCreateWithPriority(&sl.st, cudaStreamNonBlocking,
                                                                   sl.express ? prio_high : prio_low);
        if (sl.borrowed) sl.st = S->slots[i - R].st;
        if (e != cudaSuccess || cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            if (sl.borrowed) sl.st = nullptr;
            server_release(S);
            return CM_EDEVICE;
        }
    }
    ctx->server = S;
    S->worker = std::thread(worker_main, S);
    return CM_OK;
}

extern "C" cm_status cm_server_stop(cm_ctx *ctx) {
    if (!ctx || !ctx->server) return CM_EINVAL;
    server_release(ctx->server);
    ctx->server = nullptr;
    return CM_OK;
}

extern "C" cm_status cm_submit(cm_ctx *ctx, const cm_request *rq, uint64_t *ticket) {
    if (!ctx || !rq || !ticket) return CM_EINVAL;
    cm_server *S = ctx->server;
    if (!S) return CM_EINVAL;
    Req r;
    r.d.kind = rq->kind;
    r.d.reserved = 0;
    r.d.n = rq->n;
    r.d.m = rq->m;
    r.d.x = rq->x;
    r.d.y = rq->y;
    r.d.z = rq->z;
    r.flags = rq->flags;
    r.seed_id = rq->seed_id;
    if (rq->flags & ~CM_REQ_SEED_CACHE) return CM_EINVAL;
    if (!rq->x || !rq->y || !rq->z || !make_plan(rq->kind, rq->n, rq->m, &r.p, worklist_fields(ctx->popt))) return CM_EINVAL;
    if (!on_worklist(r.p)) {
        // too long for the work list: the single-call planner (one product, or
        // sums of shorter products and a dense tail) within the server's budget
        PlanOptions po = ctx->popt;
        po.budget = S->budget;
        if (!make_blocks(rq->kind, rq->n, rq->m, po, &r.blocks)) return CM_EINVAL;
        r.foot = r256(blocks_scratch(r.blocks, &r.tmp_off, &r.pre_off));
    } else {
        r.foot = worklist_scratch_bytes(r.p);
    }
    r.foot += 256;  // work-list and flag share
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (r.foot > S->budget) {
            ++S->rejected;
            return CM_ENOMEM;
        }
        if (S->pending.size() >= S->opt.max_queue || S->stop) {
            ++S->rejected;
            return CM_EAGAIN;
        }
        const uint64_t t = S->next_ticket++;
        r.t_submit = now_ns();
        S->reqs.emplace(t, r);
        S->pending.push_back(t);
        ++S->submitted;
        *ticket = t;
    }
    S->cv_work.notify_one();
    return CM_OK;
}

extern "C" cm_status cm_poll(cm_ctx *ctx, uint64_t ticket, cm_result *res, uint64_t timeout_ns) {
    if (!ctx || !ctx->server) return CM_EINVAL;
    cm_server *S = ctx->server;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return CM_ENOTFOUND;
    if (!it->second.done) {
        S->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), [&] {
            auto j = S->reqs.find(ticket);
            return j == S->reqs.end() || j->second.done;
        });
        it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return CM_ENOTFOUND;
        if (!it->second.done) return CM_EAGAIN;
    }
    const Req &r = it->second;
    if (res) {
        memset(res, 0, sizeof(*res));
        res->status = r.status;
        res->t_submit_ns = r.t_submit;
        res->t_admit_ns = r.t_admit;
        res->t_done_ns = r.t_done;
        res->wave = r.wave;
    }
    S->reqs.erase(it);
    return CM_OK;
}

extern "C" cm_status cm_server_get_stats(cm_ctx *ctx, cm_server_stats *st) {
    if (!ctx || !ctx->server || !st) return CM_EINVAL;
    cm_server *S = ctx->server;
    std::lock_guard<std::mutex> g(S->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->waves = S->waves;
    st->inflight_bytes = S->inflight;
    st->max_inflight_bytes = S->max_inflight;
    st->budget_bytes = S->budget;
    st->seed_cache_hits = S->seed_hits;
    st->seed_cache_misses = S->seed_misses;
    st->seed_cache_bytes = S->seed_bytes;
    st->seed_cache_entries = S->seeds.size();
    st->queued = (uint32_t)S->pending.size();
    uint32_t busy = 0;
    for (const Slot &sl : S->slots) busy += sl.busy ? 1u : 0u;
    st->busy_slots = busy;
    st->slots = (uint32_t)S->slots.size();
    return CM_OK;
}
