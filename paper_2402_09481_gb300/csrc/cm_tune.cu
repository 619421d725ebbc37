// Planner calibration on the device (cm_calibrate): the cost figures the
// planner compares shapes by, and the pass split of two-pass transforms,
// timed on this GPU with this build's kernels, kept in the context and cached
// in a text file keyed by the device's name and SM count.
//
// Each figure is the device time of one Toeplitz extraction of transform
// length 2^lg (K = L/2 + 1, m = L/4: the definition of the built-in tables),
// one warm-up, then the median of three with L2 flushed (a 256 MiB write)
// before each.  Per field: 5 * 2^25 + 1 over 2^9 .. 2^25 (the column-pass form;
// 2^14 .. 2^17 also as one cluster launch), 3 * 2^30 + 1 and Goldilocks from
// 2^14 up, to max_lg and within the context's HBM budget.  For two-pass
// lengths the first pass's log2 R is chosen among the default split and its
// two neighbours.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "cm.h"
#include "cm_ctx.h"
#include "cm_internal.h"

namespace cm {
cm_status enqueue_extract(cm_ctx *ctx, const Plan &p, const uint64_t *x, const uint64_t *y, uint64_t *z,
                          void *scratch, cudaStream_t st);
}

using namespace cm;

namespace {

constexpr size_t kFlushBytes = 256u << 20;

int field_set(int field) { return field == kFieldF25 ? kFieldsAll : field == kFieldF30 ? kFieldsQ30 : kFieldsGL; }
int lg_lo(int field) { return field == kFieldF25 ? 9 : 14; }
int lg_hi(int field) { return field == kFieldF25 ? kF25MaxLg : field == kFieldF30 ? kF30MaxLg : 32; }

// Device buffers of one timing, grown on demand.
struct TimeBufs {
    void *x = nullptr, *y = nullptr, *z = nullptr, *sc = nullptr, *flush = nullptr;
    size_t xb = 0, yb = 0, zb = 0, scb = 0;
    bool grow(void **p, size_t *have, size_t want) {
        if (want <= *have) return true;
        if (*p) cudaFree(*p);
        *p = nullptr;
        *have = 0;
        if (cudaMalloc(p, want) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        *have = want;
        return cudaMemset(*p, 0x5a, want) == cudaSuccess;
    }
    ~TimeBufs() {
        for (void *p : {x, y, z, sc, flush})
            if (p) cudaFree(p);
    }
};

// Median device time (ms) of three extractions of plan p; negative on error.
double time_plan(cm_ctx *ctx, const Plan &p, TimeBufs &b, cudaStream_t st) {
    const size_t xb = 8 * ((p.n + 63) / 64), yb = 8 * ((p.n + p.m - 1 + 63) / 64), zb = 8 * ((p.m + 63) / 64);
    if (!b.grow(&b.x, &b.xb, xb) || !b.grow(&b.y, &b.yb, yb) || !b.grow(&b.z, &b.zb, zb) ||
        !b.grow(&b.sc, &b.scb, std::max<size_t>(p.scratch_bytes, 256)))
        return -1;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
    std::vector<float> ms;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {
        ok = cudaMemsetAsync(b.flush, rep, kFlushBytes, st) == cudaSuccess &&
             cudaEventRecord(e0, st) == cudaSuccess &&
             enqueue_extract(ctx, p, static_cast<uint64_t *>(b.x), static_cast<uint64_t *>(b.y),
                             static_cast<uint64_t *>(b.z), b.sc, st) == CM_OK &&
             cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float t = 0.f;
        if (ok && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) ok = false;
        if (ok && rep > 0) ms.push_back(t);  // the first is the warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) {
        cudaGetLastError();
        return -1;
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

// The timed plan of length 2^lg in `field` (Toeplitz, K = L/2 + 1, m = L/4).
bool timed_plan(int field, int lg, bool cluster, int split, Plan *p) {
    const uint64_t L = 1ull << lg;
    Tuning t{};
    if (split) t.split[field][lg] = (int8_t)split;
    if (!make_plan(CM_TOEPLITZ, L / 2 + 1, L / 4, p, field_set(field), split ? &t : nullptr)) return false;
    if (p->lg != lg || p->field != field) return false;
    p->cluster = p->cluster && cluster;
    return true;
}

std::string device_key(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return std::string();
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ' || c == '\t' || c == '\n') c = '_';
    return name + " " + std::to_string(prop.multiProcessorCount);
}

bool load_cache(const char *path, const std::string &key, Tuning *t) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool head = false, dev = false;
    Tuning r{};
    while (fgets(line, sizeof line, f)) {
        char kind[32] = {0}, a[256] = {0};
        int fld = 0, lg = 0, sp = 0, sms = 0;
        double ms = 0;
        if (sscanf(line, "cm-tune %d", &fld) == 1) {
            head = fld == 2;
        } else if (sscanf(line, "device %255s %d", a, &sms) == 2) {
            dev = key == std::string(a) + " " + std::to_string(sms);
        } else if (sscanf(line, "%31s", kind) == 1) {
            if (!strcmp(kind, "cost") && sscanf(line, "cost %d %d %lf", &fld, &lg, &ms) == 3 && fld >= 0 && fld < 3 &&
                lg >= 0 && lg <= 32 && ms > 0)
                r.cost[fld][lg] = ms;
            else if (!strcmp(kind, "cluster") && sscanf(line, "cluster %d %lf", &lg, &ms) == 2 &&
                     lg >= kClusterMinLg && lg <= kClusterMaxLg && ms > 0)
                r.cluster[lg - kClusterMinLg] = ms;
            else if (!strcmp(kind, "split") && sscanf(line, "split %d %d %d", &fld, &lg, &sp) == 3 && fld >= 0 &&
                     fld < 3 && lg >= 0 && lg <= 32)
                r.split[fld][lg] = (int8_t)sp;
        }
    }
    fclose(f);
    if (!head || !dev) return false;
    *t = r;
    return true;
}

bool save_cache(const char *path, const std::string &key, const Tuning &t) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "cm-tune 2\ndevice %s\n", key.c_str());
    for (int fld = 0; fld < 3; ++fld)
        for (int lg = 0; lg <= 32; ++lg)
            if (t.cost[fld][lg] > 0) fprintf(f, "cost %d %d %.17g\n", fld, lg, t.cost[fld][lg]);
    for (int i = 0; i <= kClusterMaxLg - kClusterMinLg; ++i)
        if (t.cluster[i] > 0) fprintf(f, "cluster %d %.17g\n", kClusterMinLg + i, t.cluster[i]);
    for (int fld = 0; fld < 3; ++fld)
        for (int lg = 0; lg <= 32; ++lg)
            if (t.split[fld][lg]) fprintf(f, "split %d %d %d\n", fld, lg, (int)t.split[fld][lg]);
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

}  // namespace

extern "C" cm_status cm_calibrate(cm_ctx *ctx, const char *cache_path, uint32_t flags, uint32_t max_lg) {
    if (!ctx || (flags & ~CM_TUNE_FORCE) || max_lg > 32 || (max_lg && max_lg < 9)) return CM_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    const std::string key = device_key(ctx->device);
    if (key.empty()) return CM_EDEVICE;
    Tuning t{};
    if (cache_path && !(flags & CM_TUNE_FORCE) && load_cache(cache_path, key, &t)) {
        ctx->tune = t;
        ctx->popt.tune = &ctx->tune;
        return CM_OK;
    }
    const int top = max_lg ? (int)max_lg : 30;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return CM_EDEVICE;
    TimeBufs b;
    size_t flush_have = 0;
    cm_status s = b.grow(&b.flush, &flush_have, kFlushBytes) ? CM_OK : CM_ENOMEM;
    for (int field : {kFieldF25, kFieldF30, kFieldGL}) {
        for (int lg = lg_lo(field); s == CM_OK && lg <= std::min(top, lg_hi(field)); ++lg) {
            Plan p;
            if (!timed_plan(field, lg, false, 0, &p)) continue;
            if (p.scratch_bytes > ctx->budget) break;  // longer lengths keep the built-in figures
            double best = time_plan(ctx, p, b, st);
            if (best < 0) {
                s = CM_EDEVICE;
                break;
            }
            if (p.npass == 2) {
                // the first pass's length: the default and its neighbours
                const int rest = lg - kMidLgMax, d = p.pass_lg[0];
                for (int f : {d - 1, d + 1}) {
                    if (f < 1 || f > 12 || rest - f < 1 || rest - f > 12) continue;
                    Plan q;
                    if (!timed_plan(field, lg, false, f, &q) || q.pass_lg[0] != f) continue;
                    const double ms = time_plan(ctx, q, b, st);
                    if (ms > 0 && ms < best) {
                        best = ms;
                        t.split[field][lg] = (int8_t)f;
                    }
                }
            }
            t.cost[field][lg] = best;
            if (field == kFieldF25 && lg >= kClusterMinLg && lg <= kClusterMaxLg) {
                Plan c;
                if (timed_plan(field, lg, true, 0, &c) && c.cluster) {
                    const double ms = time_plan(ctx, c, b, st);
                    if (ms > 0) t.cluster[lg - kClusterMinLg] = ms;
                }
            }
        }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (s != CM_OK) return s;
    ctx->tune = t;
    ctx->popt.tune = &ctx->tune;
    if (cache_path && !save_cache(cache_path, key, t)) return CM_EINVAL;
    return CM_OK;
}

extern "C" cm_status cm_tune_query(const cm_ctx *ctx, uint32_t field, uint32_t lg, double *ms, double *cluster_ms,
                                   int32_t *split) {
    if (!ctx || lg > 32) return CM_EINVAL;
    int f;
    switch (field) {
        case CM_FIELD_GOLDILOCKS: f = kFieldGL; break;
        case CM_FIELD_Q30: f = kFieldF30; break;
        case CM_FIELD_Q25: f = kFieldF25; break;
        default: return CM_EINVAL;
    }
    const bool on = ctx->popt.tune != nullptr;
    if (ms) *ms = on ? ctx->tune.cost[f][lg] : 0.0;
    if (cluster_ms)
        *cluster_ms = on && f == kFieldF25 && (int)lg >= kClusterMinLg && (int)lg <= kClusterMaxLg
                          ? ctx->tune.cluster[lg - kClusterMinLg]
                          : 0.0;
    if (split) *split = on ? ctx->tune.split[f][lg] : 0;
    return CM_OK;
}
