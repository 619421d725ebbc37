// C ABI entry points: context, plans, single extractions.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "cm.h"
#include "cm_internal.h"
#include "cm_ctx.h"
#include "ntt25.cuh"

namespace cm {

uint64_t current_ctx_id() {
    typedef int (*GetCurrent)(void **);
    typedef int (*GetId)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess && qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(a);
            get_id = reinterpret_cast<GetId>(b);
        }
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    void *c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != 0 || !c || get_id(c, &id) != 0) return 0;
    return id;
}

static int ceil_log2(uint64_t v) {
    int k = 0;
    while ((1ull << k) < v) ++k;  // v <= 2^33 here
    return k;
}

// Operand maps of (kind, n, m) (lengths up to 2^40); false if invalid.
static bool base_maps(int kind, uint64_t n, uint64_t m, Plan *p) {
    memset(p, 0, sizeof(*p));
    p->kind = kind;
    p->n = n;
    p->m = m;
    if (m == 0 || n == 0) return false;
    // every length below is checked against 2^40 before any sum can overflow
    if (n > kMaxBits || m > kMaxBits) return false;
    switch (kind) {
        case CM_TOEPLITZ: {
            const uint64_t N = n + m - 1;  // seed length
            p->K = n;
            p->amode = kIdentity; p->alen = n; p->asrclen = n; p->aoff = 0;
            // b_k = y[(k - n + 1) mod N] = y[(k + m) mod N]
            p->bmode = kModForward; p->blen = N; p->bsrclen = N; p->boff = m % N;
            break;
        }
        case CM_CIRCULANT: {
            const uint64_t P = n + 1;
            if (m > n || !is_na_prime(P)) return false;
            p->K = P;
            // rev(x')_u = x'_{P-1-u}, x' = [x, 0]: u = 0 reads the pad bit (index n, zero)
            p->amode = kReverse; p->alen = P; p->asrclen = n; p->aoff = n;
            p->bmode = kModForward; p->blen = P + m - 1; p->bsrclen = P; p->boff = 0;
            break;
        }
        case CM_DODIS: {
            if (m > n || !is_na_prime(n)) return false;
            p->K = n;
            p->amode = kReverse; p->alen = n; p->asrclen = n; p->aoff = n - 1;
            p->bmode = kModForward; p->blen = n + m - 1; p->bsrclen = n; p->boff = 0;
            break;
        }
        default:
            return false;
    }
    return true;
}

bool valid_args(int kind, uint64_t n, uint64_t m) {
    Plan p;
    return base_maps(kind, n, m, &p);
}

// Scratch of one product: the operands A and B (and the transform-domain sum C
// of a summed window) and the parity bytes; one-CTA plans (lg <= 13) keep
// everything on chip.  A single call's plan adds 256 bytes of Dodis et al.
// precondition flags (kFlagBytes).
constexpr uint64_t kFlagBytes = 256;
static uint64_t flag_bytes(int kind) { return kind == CM_DODIS ? kFlagBytes : 0; }
static uint64_t plan_scratch(int lg, uint64_t m, int field, bool summed) {
    if (lg <= kMidLgMax) return 0;
    const uint64_t esz = field == kFieldGL ? 8 : 4;
    return (summed ? 3 : 2) * esz * (1ull << lg) + ((m + 255) & ~255ull);
}

// Transform length (at least 2^min_lg), field, pass split, scratch and launch
// count for K + m - 1 <= 2^32.
static void finish_plan(Plan *p, int fields, int min_lg, bool summed, const Tuning *tune = nullptr) {
    const uint64_t need = p->K + p->m - 1;
    p->lg = ceil_log2(need);
    if (p->lg < min_lg) p->lg = min_lg;
    if (p->lg < 1) p->lg = 1;
    p->L = 1ull << p->lg;
    p->lo = p->K - 1;
    p->field = field_for(fields, p->lg);
    p->summed = summed;
    const int rest = p->lg - kMidLgMax;
    if (rest <= 0) {
        p->npass = 0;
    } else if (rest <= 12) {
        p->npass = 1;
        p->pass_lg[0] = rest;
    } else {
        p->npass = 2;
        p->pass_lg[0] = (rest + 1) / 2;
        const int f = tune ? tune->split[p->field][p->lg] : 0;  // a calibrated split, if valid
        if (f >= 1 && f <= 12 && rest - f >= 1 && rest - f <= 12) p->pass_lg[0] = f;
        p->pass_lg[1] = rest - p->pass_lg[0];
    }
    p->scratch_bytes = plan_scratch(p->lg, p->m, p->field, summed) + flag_bytes(p->kind);
    p->cluster = p->field == kFieldF25 && !summed && p->lg >= kClusterMinLg && p->lg <= kClusterMaxLg;
    // forward passes (both operands per launch), middle, inverse passes, pack;
    // one launch on chip or on a cluster
    p->launches = (p->npass == 0 || p->cluster) ? 1 : p->npass + 1 + p->npass + 1;
    if (p->kind == CM_DODIS) p->launches += 1;  // precondition check
}

bool make_plan(int kind, uint64_t n, uint64_t m, Plan *p, int fields, const Tuning *tune) {
    if (!base_maps(kind, n, m, p)) return false;
    if (p->K + m - 1 > (1ull << 32)) return false;
    finish_plan(p, fields, 1, false, tune);
    return true;
}

// ---------------------------------------------------------------------------
// Block planner.
//
// z_i = sum_{t<K} a_t b_{t+i} splits over input blocks t in [T0, T0 + kb)
// (each a middle product of a[T0 .. T0 + kb) with b[T0 .. T0 + kb + m - 1))
// and over output windows i in [I0, I0 + mb) (b shifted by I0).  In transform
// positions u = K - 1 - t, input block [D, D + kb) of A is A shifted by D.
// Every input block of a window is planned with the same K = Kb (a shorter
// last block is zero beyond its kb positions and its b map moves back by
// Kb - kb), so all of them share the transform length and the output window
// position: their transform-domain products are added (exact integer counts,
// at most K < q in total) and one inverse transform with parity serves the
// window.
//
// Shapes (block transform length 2^lg, output windows, input blocks) are
// compared by an estimate of GPU time built from measured whole-extraction
// times per transform length and field: a summed window costs nin times the
// forward share (both forward transforms and the middle) plus one inverse
// share.
// ---------------------------------------------------------------------------

// Measured on one GB300 (SM clock 2070 MHz): ms per extraction of transform
// length 2^lg (Toeplitz, K = L/2 + 1, m = L/4, one transform); below 2^21
// launch latency dominates and the figures are floors.
static const double kCostF30[kF30MaxLg + 1] = {
    0.02,  0.02,  0.02,  0.02,  0.02,  0.02,  0.02,   0.02,   0.02,   0.02,   0.02,
    0.02,  0.02,  0.02,  0.080, 0.081, 0.0822, 0.0829, 0.0857, 0.0950, 0.0991, 0.1162,
    0.1907, 0.3389, 0.6710, 1.3995, 2.6839, 5.4039, 10.960, 22.246, 45.643};
static const double kCostF25[kF25MaxLg + 1] = {
    0.0106, 0.0106, 0.0106, 0.0106, 0.0106, 0.0106, 0.0106, 0.0106, 0.0106, 0.0106, 0.0106,
    0.0126, 0.0188, 0.0328, 0.0551, 0.0582, 0.0579, 0.0598, 0.0616, 0.0632, 0.0653, 0.0824,
    0.1060, 0.1668, 0.3264, 0.7317};
// A product standing alone at 2^14 .. 2^17 runs as one cluster launch
// (cm_cluster25.cu); L2 flushed before each call as above.
static const double kCostCluster25[kClusterMaxLg - kClusterMinLg + 1] = {0.0312, 0.0309, 0.0312, 0.0333};
static const double kCostGL[33] = {
    0.03,  0.03,  0.03,  0.03,  0.03,  0.03,  0.03,  0.03,  0.03,   0.03,   0.03,
    0.03,  0.03,  0.03,  0.130, 0.133, 0.1356, 0.1419, 0.1459, 0.1604, 0.1678, 0.2221,
    0.4375, 0.8792, 1.6702, 3.3082, 7.4412, 15.095, 30.538, 62.422, 127.87, 261.78, 534.40};
constexpr double kFwdShare = 0.77;     // forward passes of both operands + middle
constexpr double kInvRowShare = 0.15;  // the middle's inverse row transform (a third of it)
constexpr double kSumShare = kFwdShare - kInvRowShare;  // a product summed into C
constexpr double kXorMs = 0.005;       // one k_xor_into launch
// the dense tail: a launch plus about 1.5 ns per 1000 outputs (a fixed
// kTailMax-term loop per output word)
static double tail_cost(uint64_t m) { return 0.005 + 1.5e-9 * (double)m; }
constexpr double kSingleMargin = 0.97;  // a blocked shape must beat one transform by 3%
constexpr int kSumMinLg = kMidLgMax + 1;  // summed windows need a column pass

static uint64_t words_of(uint64_t bits) { return (bits + 63) / 64; }
static uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

static double plan_cost(int field, int lg, const Tuning *tune = nullptr) {
    if (tune && tune->cost[field][lg] > 0) return tune->cost[field][lg];
    return field == kFieldF25 ? kCostF25[lg] : field == kFieldF30 ? kCostF30[lg] : kCostGL[lg];
}
// A product that is not summed with others (its own inverse transform).
static double alone_cost(int field, int lg, const Tuning *tune = nullptr) {
    if (field == kFieldF25 && lg >= kClusterMinLg && lg <= kClusterMaxLg) {
        if (tune && tune->cluster[lg - kClusterMinLg] > 0) return tune->cluster[lg - kClusterMinLg];
        return kCostCluster25[lg - kClusterMinLg];
    }
    return plan_cost(field, lg, tune);
}

// Input blocks whose products one sum may hold: the counts of G blocks add up
// to at most G Kb, which must stay below the field's characteristic (the
// Goldilocks prime exceeds every count up to 2^40).  Windows with more blocks
// sum in groups, each with its own inverse transform; the groups' parities XOR.
static uint64_t group_size(int field, uint64_t Kb, uint64_t nin, uint32_t cap) {
    // >= 3: Kb <= 2^30 (F30), Kb <= 2^25 (F25)
    uint64_t g = field == kFieldF30 ? (F30_Q - 1) / Kb : field == kFieldF25 ? (F25_Q - 1) / Kb : nin;
    if (cap && g > cap) g = cap;
    return g < nin ? g : nin;
}

// One window of nin input blocks summed in groups of G (G = 1: every block
// inverse-transformed on its own and XORed): a group's last block costs a
// whole extraction, the others their forward passes and the middle without
// its inverse row transform.
static double window_cost(int field, int lg, uint64_t nin, uint64_t G, const Tuning *tune) {
    const double t = plan_cost(field, lg, tune);
    const uint64_t ng = ceil_div(nin, G);
    if (G == 1) return (double)nin * alone_cost(field, lg, tune) + (double)(nin - 1) * kXorMs;
    return ((double)(nin - ng) * kSumShare + (double)ng) * t + (double)(ng - 1) * kXorMs;
}


struct Shape {
    int lg;          // limit of the block transforms
    uint64_t Mb;     // outputs per window (a multiple of 64 when m splits)
    uint64_t nout;   // windows
    uint64_t nin;    // input blocks per window
    uint64_t Kb;     // terms per input block
    uint64_t tail;   // terms left to the dense tail (t < tail)
    bool summed;
    double cost;
    uint64_t scratch;
};

// Window transform length, field and scratch of a shape.
static int window_lg(const Shape &s, uint64_t mr) {
    int lg = ceil_log2(s.Kb + mr - 1);
    if (s.summed && lg < kSumMinLg) lg = kSumMinLg;
    return lg < 1 ? 1 : lg;
}

static void evaluate(int kind, uint64_t m, int fields, uint32_t max_sum, const Tuning *tune, Shape *s) {
    const uint64_t mlast = m - (s->nout - 1) * s->Mb;
    s->cost = 0;
    s->scratch = 0;
    bool xors = false;
    for (int w = 0; w < 2; ++w) {  // the nout - 1 full windows, then the last
        const uint64_t cnt = w == 0 ? s->nout - 1 : 1, mr = w == 0 ? s->Mb : mlast;
        if (!cnt) continue;
        const int lg = window_lg(*s, mr);
        const int field = field_for(fields, lg);
        const uint64_t G = s->summed ? group_size(field, s->Kb, s->nin, max_sum) : 1;
        s->cost += (double)cnt * window_cost(field, lg, s->nin, G, tune);
        const uint64_t sc = plan_scratch(lg, mr, field, s->summed);
        if (sc > s->scratch) s->scratch = sc;
        xors = xors || G < s->nin;
    }
    if (s->tail) s->cost += tail_cost(m);
    // blocks_scratch's layout: XOR temporary, then the precondition flags
    const uint64_t tmp_off = (s->scratch + 255) & ~255ull, tmpw = xors ? words_of(s->Mb) : 0;
    if (kind == CM_DODIS) s->scratch = ((tmp_off + 8 * tmpw + 255) & ~255ull) + kFlagBytes;
    else if (tmpw) s->scratch = tmp_off + 8 * tmpw;
}

bool plan_options(const cm_options *opt, PlanOptions *o) {
    *o = PlanOptions();
    if (!opt) return true;
    if (opt->max_transform_lg) {
        if (opt->max_transform_lg < 8 || opt->max_transform_lg > 32) return false;
        o->max_lg = (int)opt->max_transform_lg;
    }
    switch (opt->field) {
        case CM_FIELD_AUTO: o->fields = kFieldsAll; break;
        case CM_FIELD_Q30: o->fields = kFieldsQ30; break;
        case CM_FIELD_GOLDILOCKS: o->fields = kFieldsGL; break;
        default: return false;
    }
    o->budget = opt->hbm_budget_bytes;
    o->max_sum = opt->max_sum_blocks;
    if (opt->plan_mode > CM_PLAN_SINGLE) return false;
    o->single = opt->plan_mode == CM_PLAN_SINGLE;
    return true;
}

bool make_blocks(int kind, uint64_t n, uint64_t m, const PlanOptions &o, std::vector<Block> *out) {
    const int max_lg = o.max_lg;
    const int fields = o.fields;
    const uint64_t budget = o.budget;
    out->clear();
    Plan b;
    if (max_lg < 8 || max_lg > 32 || !base_maps(kind, n, m, &b)) return false;
    const uint64_t K = b.K;
    // candidate block limits: the single transform (when it fits) and, when the
    // limit allows column-pass plans, every limit from 2^14 up
    const int lg_single = ceil_log2(K + m - 1);
    std::vector<int> lgs;
    if (lg_single <= max_lg) lgs.push_back(lg_single);
    if (lg_single <= max_lg && o.single) {
        // one transform, as asked
    } else if (max_lg <= kMidLgMax) {
        if (lg_single > max_lg) lgs.push_back(max_lg);
    } else {
        for (int lg = kSumMinLg; lg <= max_lg; ++lg)
            if (lg != lg_single) lgs.push_back(lg);
    }
    Shape best{};
    bool have = false, best_fits = false;
    for (int lg : lgs) {
        const uint64_t Lmax = 1ull << lg;
        const uint64_t nout_min = ceil_div(m, Lmax);
        uint64_t nout_max = nout_min * 4 + 16;
        if (nout_max > kMaxBlocks) nout_max = kMaxBlocks;
        for (uint64_t nout = nout_min; nout <= nout_max; ++nout) {
            Shape s{};
            s.lg = lg;
            s.Mb = nout == 1 ? m : ceil_div(ceil_div(m, nout), 64) * 64;
            if (ceil_div(m, s.Mb) != nout || s.Mb > Lmax) continue;
            s.nout = nout;
            const uint64_t kmax = Lmax - s.Mb + 1;
            const uint64_t nin0 = ceil_div(K, kmax);
            // the fewest input blocks, and (column-pass limits, cost mode) one
            // block fewer when the terms left over fit the dense tail
            for (int with_tail = 0; with_tail < 2; ++with_tail) {
                Shape c = s;
                if (with_tail) {
                    if (max_lg <= kMidLgMax || o.single || lg < kSumMinLg || nin0 < 2) break;
                    const uint64_t left = K - (nin0 - 1) * kmax;
                    if (left > (uint64_t)kTailMax) break;
                    c.nin = nin0 - 1;
                    c.tail = left;
                } else {
                    c.nin = nin0;
                }
                if (c.nin > kMaxBlocks / c.nout) continue;  // (no overflow: both <= 2^40)
                c.Kb = ceil_div(K - c.tail, c.nin);
                c.summed = c.nin > 1 && max_lg > kMidLgMax;
                evaluate(kind, m, fields, o.max_sum, o.tune, &c);
                const bool single = c.nin == 1 && c.nout == 1 && c.tail == 0;
                const bool fits = budget == 0 || c.scratch <= budget;
                double cc = c.cost, bc = best.cost;
                if (!single) cc /= kSingleMargin;
                if (have && (best.nin * best.nout != 1 || best.tail)) bc /= kSingleMargin;
                const bool better = !have || (fits && !best_fits) ||
                                    (fits == best_fits &&
                                     (cc < bc || (cc == bc && c.nin * c.nout < best.nin * best.nout)));
                if (better) {
                    best = c;
                    have = true;
                    best_fits = fits;
                }
            }
        }
    }
    if (!have) return false;
    const Shape &s = best;
    if (s.nin == 1 && s.nout == 1 && s.tail == 0) {
        finish_plan(&b, fields, 1, false, o.tune);
        out->push_back({b, 0, kSumNone, false, 0});
        return true;
    }
    const uint64_t Kc = K - s.tail;  // terms t in [tail, K): transform positions u < Kc
    for (uint64_t r = 0; r < s.nout; ++r) {
        const uint64_t I0 = r * s.Mb, mr = (m - I0 < s.Mb) ? m - I0 : s.Mb;
        const int lg_r = window_lg(s, mr);
        const uint64_t G = s.summed ? group_size(field_for(fields, lg_r), s.Kb, s.nin, o.max_sum) : 1;
        for (uint64_t j = 0; j < s.nin; ++j) {
            const uint64_t D = j * s.Kb;  // < Kc: (nin - 1) Kb < Kc
            const uint64_t kb = (Kc - D < s.Kb) ? Kc - D : s.Kb;
            const uint64_t T0 = K - D - kb;
            Plan q = b;
            q.m = mr;
            q.K = s.Kb;
            if (b.amode == kIdentity) {  // A'_u = x_{D+u}: no wrap, u + D < K = srclen
                q.amode = kModForward;
                q.aoff = D;
            } else {  // A'_u = src[aoff - D - u]
                q.aoff = b.aoff - D;
            }
            q.alen = kb;  // zero beyond: the padded positions of a short block
            q.blen = s.Kb + mr - 1;
            // B'_v = B_{v + T0 + I0 - (Kb - kb)}, kept in [0, bsrclen)
            const uint64_t src = b.bsrclen;
            q.boff = ((b.boff + T0 + I0) % src + src - (s.Kb - kb) % src) % src;
            finish_plan(&q, fields, lg_r, s.summed, o.tune);
            // sum group [g0, g1) of this window; a group of one stands alone
            const uint64_t g0 = j / G * G, g1 = (g0 + G < s.nin) ? g0 + G : s.nin;
            int sum = kSumNone;
            if (g1 - g0 > 1) sum = j == g0 ? kSumFirst : (j + 1 == g1 ? kSumLast : kSumInner);
            const bool packs = sum == kSumNone || sum == kSumLast;
            out->push_back({q, I0 / 64, sum, packs && g0 != 0, 0});
        }
    }
    if (s.tail) {
        finish_plan(&b, fields, 1, false);  // maps only: the tail runs no transform
        out->push_back({b, 0, kSumTail, true, (uint32_t)s.tail});
    }
    return true;
}

double blocks_cost_ms(const std::vector<Block> &bl, const Tuning *tune) {
    double c = 0;
    for (const Block &b : bl) {
        if (b.sum == kSumTail) {
            c += tail_cost(b.p.m);
            continue;
        }
        const double t = b.sum == kSumNone ? alone_cost(b.p.field, b.p.lg, tune) : plan_cost(b.p.field, b.p.lg, tune);
        c += (b.sum == kSumFirst || b.sum == kSumInner) ? kSumShare * t : t;
        if (b.xor_into) c += kXorMs;
    }
    return c;
}

static BitMap bitmap(const uint64_t *src, int mode, uint64_t len, uint64_t srclen, uint64_t off) {
    BitMap b;
    b.src = src;
    b.mode = mode;
    b.len = len;
    b.srclen = srclen;
    b.off = off;
    return b;
}

static cm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CM_OK;
    if (e == cudaErrorMemoryAllocation) return CM_ENOMEM;
    return CM_EDEVICE;
}

// Whether the one-launch cluster kernel for 2^lg runs on this context's device
// (attributes set and the cluster size checked on first use).
static bool cluster25_ready(cm_ctx *ctx, int lg) {
    std::atomic<int> &st = ctx->cluster25[lg - kClusterMinLg];
    int v = st.load(std::memory_order_acquire);
    if (v < 0) {
        bool fits = false;
        if (cluster25_prepare(lg, &fits) != cudaSuccess) {
            cudaGetLastError();
            fits = false;
        }
        v = fits ? 1 : 0;
        st.store(v, std::memory_order_release);
    }
    return v == 1;
}

// Enqueue the product of plan p (no precondition check; pre: the Dodis et al.
// flags the pack kernel reads, or null).  scratch holds p.scratch_bytes; sum
// (SumMode) says whether the product stands alone or joins its window's sum.
static cm_status enqueue_product(cm_ctx *ctx, const Plan &p, const uint64_t *x, const uint64_t *y,
                                 uint64_t *z, void *scratch, const uint32_t *pre, int sum, cudaStream_t st,
                                 const TailArgs *tail = nullptr) {
    const BitMap am = bitmap(x, p.amode, p.alen, p.asrclen, p.aoff);
    const BitMap bm = bitmap(y, p.bmode, p.blen, p.bsrclen, p.boff);
    const bool f30 = p.field == kFieldF30, f25 = p.field == kFieldF25;
    const uint64_t linv = f25 ? f25_linv_shoup(p.L) : f30 ? f30_linv_mont2(p.L) : gl_inv_pow2_host(p.L);
    const size_t esz = p.field == kFieldGL ? sizeof(uint64_t) : sizeof(uint32_t);
    // kernel names for the trace: Goldilocks, F30 or F25 forms
    auto kname = [&](const char *gl, const char *k30, const char *k25) { return f25 ? k25 : f30 ? k30 : gl; };
    cudaError_t e;
    uint8_t *sc = static_cast<uint8_t *>(scratch);
    if (p.cluster && sum == kSumNone && cluster25_ready(ctx, p.lg)) {
        Launch q;
        q.amap = am;
        q.bmap = bm;
        q.lo = p.lo;
        q.m = p.m;
        q.linv = linv;
        q.z = z;
        q.pre = pre;
        q.status = ctx->d_status;
        q.field = p.field;
        q.rt = ctx->rt;
        q.rt30 = ctx->rt30;
        q.rt25 = ctx->rt25;
        q.stream = st;
        ProfScope ps(ctx, "k_cluster_f25", st);
        return cuda_status(launch_cluster25(q, p.lg));
    }
    if (p.npass == 0) {
        Launch q;
        q.amap = am;
        q.bmap = bm;
        q.lo = p.lo;
        q.m = p.m;
        q.linv = linv;
        q.z = z;
        q.pre = pre;
        q.status = ctx->d_status;
        q.field = p.field;
        q.rt = ctx->rt;
        q.rt30 = ctx->rt30;
        q.rt25 = ctx->rt25;
        q.stream = st;
        ProfScope ps(ctx, kname("k_fused_small", "k_fused_small_f30", "k_fused_small_f25"), st);
        return cuda_status(launch_small(q, p.lg));
    }
    void *A = sc;
    void *B = sc + esz * p.L;
    void *C = sum == kSumNone ? nullptr : sc + 2 * esz * p.L;
    uint8_t *par = sc + (sum == kSumNone ? 2 : 3) * esz * p.L;

    int lgN[2], lgS[2];
    int cur = p.lg;
    for (int j = 0; j < p.npass; ++j) {
        lgN[j] = cur;
        lgS[j] = cur - p.pass_lg[j];
        cur = lgS[j];
    }
    // forward passes, both operands in each launch
    for (int j = 0; j < p.npass; ++j) {
        {
            PassArgs a;
            memset(&a, 0, sizeof(a));
            a.data = A;
            a.map = am;
            a.data2 = B;
            a.map2 = bm;
            a.lgN = lgN[j];
            a.lgS = lgS[j];
            a.field = p.field;
            a.rt = ctx->rt;
            a.rt30 = ctx->rt30;
            a.rt25 = ctx->rt25;
            a.L = p.L;
            a.inv = false;
            a.bits_in = (j == 0);
            ProfScope ps(ctx, j == 0 ? kname("k_pass_fwd_bits", "k_pass_fwd_bits_f30", "k_pass_fwd_bits_f25")
                                     : kname("k_pass_fwd", "k_pass_fwd_f30", "k_pass_fwd_f25"), st);
            if ((e = launch_pass(a, p.pass_lg[j], st)) != cudaSuccess) return cuda_status(e);
        }
    }
    {
        ProfScope ps(ctx, kname("k_middle", "k_middle_f30", "k_middle_f25"), st);
        const int mode = sum == kSumFirst ? kMidFirst : sum == kSumInner ? kMidInner
                         : sum == kSumLast ? kMidLast : kMidAlone;
        e = launch_middle(p.field, A, B, C, mode, p.L, linv, ctx->rt, ctx->rt30, ctx->rt25, ctx->nsm, st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (sum == kSumFirst || sum == kSumInner) return CM_OK;  // the group's last block finishes
    void *R = A;
    for (int j = p.npass - 1; j >= 0; --j) {
        PassArgs a;
        memset(&a, 0, sizeof(a));
        a.data = R;
        a.lgN = lgN[j];
        a.lgS = lgS[j];
        a.field = p.field;
        a.rt = ctx->rt;
        a.rt30 = ctx->rt30;
        a.rt25 = ctx->rt25;
        a.L = p.L;
        a.inv = true;
        a.parity_out = (j == 0);
        a.par = par;
        a.lo = p.lo;
        a.m = p.m;
        ProfScope ps(ctx, j == 0 ? kname("k_pass_inv_parity", "k_pass_inv_parity_f30", "k_pass_inv_parity_f25")
                                 : kname("k_pass_inv", "k_pass_inv_f30", "k_pass_inv_f25"), st);
        if ((e = launch_pass(a, p.pass_lg[j], st)) != cudaSuccess) return cuda_status(e);
    }
    if (tail) {  // the extraction's dense tail joins the pack of its only window
        ProfScope ps(ctx, "k_pack_tail", st);
        return cuda_status(launch_pack_tail(par, p.m, z, pre, ctx->d_status, *tail, ctx->nsm, st));
    }
    ProfScope ps(ctx, "k_pack", st);
    return cuda_status(launch_pack(par, p.m, z, pre, ctx->d_status, ctx->nsm, st));
}

// Dodis et al. precondition flags at pre (two words, reset first).
static cm_status enqueue_precondition(cm_ctx *ctx, const uint64_t *x, uint64_t n, uint32_t *pre, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(pre, 0, 2 * sizeof(uint32_t), st)) != cudaSuccess) return cuda_status(e);
    ProfScope ps(ctx, "k_allsame", st);
    return cuda_status(launch_allsame(x, n, pre, ctx->nsm, st));
}

// Enqueue one single-transform extraction described by plan p.  scratch holds
// p.scratch_bytes (the Dodis et al. flags in its last 256 bytes).
cm_status enqueue_extract(cm_ctx *ctx, const Plan &p, const uint64_t *x, const uint64_t *y,
                          uint64_t *z, void *scratch, cudaStream_t st) {
    uint32_t *pre = nullptr;
    if (p.kind == CM_DODIS) {
        pre = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(scratch) + p.scratch_bytes - 256);
        cm_status s = enqueue_precondition(ctx, x, p.n, pre, st);
        if (s != CM_OK) return s;
    }
    return enqueue_product(ctx, p, x, y, z, scratch, pre, kSumNone, st);
}

// Scratch of a blocked run: the largest block's scratch; then (one-CTA windows
// whose blocks XOR) one output window of temporary at *tmp_off; then 256 bytes
// of precondition flags at *pre_off.
uint64_t blocks_scratch(const std::vector<Block> &bl, uint64_t *tmp_off, uint64_t *pre_off) {
    uint64_t sc = 0, tmpw = 0;
    for (const Block &b : bl) {
        if (b.sum == kSumTail) continue;  // no scratch; XORs straight into z
        const uint64_t own = b.p.scratch_bytes - flag_bytes(b.p.kind);  // flags are shared
        if (own > sc) sc = own;
        if (b.xor_into && words_of(b.p.m) > tmpw) tmpw = words_of(b.p.m);
    }
    *tmp_off = (sc + 255) & ~255ull;
    *pre_off = (*tmp_off + 8 * tmpw + 255) & ~255ull;
    const bool dodis = !bl.empty() && bl[0].p.kind == CM_DODIS;
    if (!dodis && !tmpw) return sc;
    return dodis ? *pre_off + kFlagBytes : *tmp_off + 8 * tmpw;
}

// Index of the product whose pack also applies the dense tail: the last
// product, when the list ends in a tail, every product writes the one window
// in place (word 0, no XOR temporary) and the last one packs through the
// column-pass form; else -1.
static int tail_fold(const std::vector<Block> &bl) {
    if (bl.size() < 2 || bl.back().sum != kSumTail) return -1;
    for (size_t i = 0; i + 1 < bl.size(); ++i)
        if (bl[i].zword != 0 || bl[i].xor_into) return -1;
    const Block &last = bl[bl.size() - 2];
    if (last.sum != kSumNone && last.sum != kSumLast) return -1;
    if (last.p.npass == 0 || (last.p.cluster && last.sum == kSumNone)) return -1;  // packs on chip
    return (int)bl.size() - 2;
}

// Enqueue every block of an extraction; scratch holds blocks_scratch() bytes.
cm_status enqueue_blocks(cm_ctx *ctx, const std::vector<Block> &bl, const uint64_t *x, const uint64_t *y,
                         uint64_t *z, uint8_t *scratch, uint64_t tmp_off, uint64_t pre_off, cudaStream_t st) {
    uint32_t *pre = nullptr;
    if (!bl.empty() && bl[0].p.kind == CM_DODIS) {
        pre = reinterpret_cast<uint32_t *>(scratch + pre_off);
        cm_status s = enqueue_precondition(ctx, x, bl[0].p.n, pre, st);
        if (s != CM_OK) return s;
    }
    // A dense tail folds into the pack of the last product when the extraction
    // has one output window written in place and that product runs the
    // column-pass form (its pack is a separate launch).
    const int fold = tail_fold(bl);
    TailArgs ta{};
    if (fold >= 0) {
        const Plan &tp = bl.back().p;
        ta.amap = bitmap(x, tp.amode, tp.alen, tp.asrclen, tp.aoff);
        ta.bmap = bitmap(y, tp.bmode, tp.blen, tp.bsrclen, tp.boff);
        ta.K = tp.K;
        ta.T = bl.back().tail;
    }
    for (size_t i = 0; i < bl.size(); ++i) {
        const Block &b = bl[i];
        if (b.sum == kSumTail) {
            if (fold >= 0) continue;  // done by the pack
            const Plan &p = b.p;
            ProfScope ps(ctx, "k_tail", st);
            if (launch_tail(bitmap(x, p.amode, p.alen, p.asrclen, p.aoff), bitmap(y, p.bmode, p.blen, p.bsrclen, p.boff),
                            p.K, b.tail, p.m, z, pre, ctx->nsm, st) != cudaSuccess)
                return CM_EDEVICE;
            continue;
        }
        uint64_t *dst = b.xor_into ? reinterpret_cast<uint64_t *>(scratch + tmp_off) : z + b.zword;
        cm_status s = enqueue_product(ctx, b.p, x, y, dst, b.p.scratch_bytes ? scratch : nullptr, pre, b.sum, st,
                                      (int)i == fold ? &ta : nullptr);
        if (s != CM_OK) return s;
        if (b.xor_into) {
            ProfScope ps(ctx, "k_xor_into", st);
            if (launch_xor_into(z + b.zword, dst, words_of(b.p.m), ctx->nsm, st) != cudaSuccess)
                return CM_EDEVICE;
        }
    }
    return CM_OK;
}

cm_status run_single(cm_ctx *ctx, int kind, const uint64_t *x, uint64_t n, const uint64_t *y,
                     uint64_t m, uint64_t *z, cudaStream_t st) {
    if (!ctx || !x || !y || !z) return CM_EINVAL;
    std::vector<Block> bl;
    if (!make_blocks(kind, n, m, ctx->popt, &bl)) return CM_EINVAL;
    uint64_t tmp_off = 0, pre_off = 0;
    const uint64_t need = blocks_scratch(bl, &tmp_off, &pre_off);
    if (need > ctx->budget) return CM_ENOMEM;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return CM_EDEVICE;
    void *scratch = nullptr;
    if (need) {
        e = cudaMallocFromPoolAsync(&scratch, need, ctx->pool, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return CM_ENOMEM;
        }
    }
    cm_status s = enqueue_blocks(ctx, bl, x, y, z, static_cast<uint8_t *>(scratch), tmp_off, pre_off, st);
    if (scratch) {
        e = cudaFreeAsync(scratch, st);
        if (s == CM_OK && e != cudaSuccess) s = CM_EDEVICE;
    }
    return s;
}

static cudaEvent_t get_event(cm_ctx *c) {
    cudaEvent_t ev = nullptr;
    if (!c->ev_pool.empty()) {
        ev = c->ev_pool.back();
        c->ev_pool.pop_back();
    } else if (cudaEventCreate(&ev) != cudaSuccess) {
        return nullptr;
    }
    return ev;
}

ProfScope::ProfScope(cm_ctx *c_, const char *name_, cudaStream_t st_) : c(c_), name(name_), st(st_) {
    if (!c->prof_on) return;
    std::lock_guard<std::mutex> g(c->prof_mu);
    a = get_event(c);
    if (a) cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
    if (!a) return;
    std::lock_guard<std::mutex> g(c->prof_mu);
    cudaEvent_t b = get_event(c);
    if (!b) return;
    cudaEventRecord(b, st);
    c->prof_pending.push_back({name, a, b});
}

static void build_tables(std::vector<uint64_t> &h) {
    // layout: small[8192] = omega_8192^e; big_lo_fwd[65536] = g^e;
    //         big_hi_fwd[65536] = g^(65536 e); big_lo_inv, big_hi_inv likewise for g^-1
    h.assign(kTableWords, 0);
    const uint64_t g = gl_root_2_32_host(0), gi = gl_root_2_32_host(1);
    const uint64_t w = gl_pow_host(g, 1ull << (32 - kSmallLg));  // omega_8192
    uint64_t a = 1;
    for (int e = 0; e < 8192; ++e) {
        h[e] = a;
        a = gl_mul_host(a, w);
    }
    uint64_t *lf = &h[8192], *hf = lf + 65536, *li = hf + 65536, *hi = li + 65536;
    const uint64_t g16 = gl_pow_host(g, 65536), gi16 = gl_pow_host(gi, 65536);
    uint64_t c0 = 1, c1 = 1, c2 = 1, c3 = 1;
    for (int e = 0; e < 65536; ++e) {
        lf[e] = c0;
        hf[e] = c1;
        li[e] = c2;
        hi[e] = c3;
        c0 = gl_mul_host(c0, g);
        c1 = gl_mul_host(c1, g16);
        c2 = gl_mul_host(c2, gi);
        c3 = gl_mul_host(c3, gi16);
    }
}

// F30 root tables, entries in Montgomery form w R mod q: small[8192] =
// omega_8192^e; big_lo_fwd[32768] = g30^e; big_hi_fwd[32768] = g30^(32768 e);
// big_lo_inv, big_hi_inv likewise for g30^-1.
static void build_tables30(std::vector<uint32_t> &h) {
    h.assign(kTable30Words, 0);
    const uint32_t g = f30_root_2_30(false), gi = f30_root_2_30(true);
    const uint32_t w = f30_pow(g, 1ull << (kF30MaxLg - kSmallLg));  // omega_8192
    uint32_t a = 1;
    for (int e = 0; e < 8192; ++e) {
        h[e] = f30_to_mont(a);
        a = f30_mulmod(a, w);
    }
    uint32_t *lf = &h[8192], *hf = lf + 32768, *li = hf + 32768, *hi = li + 32768;
    const uint32_t g15 = f30_pow(g, 32768), gi15 = f30_pow(gi, 32768);
    uint32_t c0 = 1, c1 = 1, c2 = 1, c3 = 1;
    for (int e = 0; e < 32768; ++e) {
        lf[e] = f30_to_mont(c0);
        hf[e] = f30_to_mont(c1);
        li[e] = f30_to_mont(c2);
        hi[e] = f30_to_mont(c3);
        c0 = f30_mulmod(c0, g);
        c1 = f30_mulmod(c1, g15);
        c2 = f30_mulmod(c2, gi);
        c3 = f30_mulmod(c3, gi15);
    }
    // bits16[k * 256 + p] = sum over the set bits j of p of w^(j k), w = omega_16
    // (the root the on-chip radix-16 DFT uses: g30^(2^26))
    uint32_t *b16 = hi + 32768;
    const uint32_t w16 = f30_pow(F30_G30, 1ull << 26);
    for (int k = 0; k < 16; ++k)
        for (int p = 0; p < 256; ++p) {
            uint64_t acc = 0;
            for (int j = 0; j < 8; ++j)
                if ((p >> j) & 1) acc += f30_pow(w16, (uint64_t)((j * k) & 15));
            b16[k * 256 + p] = (uint32_t)(acc % F30_Q);
        }
}

// F25 root tables, entries in Montgomery form w 2^32 mod q: small[8192] =
// omega_8192^e; big_lo_fwd[8192] = g25^e; big_hi_fwd[4096] = g25^(8192 e);
// big_lo_inv, big_hi_inv likewise for g25^-1; then the bit DFT table (plain,
// canonical) of the radix-16 root omega_16 = g25^(2^21).
static void build_tables25(std::vector<uint32_t> &h) {
    h.assign(kTable25Words, 0);
    const uint32_t g = f25_root_2_25(false), gi = f25_root_2_25(true);
    const uint32_t w = f25_pow(g, 1ull << (kF25MaxLg - kSmallLg));  // omega_8192
    uint32_t a = 1;
    for (int e = 0; e < 8192; ++e) {
        h[e] = f25_to_mont(a);
        a = f25_mulmod(a, w);
    }
    uint32_t *lf = &h[8192], *hf = lf + 8192, *li = hf + 4096, *hi = li + 8192;
    const uint32_t g13 = f25_pow(g, 8192), gi13 = f25_pow(gi, 8192);
    uint32_t c0 = 1, c1 = 1, c2 = 1, c3 = 1;
    for (int e = 0; e < 8192; ++e) {
        lf[e] = f25_to_mont(c0);
        li[e] = f25_to_mont(c2);
        c0 = f25_mulmod(c0, g);
        c2 = f25_mulmod(c2, gi);
        if (e < 4096) {
            hf[e] = f25_to_mont(c1);
            hi[e] = f25_to_mont(c3);
            c1 = f25_mulmod(c1, g13);
            c3 = f25_mulmod(c3, gi13);
        }
    }
    uint32_t *b16 = hi + 4096;
    const uint32_t w16 = f25_pow(F25_G25, 1ull << 21);
    for (int k = 0; k < 16; ++k)
        for (int p = 0; p < 256; ++p) {
            uint64_t acc = 0;
            for (int j = 0; j < 8; ++j)
                if ((p >> j) & 1) acc += f25_pow(w16, (uint64_t)((j * k) & 15));
            b16[k * 256 + p] = (uint32_t)(acc % F25_Q);
        }
    // per-step tables (ntt25.cuh): length 2^l at pair 2^l, step J's roots
    // omega_(N_J)^(i2 k1) at pair [(k1 - 1) M_J + i2] as (root, Shoup quotient)
    uint32_t *steps = b16 + 4096;
    for (int l = 1; l <= kSmallLg; ++l)
        for (int j = 0; j + 1 < st_n(l); ++j) {
            const int lq = st_q(l, j), rd = 1 << lq, lnj = l - st_off(l, j), mj = 1 << (lnj - lq);
            const uint32_t wn = f25_pow(F25_G25, 1ull << (kF25MaxLg - lnj));  // omega_(N_J)
            uint32_t *t = steps + 2 * ((1 << l) + st25_tab_off(l, j));
            for (int k1 = 1; k1 < rd; ++k1)
                for (int i2 = 0; i2 < mj; ++i2) {
                    const uint32_t w = f25_pow(wn, (uint64_t)i2 * k1);
                    t[2 * ((k1 - 1) * mj + i2)] = w;
                    t[2 * ((k1 - 1) * mj + i2) + 1] = f25_shoup_q(w);
                }
        }
}

}  // namespace cm

using namespace cm;

extern "C" cm_status cm_create(cm_ctx **out, int device, const cm_options *opt) {
    if (!out) return CM_EINVAL;
    *out = nullptr;
    PlanOptions po;
    if (!plan_options(opt, &po)) return CM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return CM_EDEVICE;
    cm_ctx *c = new cm_ctx();
    c->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return CM_EDEVICE;
    }
    c->nsm = prop.multiProcessorCount;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    c->budget = (opt && opt->hbm_budget_bytes) ? opt->hbm_budget_bytes : (uint64_t)(free_b * 0.8);
    c->popt = po;
    c->popt.budget = c->budget;

    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof(pp));
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &pp) != cudaSuccess) {
        delete c;
        return CM_EDEVICE;
    }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);

    std::vector<uint64_t> h;
    build_tables(h);
    std::vector<uint32_t> h30, h25;
    build_tables30(h30);
    build_tables25(h25);
    if (cudaMalloc(&c->d_tables, h.size() * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&c->d_tables30, h30.size() * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_tables25, h25.size() * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_status, 64) != cudaSuccess) {
        cm_destroy(c);
        return CM_ENOMEM;
    }
    cudaMemcpy(c->d_tables, h.data(), h.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_tables30, h30.data(), h30.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_tables25, h25.data(), h25.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    c->rt25.small = c->d_tables25;
    c->rt25.big_lo_fwd = c->d_tables25 + 8192;
    c->rt25.big_hi_fwd = c->rt25.big_lo_fwd + 8192;
    c->rt25.big_lo_inv = c->rt25.big_hi_fwd + 4096;
    c->rt25.big_hi_inv = c->rt25.big_lo_inv + 8192;
    c->rt25.bits16 = c->rt25.big_hi_inv + 4096;
    c->rt25.steps = c->rt25.bits16 + 4096;
    c->rt30.small = c->d_tables30;
    c->rt30.big_lo_fwd = c->d_tables30 + 8192;
    c->rt30.big_hi_fwd = c->rt30.big_lo_fwd + 32768;
    c->rt30.big_lo_inv = c->rt30.big_hi_fwd + 32768;
    c->rt30.big_hi_inv = c->rt30.big_lo_inv + 32768;
    c->rt30.bits16 = c->rt30.big_hi_inv + 32768;
    cudaMemset(c->d_status, 0, 64);
    c->rt.small = c->d_tables;
    c->rt.big_lo_fwd = c->d_tables + 8192;
    c->rt.big_hi_fwd = c->rt.big_lo_fwd + 65536;
    c->rt.big_lo_inv = c->rt.big_hi_fwd + 65536;
    c->rt.big_hi_inv = c->rt.big_lo_inv + 65536;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cm_destroy(c);
        return CM_EDEVICE;
    }
    *out = c;
    return CM_OK;
}

extern "C" void cm_destroy(cm_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    cm_ctx_release_extras(c);
    for (auto &r : c->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto ev : c->ev_pool) cudaEventDestroy(ev);
    if (c->d_tables) cudaFree(c->d_tables);
    if (c->d_tables30) cudaFree(c->d_tables30);
    if (c->d_tables25) cudaFree(c->d_tables25);
    if (c->d_status) cudaFree(c->d_status);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    delete c;
}

extern "C" const char *cm_status_str(int s) {
    switch (s) {
        case CM_OK: return "CM_OK";
        case CM_EINVAL: return "CM_EINVAL: invalid argument";
        case CM_EPRECOND: return "CM_EPRECOND: Dodis et al. input is all-0 or all-1";
        case CM_ENOMEM: return "CM_ENOMEM: out of memory or over the HBM budget";
        case CM_EAGAIN: return "CM_EAGAIN: not ready";
        case CM_ETIMEDOUT: return "CM_ETIMEDOUT: bounded wait ran out";
        case CM_EDEVICE: return "CM_EDEVICE: CUDA error";
        case CM_ENOTFOUND: return "CM_ENOTFOUND: unknown ticket";
        default: return "unknown cm_status";
    }
}

extern "C" cm_status cm_toeplitz(cm_ctx *ctx, const uint64_t *x, uint64_t n, const uint64_t *y,
                                 uint64_t m, uint64_t *z, cm_stream stream) {
    return run_single(ctx, CM_TOEPLITZ, x, n, y, m, z, static_cast<cudaStream_t>(stream));
}

extern "C" cm_status cm_circulant(cm_ctx *ctx, const uint64_t *x, uint64_t n, const uint64_t *y,
                                  uint64_t m, uint64_t *z, cm_stream stream) {
    return run_single(ctx, CM_CIRCULANT, x, n, y, m, z, static_cast<cudaStream_t>(stream));
}

extern "C" cm_status cm_dodis(cm_ctx *ctx, const uint64_t *x, const uint64_t *y, uint64_t n,
                              uint64_t m, uint64_t *z, cm_stream stream) {
    return run_single(ctx, CM_DODIS, x, n, y, m, z, static_cast<cudaStream_t>(stream));
}

extern "C" cm_status cm_device_status(cm_ctx *ctx, cm_stream stream, uint32_t *flags) {
    if (!ctx) return CM_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return CM_EDEVICE;
    uint32_t f = 0;
    if (cudaMemcpy(&f, ctx->d_status, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess) return CM_EDEVICE;
    if (cudaMemset(ctx->d_status, 0, sizeof(f)) != cudaSuccess) return CM_EDEVICE;
    if (flags) *flags = f;
    if (f & CM_FLAG_PRECOND) return CM_EPRECOND;
    if (f & CM_FLAG_TIMEOUT) return CM_ETIMEDOUT;
    return CM_OK;
}

static uint32_t blocks_launches(const std::vector<Block> &bl) {
    uint32_t c = (!bl.empty() && bl[0].p.kind == CM_DODIS) ? 1 : 0;  // precondition, once
    const bool folded = tail_fold(bl) >= 0;
    for (const Block &b : bl) {
        const Plan &p = b.p;
        if (b.sum == kSumTail) c += folded ? 0 : 1;
        else if (p.npass == 0 || (p.cluster && b.sum == kSumNone)) c += 1;  // on chip or on a cluster
        else if (b.sum == kSumFirst || b.sum == kSumInner) c += p.npass + 1;  // forward + middle
        else c += p.npass + 1 + p.npass + 1;                                   // + inverse + pack
        if (b.xor_into && b.sum != kSumTail) c += 1;
    }
    return c;
}

// The plan of (kind, n, m) under opt (NULL: defaults); false if invalid.
static bool query(int kind, uint64_t n, uint64_t m, const cm_options *opt, cm_plan_info *info) {
    memset(info, 0, sizeof(*info));
    PlanOptions o;
    std::vector<Block> bl;
    if (!plan_options(opt, &o) || !make_blocks(kind, n, m, o, &bl)) return false;
    uint64_t tmp_off = 0, pre_off = 0;
    info->scratch_bytes = blocks_scratch(bl, &tmp_off, &pre_off);
    info->products = bl.size() - (bl.back().sum == kSumTail ? 1 : 0);
    info->launches = blocks_launches(bl);
    info->field = CM_FIELD_Q25;  // the widest field of any product
    for (size_t i = 0; i < bl.size(); ++i) {
        const Block &b = bl[i];
        if (b.sum == kSumTail) {
            info->tail_terms = b.tail;
            continue;
        }
        if (b.p.L > info->transform_length) info->transform_length = b.p.L;
        if (b.p.field == kFieldGL) info->field = CM_FIELD_GOLDILOCKS;
        else if (b.p.field == kFieldF30 && info->field == CM_FIELD_Q25) info->field = CM_FIELD_Q30;
        if (i == 0 || b.zword != bl[i - 1].zword) ++info->windows;  // blocks come window by window
    }
    info->est_ms = blocks_cost_ms(bl);
    return true;
}

extern "C" cm_status cm_plan_query(int kind, uint64_t n, uint64_t m, const cm_options *opt, cm_plan_info *out) {
    if (!out) return CM_EINVAL;
    return query(kind, n, m, opt, out) ? CM_OK : CM_EINVAL;
}

extern "C" cm_status cm_plan_products(int kind, uint64_t n, uint64_t m, const cm_options *opt,
                                      cm_product_desc *out, uint64_t cap, uint64_t *count) {
    PlanOptions o;
    std::vector<Block> bl;
    if (!count || (cap && !out) || !plan_options(opt, &o) || !make_blocks(kind, n, m, o, &bl)) return CM_EINVAL;
    *count = bl.size();
    for (uint64_t i = 0; i < bl.size() && i < cap; ++i) {
        const Block &b = bl[i];
        cm_product_desc &d = out[i];
        memset(&d, 0, sizeof(d));
        d.K = b.p.K;
        d.m = b.p.m;
        d.L = b.p.L;
        d.zword = b.zword;
        d.a_len = b.p.alen;
        d.a_srclen = b.p.asrclen;
        d.a_off = b.p.aoff;
        d.b_len = b.p.blen;
        d.b_srclen = b.p.bsrclen;
        d.b_off = b.p.boff;
        d.a_mode = (uint32_t)b.p.amode;
        d.b_mode = (uint32_t)b.p.bmode;
        d.field = b.p.field == kFieldF25 ? CM_FIELD_Q25 : b.p.field == kFieldF30 ? CM_FIELD_Q30 : CM_FIELD_GOLDILOCKS;
        d.sum = b.sum;
        d.xor_into = b.xor_into ? 1u : 0u;
        d.tail_terms = b.tail;
        if (b.sum == kSumTail) d.L = 0;
    }
    return CM_OK;
}

extern "C" uint64_t cm_ntt_length(int kind, uint64_t n, uint64_t m) {
    cm_plan_info i;
    return query(kind, n, m, nullptr, &i) ? i.transform_length : 0;
}

extern "C" uint64_t cm_scratch_bytes(int kind, uint64_t n, uint64_t m) {
    cm_plan_info i;
    return query(kind, n, m, nullptr, &i) ? i.scratch_bytes : 0;
}

extern "C" uint32_t cm_launch_count(int kind, uint64_t n, uint64_t m) {
    cm_plan_info i;
    return query(kind, n, m, nullptr, &i) ? i.launches : 0;
}

extern "C" uint64_t cm_block_count(int kind, uint64_t n, uint64_t m, uint32_t max_transform_lg) {
    cm_options o;
    memset(&o, 0, sizeof(o));
    o.max_transform_lg = max_transform_lg;
    cm_plan_info i;
    return query(kind, n, m, &o, &i) ? i.products : 0;
}

extern "C" cm_status cm_profile_enable(cm_ctx *ctx, int on) {
    if (!ctx) return CM_EINVAL;
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    ctx->prof_on = on != 0;
    return CM_OK;
}

extern "C" cm_status cm_profile_read(cm_ctx *ctx, cm_profile_entry *out, uint32_t cap,
                                     uint32_t *count, int reset) {
    if (!ctx) return CM_EINVAL;
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    cm_status st = CM_OK;
    for (auto &r : ctx->prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
            st = CM_EDEVICE;
        auto &acc = ctx->prof_acc[r.name];
        acc.first += 1;
        acc.second += ms;
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    uint32_t k = 0;
    for (auto &kv : ctx->prof_acc) {
        if (out && k < cap) {
            memset(out[k].name, 0, sizeof(out[k].name));
            strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
            out[k].launches = kv.second.first;
            out[k].total_ms = kv.second.second;
        }
        ++k;
    }
    if (count) *count = k;
    if (reset) ctx->prof_acc.clear();
    return st;
}

extern "C" cm_status cm_extract_host(cm_ctx *ctx, int kind, const uint64_t *xh, uint64_t n,
                                     const uint64_t *yh, uint64_t m, uint64_t *zh, cm_stream stream) {
    if (!ctx || !xh || !yh || !zh) return CM_EINVAL;
    std::vector<Block> bl;
    if (!make_blocks(kind, n, m, ctx->popt, &bl)) return CM_EINVAL;
    uint64_t tmp_off = 0, pre_off = 0;
    const uint64_t sb = blocks_scratch(bl, &tmp_off, &pre_off);
    const uint64_t sbr = (sb + 255) & ~255ull;
    const uint64_t ybits = kind == CM_TOEPLITZ ? n + m - 1 : (kind == CM_CIRCULANT ? n + 1 : n);
    const uint64_t xw = words_of(n), yw = words_of(ybits), zw = words_of(m);
    const uint64_t io = 8 * (xw + yw + zw) + 3 * 256;
    if (sbr + io > ctx->budget) return CM_ENOMEM;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *buf = nullptr;
    if (cudaMallocFromPoolAsync(&buf, sbr + io, ctx->pool, st) != cudaSuccess) {
        cudaGetLastError();
        return CM_ENOMEM;
    }
    uint8_t *b = static_cast<uint8_t *>(buf);
    uint64_t *xd = reinterpret_cast<uint64_t *>(b + sbr);
    uint64_t *yd = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(xd) + ((8 * xw + 255) & ~255ull));
    uint64_t *zd = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(yd) + ((8 * yw + 255) & ~255ull));
    cm_status s = CM_OK;
    if (cudaMemcpyAsync(xd, xh, 8 * xw, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(yd, yh, 8 * yw, cudaMemcpyHostToDevice, st) != cudaSuccess)
        s = CM_EDEVICE;
    uint32_t pre_h[2] = {1, 1};
    if (s == CM_OK) s = enqueue_blocks(ctx, bl, xd, yd, zd, b, tmp_off, pre_off, st);
    if (s == CM_OK && cudaMemcpyAsync(zh, zd, 8 * zw, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = CM_EDEVICE;
    if (s == CM_OK && kind == CM_DODIS &&
        cudaMemcpyAsync(pre_h, b + pre_off, sizeof(pre_h), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = CM_EDEVICE;
    cudaFreeAsync(buf, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CM_EDEVICE;
    if (s == CM_OK && kind == CM_DODIS && (pre_h[0] == 0 || pre_h[1] == 0)) s = CM_EPRECOND;
    return s;
}
