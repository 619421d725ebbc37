// C ABI entry points: context, plans, single extractions.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "cm.h"
#include "cm_internal.h"
#include "cm_ctx.h"

namespace cm {

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

// Transform length, pass split, scratch and launch count for K + m - 1 <= 2^32.
static void finish_plan(Plan *p) {
    const uint64_t need = p->K + p->m - 1;
    p->lg = ceil_log2(need);
    if (p->lg < 1) p->lg = 1;
    p->L = 1ull << p->lg;
    p->lo = p->K - 1;
    const int rest = p->lg - kMidLgMax;
    if (rest <= 0) {
        p->npass = 0;
    } else if (rest <= 12) {
        p->npass = 1;
        p->pass_lg[0] = rest;
    } else {
        p->npass = 2;
        p->pass_lg[0] = (rest + 1) / 2;
        p->pass_lg[1] = rest / 2;
    }
    const uint64_t flags = (p->kind == CM_DODIS) ? 256 : 0;
    if (p->npass == 0) {
        p->scratch_bytes = flags;
        p->launches = 1;
    } else {
        p->scratch_bytes = 2 * 8 * p->L + ((p->m + 255) & ~255ull) + flags;
        // forward passes of both operands, middle, inverse passes, pack
        p->launches = 2 * p->npass + 1 + p->npass + 1;
    }
    if (p->kind == CM_DODIS) p->launches += 1;  // precondition check
}

bool make_plan(int kind, uint64_t n, uint64_t m, Plan *p, bool allow_f30) {
    if (!base_maps(kind, n, m, p)) return false;
    if (p->K + m - 1 > (1ull << 32)) return false;
    finish_plan(p);
    if (allow_f30 && p->lg <= kF30MaxLg) p->field = kFieldF30;
    return true;
}

// z_i = sum_{t<K} a_t b_{t+i} splits over input blocks t in [T0, T0 + kb)
// (each a middle product of a[T0 .. T0 + kb) with b[T0 .. T0 + kb + m - 1),
// the results XORed: parity of a sum is the XOR of the parities) and over
// output blocks i in [I0, I0 + mb) (b shifted by I0).  In transform positions
// u = K - 1 - t, input block [D, D + kb) of A is A shifted by D.
bool make_blocks(int kind, uint64_t n, uint64_t m, int max_lg, bool allow_f30, std::vector<Block> *out) {
    out->clear();
    Plan b;
    if (max_lg < 8 || max_lg > 32 || !base_maps(kind, n, m, &b)) return false;
    const uint64_t Lmax = 1ull << max_lg;
    if (b.K + m - 1 <= Lmax) {
        finish_plan(&b);
        if (allow_f30 && b.lg <= kF30MaxLg) b.field = kFieldF30;
        out->push_back({b, 0, false});
        return true;
    }
    const uint64_t Mb = m > Lmax / 2 ? Lmax / 2 : m;  // a multiple of 64 when it splits m
    const uint64_t nout = (m + Mb - 1) / Mb;
    const uint64_t kmax = Lmax - Mb + 1;
    const uint64_t nin = (b.K + kmax - 1) / kmax;
    if (nin * nout > kMaxBlocks) return false;
    const uint64_t Kb = (b.K + nin - 1) / nin;
    for (uint64_t r = 0; r < nout; ++r) {
        const uint64_t I0 = r * Mb, mr = (m - I0 < Mb) ? m - I0 : Mb;
        for (uint64_t j = 0; j < nin; ++j) {
            const uint64_t D = j * Kb;
            if (D >= b.K) break;
            const uint64_t kb = (b.K - D < Kb) ? b.K - D : Kb;
            const uint64_t T0 = b.K - D - kb;
            Plan q = b;
            q.m = mr;
            q.K = kb;
            if (b.amode == kIdentity) {  // A'_u = x_{D+u}: no wrap, u + D < K = srclen
                q.amode = kModForward;
                q.aoff = D;
            } else {  // A'_u = src[aoff - D - u]
                q.aoff = b.aoff - D;
            }
            q.alen = kb;
            q.blen = kb + mr - 1;
            q.boff = (b.boff + T0 + I0) % b.bsrclen;
            finish_plan(&q);
            if (allow_f30 && q.lg <= kF30MaxLg) q.field = kFieldF30;
            out->push_back({q, I0 / 64, j != 0});
        }
    }
    return true;
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

// Enqueue one extraction described by plan p.  scratch holds p.scratch_bytes.
cm_status enqueue_extract(cm_ctx *ctx, const Plan &p, const uint64_t *x, const uint64_t *y,
                          uint64_t *z, void *scratch, cudaStream_t st) {
    const BitMap am = bitmap(x, p.amode, p.alen, p.asrclen, p.aoff);
    const BitMap bm = bitmap(y, p.bmode, p.blen, p.bsrclen, p.boff);
    const bool f30 = p.field == kFieldF30;
    const uint64_t linv = f30 ? f30_linv_mont2(p.L) : gl_inv_pow2_host(p.L);
    const size_t esz = f30 ? sizeof(uint32_t) : sizeof(uint64_t);
    uint32_t *pre = nullptr;
    cudaError_t e;
    uint8_t *sc = static_cast<uint8_t *>(scratch);
    if (p.kind == CM_DODIS) {
        pre = reinterpret_cast<uint32_t *>(sc + p.scratch_bytes - 256);
        if ((e = cudaMemsetAsync(pre, 0, 2 * sizeof(uint32_t), st)) != cudaSuccess) return cuda_status(e);
        ProfScope ps(ctx, "k_allsame", st);
        if ((e = launch_allsame(x, p.n, pre, ctx->nsm, st)) != cudaSuccess) return cuda_status(e);
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
        q.stream = st;
        ProfScope ps(ctx, f30 ? "k_fused_small_f30" : "k_fused_small", st);
        return cuda_status(launch_small(q, p.lg));
    }
    void *A = sc;
    void *B = sc + esz * p.L;
    uint8_t *par = sc + 2 * esz * p.L;

    int lgN[2], lgS[2];
    int cur = p.lg;
    for (int j = 0; j < p.npass; ++j) {
        lgN[j] = cur;
        lgS[j] = cur - p.pass_lg[j];
        cur = lgS[j];
    }
    // forward passes
    for (int op = 0; op < 2; ++op) {
        for (int j = 0; j < p.npass; ++j) {
            PassArgs a;
            memset(&a, 0, sizeof(a));
            a.data = op == 0 ? A : B;
            a.map = op == 0 ? am : bm;
            a.lgN = lgN[j];
            a.lgS = lgS[j];
            a.field = p.field;
            a.rt = ctx->rt;
            a.rt30 = ctx->rt30;
            a.L = p.L;
            a.inv = false;
            a.bits_in = (j == 0);
            ProfScope ps(ctx, j == 0 ? (f30 ? "k_pass_fwd_bits_f30" : "k_pass_fwd_bits")
                                     : (f30 ? "k_pass_fwd_f30" : "k_pass_fwd"), st);
            if ((e = launch_pass(a, p.pass_lg[j], st)) != cudaSuccess) return cuda_status(e);
        }
    }
    {
        ProfScope ps(ctx, f30 ? "k_middle_f30" : "k_middle", st);
        if ((e = launch_middle(p.field, A, B, p.L, linv, ctx->rt, ctx->rt30, ctx->nsm, st)) != cudaSuccess)
            return cuda_status(e);
    }
    for (int j = p.npass - 1; j >= 0; --j) {
        PassArgs a;
        memset(&a, 0, sizeof(a));
        a.data = A;
        a.lgN = lgN[j];
        a.lgS = lgS[j];
        a.field = p.field;
        a.rt = ctx->rt;
        a.rt30 = ctx->rt30;
        a.L = p.L;
        a.inv = true;
        a.parity_out = (j == 0);
        a.par = par;
        a.lo = p.lo;
        a.m = p.m;
        ProfScope ps(ctx, j == 0 ? (f30 ? "k_pass_inv_parity_f30" : "k_pass_inv_parity")
                                 : (f30 ? "k_pass_inv_f30" : "k_pass_inv"), st);
        if ((e = launch_pass(a, p.pass_lg[j], st)) != cudaSuccess) return cuda_status(e);
    }
    ProfScope ps(ctx, "k_pack", st);
    return cuda_status(launch_pack(par, p.m, z, pre, ctx->d_status, ctx->nsm, st));
}

static uint64_t words_of(uint64_t bits) { return (bits + 63) / 64; }

// Scratch of a blocked run: the largest block's scratch, then (when blocks
// accumulate) one output window of XOR temporary at *tmp_off.
static uint64_t blocks_scratch(const std::vector<Block> &bl, uint64_t *tmp_off) {
    uint64_t sc = 0, tmpw = 0;
    for (const Block &b : bl) {
        if (b.p.scratch_bytes > sc) sc = b.p.scratch_bytes;
        if (b.accumulate && words_of(b.p.m) > tmpw) tmpw = words_of(b.p.m);
    }
    *tmp_off = (sc + 255) & ~255ull;
    return tmpw ? *tmp_off + 8 * tmpw : sc;
}

// Enqueue every block of an extraction; scratch holds blocks_scratch() bytes.
static cm_status enqueue_blocks(cm_ctx *ctx, const std::vector<Block> &bl, const uint64_t *x,
                                const uint64_t *y, uint64_t *z, uint8_t *scratch, uint64_t tmp_off,
                                cudaStream_t st) {
    for (const Block &b : bl) {
        uint64_t *dst = b.accumulate ? reinterpret_cast<uint64_t *>(scratch + tmp_off) : z + b.zword;
        cm_status s = enqueue_extract(ctx, b.p, x, y, dst, b.p.scratch_bytes ? scratch : nullptr, st);
        if (s != CM_OK) return s;
        if (b.accumulate) {
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
    if (!make_blocks(kind, n, m, ctx->max_lg, ctx->allow_f30, &bl)) return CM_EINVAL;
    uint64_t tmp_off = 0;
    const uint64_t need = blocks_scratch(bl, &tmp_off);
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
    cm_status s = enqueue_blocks(ctx, bl, x, y, z, static_cast<uint8_t *>(scratch), tmp_off, st);
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
}

}  // namespace cm

using namespace cm;

extern "C" cm_status cm_create(cm_ctx **out, int device, const cm_options *opt) {
    if (!out) return CM_EINVAL;
    *out = nullptr;
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
    if (opt && opt->max_transform_lg) {
        if (opt->max_transform_lg < 8 || opt->max_transform_lg > 32) {
            delete c;
            return CM_EINVAL;
        }
        c->max_lg = (int)opt->max_transform_lg;
    }
    if (opt && opt->field > CM_FIELD_GOLDILOCKS) {
        delete c;
        return CM_EINVAL;
    }
    c->allow_f30 = !(opt && opt->field == CM_FIELD_GOLDILOCKS);

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
    std::vector<uint32_t> h30;
    build_tables30(h30);
    if (cudaMalloc(&c->d_tables, h.size() * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&c->d_tables30, h30.size() * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_status, 64) != cudaSuccess) {
        cm_destroy(c);
        return CM_ENOMEM;
    }
    cudaMemcpy(c->d_tables, h.data(), h.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_tables30, h30.data(), h30.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    c->rt30.small = c->d_tables30;
    c->rt30.big_lo_fwd = c->d_tables30 + 8192;
    c->rt30.big_hi_fwd = c->rt30.big_lo_fwd + 32768;
    c->rt30.big_lo_inv = c->rt30.big_hi_fwd + 32768;
    c->rt30.big_hi_inv = c->rt30.big_lo_inv + 32768;
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

extern "C" uint64_t cm_ntt_length(int kind, uint64_t n, uint64_t m) {
    std::vector<Block> bl;
    if (!make_blocks(kind, n, m, 32, true, &bl)) return 0;
    uint64_t L = 0;
    for (const Block &b : bl)
        if (b.p.L > L) L = b.p.L;
    return L;
}

extern "C" uint64_t cm_scratch_bytes(int kind, uint64_t n, uint64_t m) {
    std::vector<Block> bl;
    if (!make_blocks(kind, n, m, 32, true, &bl)) return 0;
    uint64_t tmp_off = 0;
    return blocks_scratch(bl, &tmp_off);
}

extern "C" uint32_t cm_launch_count(int kind, uint64_t n, uint64_t m) {
    std::vector<Block> bl;
    if (!make_blocks(kind, n, m, 32, true, &bl)) return 0;
    uint32_t c = 0;
    for (const Block &b : bl) c += b.p.launches + (b.accumulate ? 1 : 0);
    return c;
}

extern "C" uint64_t cm_block_count(int kind, uint64_t n, uint64_t m, uint32_t max_transform_lg) {
    std::vector<Block> bl;
    const int lg = max_transform_lg ? (int)max_transform_lg : 32;
    return make_blocks(kind, n, m, lg, true, &bl) ? bl.size() : 0;
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
    if (!make_blocks(kind, n, m, ctx->max_lg, ctx->allow_f30, &bl)) return CM_EINVAL;
    uint64_t tmp_off = 0;
    const uint64_t sb = blocks_scratch(bl, &tmp_off);
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
    if (s == CM_OK) s = enqueue_blocks(ctx, bl, xd, yd, zd, b, tmp_off, st);
    if (s == CM_OK && cudaMemcpyAsync(zh, zd, 8 * zw, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = CM_EDEVICE;
    // the last block's precondition flags (every block checks the whole x)
    const Plan &last = bl.back().p;
    if (s == CM_OK && kind == CM_DODIS &&
        cudaMemcpyAsync(pre_h, b + last.scratch_bytes - 256, sizeof(pre_h), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        s = CM_EDEVICE;
    cudaFreeAsync(buf, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CM_EDEVICE;
    if (s == CM_OK && kind == CM_DODIS && (pre_h[0] == 0 || pre_h[1] == 0)) s = CM_EPRECOND;
    return s;
}
