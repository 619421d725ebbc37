// Trevisan's extractor, one-bit step (Section "Trevisan implementation"): m
// Reed-Solomon-Hadamard one-bit extractions of one input, one output bit per
// GPU thread.
//
// GF(2^l) elements are polynomials over GF(2) modulo f (cm_rsh_modulus), held
// "left-aligned" in W = ceil(l / 64) words: the element e is stored as
// e x^delta, delta = 64 W - l, so that the high half of a double-length
// product starts on a word boundary whatever l is.  With p' = p x^delta and
// alpha1 plain, p' alpha1 = (p alpha1) x^delta: its low W words are the low
// part of p alpha1 (aligned) and its high W words are p alpha1's coefficients
// from x^l up.  Horner's rule p <- p alpha1 + x_i then takes per step
//   - a carry-less product by 4-bit windows of p': each thread keeps the 16
//     multiples v alpha1 (v < 16) in shared memory;
//   - a reduction of the high half h by x^l mod f = 1 + x^t (one or three
//     taps t) with shifts: h g = lo + x^l h2, and h2 g has degree below l,
//     since every tap of the moduli up to l = 256 is at most (l + 1) / 2;
//   - an XOR of the next chunk (pre-aligned by k_rsh_chunks).
// The output bit is the parity of alpha2' AND p' (both aligned alike).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>

#include "cm_ctx.h"
#include "cm_internal.h"
#include "cm_trevisan.h"

namespace cm {
namespace {

constexpr uint32_t kMaxL = 256;
constexpr int kRshThreads = 128;

// ---------------------------------------------------------------------------
// Host: GF(2)[x] polynomials of degree < 64 kPolyWords and the modulus search
// (Rabin's irreducibility test).
// ---------------------------------------------------------------------------
constexpr int kPolyWords = 9;  // degree < 576 >= 2 * 256 + 4
struct Poly {
    uint64_t w[kPolyWords];
};

static Poly pzero() {
    Poly p;
    memset(&p, 0, sizeof(p));
    return p;
}
static int pdeg(const Poly &p) {
    for (int i = kPolyWords - 1; i >= 0; --i)
        if (p.w[i]) return 64 * i + 63 - __builtin_clzll(p.w[i]);
    return -1;
}
static bool pbit(const Poly &p, int k) { return (p.w[k >> 6] >> (k & 63)) & 1; }
static void pset(Poly &p, int k) { p.w[k >> 6] ^= 1ull << (k & 63); }
static Poly pshl(const Poly &p, int s) {
    Poly r = pzero();
    const int ws = s >> 6, bs = s & 63;
    for (int i = kPolyWords - 1; i >= ws; --i) {
        uint64_t v = p.w[i - ws] << bs;
        if (bs && i - ws - 1 >= 0) v |= p.w[i - ws - 1] >> (64 - bs);
        r.w[i] = v;
    }
    return r;
}
static void pxor(Poly &a, const Poly &b) {
    for (int i = 0; i < kPolyWords; ++i) a.w[i] ^= b.w[i];
}
static Poly pmod(Poly a, const Poly &f) {
    const int df = pdeg(f);
    for (int d = pdeg(a); d >= df; d = pdeg(a)) pxor(a, pshl(f, d - df));
    return a;
}
static Poly pmulmod(const Poly &a, const Poly &b, const Poly &f) {
    Poly r = pzero();
    const int db = pdeg(b);
    for (int k = 0; k <= db; ++k)
        if (pbit(b, k)) pxor(r, pshl(a, k));
    return pmod(r, f);
}
static Poly pgcd(Poly a, Poly b) {
    while (pdeg(b) >= 0) {
        Poly t = pmod(a, b);
        a = b;
        b = t;
    }
    return a;
}
static bool pequal(const Poly &a, const Poly &b) { return memcmp(&a, &b, sizeof(Poly)) == 0; }

// x^(2^k) mod f by k squarings.
static Poly x_pow_2k(int k, const Poly &f) {
    Poly r = pzero();
    pset(r, 1);
    r = pmod(r, f);
    for (int i = 0; i < k; ++i) r = pmulmod(r, r, f);
    return r;
}

static bool irreducible(const Poly &f) {
    const int l = pdeg(f);
    Poly x = pzero();
    pset(x, 1);
    if (!pequal(x_pow_2k(l, f), pmod(x, f))) return false;
    int n = l;
    for (int p = 2; p <= n; ++p) {
        if (n % p) continue;
        while (n % p == 0) n /= p;
        Poly g = x_pow_2k(l / p, f);
        pxor(g, x);
        const Poly d = pgcd(f, pmod(g, f));
        if (pdeg(d) != 0) return false;
    }
    return true;
}

struct Modulus {
    uint32_t taps[3];
    uint32_t count;
};

static bool find_modulus(uint32_t l, Modulus *out) {
    static std::mutex mu;
    static std::map<uint32_t, Modulus> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(l);
    if (it != cache.end()) {
        *out = it->second;
        return true;
    }
    auto make = [&](std::initializer_list<uint32_t> taps) {
        Poly f = pzero();
        pset(f, (int)l);
        pset(f, 0);
        for (uint32_t t : taps) pset(f, (int)t);
        return f;
    };
    Modulus m;
    memset(&m, 0, sizeof(m));
    bool found = false;
    for (uint32_t k = 1; k < l && !found; ++k) {
        if (irreducible(make({k}))) {
            m.taps[0] = k;
            m.count = 1;
            found = true;
        }
    }
    for (uint32_t a = 3; a < l && !found; ++a)
        for (uint32_t b = 2; b < a && !found; ++b)
            for (uint32_t c = 1; c < b && !found; ++c)
                if (irreducible(make({a, b, c}))) {
                    m.taps[0] = a;
                    m.taps[1] = b;
                    m.taps[2] = c;
                    m.count = 3;
                    found = true;
                }
    if (!found) return false;
    cache[l] = m;
    *out = m;
    return true;
}

// ---------------------------------------------------------------------------
// Device
// ---------------------------------------------------------------------------

// 64 bits of a packed bit string from bit `pos` (bits at or past nbits read 0).
__device__ __forceinline__ uint64_t bits64(const uint64_t *__restrict__ src, uint64_t nbits, uint64_t pos) {
    if (pos >= nbits) return 0;
    const uint64_t nw = (nbits + 63) >> 6;
    const uint64_t w = pos >> 6;
    const int sh = (int)(pos & 63);
    uint64_t r = __ldg(src + w) >> sh;
    if (sh && w + 1 < nw) r |= __ldg(src + w + 1) << (64 - sh);
    if (nbits - pos < 64) r &= (1ull << (nbits - pos)) - 1;
    return r;
}

// The l bits at `pos` as an aligned element: bit j of the run (the j-th listed
// bit) is the coefficient of x^(l-1-j), times x^delta: the bit reversal of
// the run zero-extended to 64 W bits.
template <int W>
__device__ __forceinline__ void aligned_element(const uint64_t *__restrict__ src, uint64_t nbits, uint64_t pos,
                                                uint32_t l, uint64_t (&e)[W]) {
    uint64_t raw[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        const uint32_t lo = 64u * q;
        raw[q] = lo < l ? bits64(src, nbits, pos + lo) : 0ull;
        if (lo < l && l - lo < 64) raw[q] &= (1ull << (l - lo)) - 1;
    }
#pragma unroll
    for (int q = 0; q < W; ++q) e[q] = __brevll(raw[W - 1 - q]);
}

// Chunks x_1 .. x_s of the input, aligned: X[i * W + q].
template <int W>
__global__ void k_rsh_chunks(const uint64_t *__restrict__ x, uint64_t n, uint32_t l, uint64_t s,
                             uint64_t *__restrict__ X) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t e[W];
        aligned_element<W>(x, n, i * l, l, e);
#pragma unroll
        for (int q = 0; q < W; ++q) X[i * W + q] = e[q];
    }
}

// out = in << s (s < 64 NO), words past NO dropped.  s is the same in every
// thread: a bit shift, then word shifts by the binary digits of s / 64 under
// uniform branches, so that every register index is a constant.
template <int NI, int NO>
__device__ __forceinline__ void shl_words(const uint64_t (&in)[NI], uint32_t s, uint64_t (&out)[NO]) {
    const int bs = (int)(s & 63);
    const uint32_t ws = s >> 6;
#pragma unroll
    for (int q = 0; q < NO; ++q) {
        const uint64_t cur = q < NI ? in[q] : 0ull;
        const uint64_t prev = (q >= 1 && q - 1 < NI) ? in[q - 1] : 0ull;
        out[q] = (cur << bs) | (bs ? prev >> (64 - bs) : 0ull);
    }
#pragma unroll
    for (int b = 1; b < NO; b <<= 1) {
        if (ws & (uint32_t)b) {
#pragma unroll
            for (int q = NO - 1; q >= 0; --q) out[q] = q >= b ? out[q - b] : 0ull;
        }
    }
}

// h (a polynomial of W words) times g = x^l mod f = 1 + x^t1 [+ x^t2 + x^t3],
// into 2W words.
template <int W>
__device__ __forceinline__ void times_g(const uint64_t (&h)[W], const uint32_t (&taps)[3], int ntaps,
                                        uint64_t (&q)[2 * W]) {
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) q[i] = i < W ? h[i] : 0ull;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k < ntaps) {
            uint64_t sh[2 * W];
            shl_words<W, 2 * W>(h, taps[k], sh);
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) q[i] ^= sh[i];
        }
    }
}

// T (this thread's column of shared memory) <- v b for v < 16, b plain.
template <int WT>
__device__ __forceinline__ void build_table(uint64_t *T, int tid, const uint64_t (&b)[WT]) {
    uint64_t t2[WT], t4[WT], t8[WT];
#pragma unroll
    for (int q = 0; q < WT; ++q) {
        t2[q] = (b[q] << 1) | (q ? b[q - 1] >> 63 : 0);
        t4[q] = (b[q] << 2) | (q ? b[q - 1] >> 62 : 0);
        t8[q] = (b[q] << 3) | (q ? b[q - 1] >> 61 : 0);
    }
#pragma unroll
    for (int v = 0; v < 16; ++v) {
#pragma unroll
        for (int q = 0; q < WT; ++q) {
            uint64_t e = 0;
            if (v & 1) e ^= b[q];
            if (v & 2) e ^= t2[q];
            if (v & 4) e ^= t4[q];
            if (v & 8) e ^= t8[q];
            T[((size_t)v * WT + q) * kRshThreads + tid] = e;
        }
    }
}

// The plain element of an aligned one (a' >> delta), in WT words.
template <int W, int WT>
__device__ __forceinline__ void to_plain(const uint64_t (&a)[W], int delta, uint64_t (&p)[WT]) {
#pragma unroll
    for (int q = 0; q < W; ++q) {
        uint64_t v = delta ? (a[q] >> delta) : a[q];
        if (delta && q + 1 < W) v |= a[q + 1] << (64 - delta);
        p[q] = v;
    }
    if (WT > W) p[WT - 1] = 0;
}

struct RshField {
    uint32_t tap0, tap1, tap2;  // scalars: a member array here ends up in local memory
    int ntaps;
    uint32_t wl, bl;  // x^l at word wl, bit bl
    int delta;        // 64 W - l
};

// r' = a' b mod f, a' and r' aligned, b plain with its 16 multiples in T.
template <int W, int WT>
__device__ __forceinline__ void mul_table(const uint64_t *T, int tid, const RshField &F, const uint64_t (&a)[W],
                                          uint64_t (&r)[W]) {
    constexpr int NWIN = 16 * W;
    uint64_t prod[2 * W + 1];
#pragma unroll
    for (int q = 0; q < 2 * W + 1; ++q) prod[q] = 0;
    // carry-less product by 4-bit windows of a'
#pragma unroll
    for (int k = 0; k < NWIN; ++k) {
        const int o = k >> 4, sh = (k & 15) * 4;
        const uint32_t nib = (uint32_t)(a[o] >> sh) & 15u;
#pragma unroll
        for (int q = 0; q < WT; ++q) {
            const uint64_t t = T[((size_t)nib * WT + q) * kRshThreads + tid];
            prod[o + q] ^= t << sh;
            if (sh && o + q + 1 < 2 * W + 1) prod[o + q + 1] ^= t >> (64 - sh);
        }
    }
#pragma unroll
    for (int q = 0; q < W; ++q) r[q] = prod[q];
    // h = coefficients from x^l up (unaligned); h g = lo + x^l h2; h2 g has
    // degree < l; add (lo + h2 g) x^delta to the low half
    uint64_t h[W], qg[2 * W], h2[W], r2[2 * W], u[W];
#pragma unroll
    for (int q = 0; q < W; ++q) h[q] = prod[W + q];
    const uint32_t taps[3] = {F.tap0, F.tap1, F.tap2};
    times_g<W>(h, taps, F.ntaps, qg);
#pragma unroll
    for (int q = 0; q < W; ++q) {  // h2 = qg >> l, lo = qg mod x^l
        const uint64_t a0 = (F.wl == (uint32_t)(W - 1)) ? qg[q + W - 1] : qg[q + W];
        const uint64_t a1 = (F.wl == (uint32_t)(W - 1)) ? qg[q + W] : (q + W + 1 < 2 * W ? qg[q + W + 1] : 0ull);
        h2[q] = F.bl ? (a0 >> F.bl) | (a1 << (64 - F.bl)) : a0;
        u[q] = q < (int)F.wl ? qg[q] : (q == (int)F.wl && F.bl ? qg[q] & ((1ull << F.bl) - 1) : 0ull);
    }
    times_g<W>(h2, taps, F.ntaps, r2);
#pragma unroll
    for (int q = 0; q < W; ++q) u[q] ^= r2[q];
#pragma unroll
    for (int q = 0; q < W; ++q)
        r[q] ^= F.delta ? (u[q] << F.delta) | (q ? u[q - 1] >> (64 - F.delta) : 0ull) : u[q];
}

// r' = (alpha1')^e aligned, by square-and-multiply; al = plain alpha1.  T is
// rebuilt for every multiplicand.
template <int W, int WT>
__device__ __forceinline__ void pow_aligned(uint64_t *T, int tid, const RshField &F, const uint64_t (&al)[WT],
                                            uint64_t e, uint64_t (&r)[W]) {
#pragma unroll
    for (int q = 0; q < W; ++q) r[q] = 0;
    r[0] = 1ull << F.delta;  // the aligned 1 (delta < 64)
    for (int b = 63 - __clzll(e | 1); b >= 0; --b) {
        uint64_t p[WT], t[W];
        to_plain<W, WT>(r, F.delta, p);
        build_table<WT>(T, tid, p);
        mul_table<W, WT>(T, tid, F, r, t);  // r^2
        if ((e >> b) & 1) {
            build_table<WT>(T, tid, al);
            mul_table<W, WT>(T, tid, F, t, r);
        } else {
#pragma unroll
            for (int q = 0; q < W; ++q) r[q] = t[q];
        }
    }
    if (e == 0) {
#pragma unroll
        for (int q = 0; q < W; ++q) r[q] = q ? 0ull : 1ull << F.delta;
    }
}

// G threads per output bit (G a power of two <= 32).  The s chunks, after
// G len - s leading zero chunks (which leave p unchanged), split into G blocks
// of len; thread g runs Horner's rule over its block (P_g) and multiplies it
// by beta^(G-1-g), beta = alpha1^len, so that p = sum_g of those terms; the
// output is the XOR over the group of parity(alpha2 AND term).  G = 1 is the
// plain one-thread Horner.  WIDE: l + 3 > 64 W, so that a multiple v b
// (v < 16, degree < l + 3) needs one more word.
template <int W, bool WIDE, int G>
__global__ void __launch_bounds__(kRshThreads)
k_rsh(const uint64_t *__restrict__ X, uint64_t s, const uint64_t *__restrict__ seeds, uint32_t l, uint64_t m,
      uint32_t t1, uint32_t t2, uint32_t t3, int ntaps, uint32_t *__restrict__ z32) {
    constexpr int WT = WIDE ? W + 1 : W;
    extern __shared__ __align__(16) uint64_t T[];   // [v][word][thread]
    const int tid = threadIdx.x;
    RshField F;
    F.tap0 = t1;
    F.tap1 = t2;
    F.tap2 = t3;
    F.ntaps = ntaps;
    F.wl = l >> 6;
    F.bl = l & 63;
    F.delta = 64 * W - (int)l;

    const uint64_t gt = (uint64_t)blockIdx.x * kRshThreads + tid;
    const uint64_t out = gt / G;
    const int g = (int)(gt % G);
    const bool active = out < m;
    uint32_t zbit = 0;
    if (active) {
        const uint64_t nb = 2ull * l * m;
        uint64_t a1[W], a2[W], al[WT];
        aligned_element<W>(seeds, nb, 2ull * l * out, l, a1);
        aligned_element<W>(seeds, nb, 2ull * l * out + l, l, a2);
        to_plain<W, WT>(a1, F.delta, al);
        build_table<WT>(T, tid, al);
        const uint64_t len = (s + G - 1) / G, pad = G * len - s;
        const uint64_t k0 = (uint64_t)g * len, k1 = k0 + len;
        uint64_t pa[W];
#pragma unroll
        for (int q = 0; q < W; ++q) pa[q] = k0 >= pad ? __ldg(X + (k0 - pad) * W + q) : 0ull;
        for (uint64_t k = k0 + 1; k < k1; ++k) {
            uint64_t r[W];
            mul_table<W, WT>(T, tid, F, pa, r);
#pragma unroll
            for (int q = 0; q < W; ++q) pa[q] = k >= pad ? r[q] ^ __ldg(X + (k - pad) * W + q) : r[q];
        }
        if (G > 1) {
            uint64_t beta[W], gam[W], pb[WT], term[W];
            pow_aligned<W, WT>(T, tid, F, al, len, beta);
            to_plain<W, WT>(beta, F.delta, pb);
            pow_aligned<W, WT>(T, tid, F, pb, (uint64_t)(G - 1 - g), gam);
            to_plain<W, WT>(gam, F.delta, pb);
            build_table<WT>(T, tid, pb);
            mul_table<W, WT>(T, tid, F, pa, term);
#pragma unroll
            for (int q = 0; q < W; ++q) pa[q] = term[q];
        }
        uint32_t par = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) par ^= __popcll(a2[q] & pa[q]) & 1u;
        zbit = par;
    }
    if (G == 1) {
        const uint32_t word = __ballot_sync(0xffffffffu, zbit);
        if ((tid & 31) == 0) z32[out >> 5] = word;
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) zbit ^= __shfl_xor_sync(0xffffffffu, zbit, o);
        if (active && g == 0 && zbit) atomicOr(z32 + (out >> 5), 1u << (out & 31));
    }
}

template <int W, bool WIDE, int G>
static cudaError_t launch_rsh_kernel(const uint64_t *X, uint64_t s, const uint64_t *seeds, uint32_t l, uint64_t m,
                                     uint64_t *z, const Modulus &md, cudaStream_t st) {
    constexpr int WT = WIDE ? W + 1 : W;
    const size_t smem = (size_t)16 * WT * kRshThreads * sizeof(uint64_t);
    auto kern = k_rsh<W, WIDE, G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    uint64_t threads;
    if (G == 1) {
        threads = (m + 63) / 64 * 64;  // every output word written by ballots, tail bits 0
    } else {
        // bits are ORed in: clear the output first
        e = cudaMemsetAsync(z, 0, (m + 63) / 64 * 8, st);
        if (e != cudaSuccess) return e;
        threads = m * G;
    }
    const uint64_t grid = (threads + kRshThreads - 1) / kRshThreads;
    kern<<<(unsigned)grid, kRshThreads, smem, st>>>(X, s, seeds, l, m, md.taps[0], md.taps[1], md.taps[2],
                                                    (int)md.count, reinterpret_cast<uint32_t *>(z));
    return cudaGetLastError();
}

// One-bit seeds from the weak design's sets: bit j < 2l of seed i is
// y[sets[i * t + j]] (an index at or past d reads 0); seeds (zeroed first)
// receive 2 l m bits.
__global__ void k_gather_seeds(const uint64_t *__restrict__ y, uint64_t d, const uint32_t *__restrict__ sets,
                               uint32_t t, uint32_t l, uint64_t m, uint64_t *__restrict__ seeds) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint64_t base = 2ull * l * i;
    uint64_t acc = 0;
    int have = 0;
    uint64_t wpos = base >> 6;
    int off = (int)(base & 63);
    for (uint32_t j = 0; j < 2 * l; ++j) {
        const uint32_t idx = __ldg(sets + i * t + j);
        const uint64_t b = idx < d ? (__ldg(y + (idx >> 6)) >> (idx & 63)) & 1ull : 0ull;
        acc |= b << (off + have);
        if (++have + off == 64) {
            atomicOr(reinterpret_cast<unsigned long long *>(seeds + wpos), (unsigned long long)acc);
            acc = 0;
            have = 0;
            off = 0;
            ++wpos;
        }
    }
    if (have) atomicOr(reinterpret_cast<unsigned long long *>(seeds + wpos), (unsigned long long)acc);
}

// The shift reduction needs 2 t_max - 2 < l: true of every modulus up to 256
// (a trinomial's smallest k is at most l / 2: its reciprocal, with l - k, is
// irreducible too; the pentanomials' taps are small).
static bool taps_ok(uint32_t l, const Modulus &md) {
    uint32_t t = 0;
    for (uint32_t i = 0; i < md.count; ++i) t = md.taps[i] > t ? md.taps[i] : t;
    return 2 * t < l + 2;
}

template <int W, int G>
static cudaError_t launch_rsh_g(const uint64_t *X, uint64_t s, const uint64_t *seeds, uint32_t l, uint64_t m,
                                uint64_t *z, const Modulus &md, cudaStream_t st) {
    return l + 3 > 64u * W ? launch_rsh_kernel<W, true, G>(X, s, seeds, l, m, z, md, st)
                           : launch_rsh_kernel<W, false, G>(X, s, seeds, l, m, z, md, st);
}

// Threads per output: enough outputs-in-flight to fill the GPU (about 2048
// threads per SM) with one thread each; fewer outputs share their chunks
// among 8 or 32 threads (when each thread still has at least 64 chunks).
static int rsh_group(uint64_t m, uint64_t s, int nsm) {
    const uint64_t fill = (uint64_t)nsm * 2048;
    if (m * 8 <= fill && s >= 64 * 32) return m * 32 <= fill ? 32 : 8;
    if (m * 8 <= fill && s >= 64 * 8) return 8;
    return 1;
}

template <int W>
static cudaError_t launch_rsh_w(const uint64_t *x, uint64_t n, uint32_t l, const uint64_t *seeds, uint64_t m,
                                uint64_t *z, uint64_t *X, const Modulus &md, int nsm, cudaStream_t st) {
    const uint64_t s = (n + l - 1) / l;
    uint64_t cb = (s + 255) / 256;
    if (cb > (uint64_t)nsm * 8) cb = (uint64_t)nsm * 8;
    k_rsh_chunks<W><<<(unsigned)cb, 256, 0, st>>>(x, n, l, s, X);
    switch (rsh_group(m, s, nsm)) {
        case 32: return launch_rsh_g<W, 32>(X, s, seeds, l, m, z, md, st);
        case 8: return launch_rsh_g<W, 8>(X, s, seeds, l, m, z, md, st);
        default: return launch_rsh_g<W, 1>(X, s, seeds, l, m, z, md, st);
    }
}

static uint64_t rsh_scratch(uint64_t n, uint32_t l) {
    const int W = (int)((l + 63) / 64);
    const uint64_t s = (n + l - 1) / l;
    return (8ull * W * s + 255) & ~255ull;
}

static cm_status cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return CM_OK;
    if (e == cudaErrorMemoryAllocation) return CM_ENOMEM;
    return CM_EDEVICE;
}

// Enqueue the RSH extractions; scratch holds rsh_scratch(n, l) bytes.
static cm_status enqueue_rsh(cm_ctx *ctx, const uint64_t *x, uint64_t n, uint32_t l, const uint64_t *seeds,
                             uint64_t m, uint64_t *z, uint8_t *scratch, cudaStream_t st) {
    Modulus md;
    if (!find_modulus(l, &md) || !taps_ok(l, md)) return CM_EINVAL;
    const int W = (int)((l + 63) / 64);
    uint64_t *X = reinterpret_cast<uint64_t *>(scratch);
    cudaError_t e;
    ProfScope ps(ctx, "k_rsh", st);
    switch (W) {
        case 1: e = launch_rsh_w<1>(x, n, l, seeds, m, z, X, md, ctx->nsm, st); break;
        case 2: e = launch_rsh_w<2>(x, n, l, seeds, m, z, X, md, ctx->nsm, st); break;
        case 3: e = launch_rsh_w<3>(x, n, l, seeds, m, z, X, md, ctx->nsm, st); break;
        default: e = launch_rsh_w<4>(x, n, l, seeds, m, z, X, md, ctx->nsm, st); break;
    }
    return cuda_st(e);
}

static bool rsh_args_ok(const void *x, uint64_t n, uint32_t l, const void *seeds, uint64_t m, const void *z) {
    return x && seeds && z && n >= 1 && n <= (1ull << 40) && l >= 2 && l <= kMaxL && m >= 1 &&
           m <= (1ull << 32);
}

}  // namespace
}  // namespace cm

using namespace cm;

extern "C" uint32_t cm_rsh_field_bits(uint64_t n, double eps1) {
    if (n == 0 || !(eps1 > 0.0) || !(eps1 < 1.0)) return 0;
    return (uint32_t)ceil(log2((double)n) + 2.0 * log2(2.0 / eps1));
}

extern "C" cm_status cm_rsh_modulus(uint32_t l, uint32_t taps[3], uint32_t *count) {
    if (!taps || !count || l < 2 || l > kMaxL) return CM_EINVAL;
    Modulus m;
    if (!find_modulus(l, &m)) return CM_EINVAL;
    memcpy(taps, m.taps, sizeof(m.taps));
    *count = m.count;
    return CM_OK;
}

extern "C" cm_status cm_trevisan_rsh(cm_ctx *ctx, const uint64_t *x, uint64_t n, uint32_t l, const uint64_t *seeds,
                                     uint64_t m, uint64_t *z, cm_stream stream) {
    if (!ctx || !rsh_args_ok(x, n, l, seeds, m, z)) return CM_EINVAL;
    const uint64_t need = rsh_scratch(n, l);
    if (need > ctx->budget) return CM_ENOMEM;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *sc = nullptr;
    if (cudaMallocFromPoolAsync(&sc, need, ctx->pool, st) != cudaSuccess) {
        cudaGetLastError();
        return CM_ENOMEM;
    }
    cm_status s = enqueue_rsh(ctx, x, n, l, seeds, m, z, static_cast<uint8_t *>(sc), st);
    if (cudaFreeAsync(sc, st) != cudaSuccess && s == CM_OK) s = CM_EDEVICE;
    return s;
}

extern "C" cm_status cm_trevisan(cm_ctx *ctx, const uint64_t *x, uint64_t n, const uint64_t *y, uint64_t d,
                                 const uint32_t *sets, uint32_t t, uint64_t m, uint32_t l, uint64_t *z,
                                 cm_stream stream) {
    if (!ctx || !y || !sets || d == 0 || !rsh_args_ok(x, n, l, sets, m, z) || t < 2 * l) return CM_EINVAL;
    const uint64_t sb = (2ull * l * m + 63) / 64 * 8;
    const uint64_t soff = (rsh_scratch(n, l) + 255) & ~255ull;
    const uint64_t need = soff + sb;
    if (need > ctx->budget) return CM_ENOMEM;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *sc = nullptr;
    if (cudaMallocFromPoolAsync(&sc, need, ctx->pool, st) != cudaSuccess) {
        cudaGetLastError();
        return CM_ENOMEM;
    }
    uint8_t *b = static_cast<uint8_t *>(sc);
    uint64_t *seeds = reinterpret_cast<uint64_t *>(b + soff);
    cm_status s = cuda_st(cudaMemsetAsync(seeds, 0, sb, st));
    if (s == CM_OK) {
        ProfScope ps(ctx, "k_gather_seeds", st);
        k_gather_seeds<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(y, d, sets, t, l, m, seeds);
        s = cuda_st(cudaGetLastError());
    }
    if (s == CM_OK) s = enqueue_rsh(ctx, x, n, l, seeds, m, z, b, st);
    if (cudaFreeAsync(sc, st) != cudaSuccess && s == CM_OK) s = CM_EDEVICE;
    return s;
}
