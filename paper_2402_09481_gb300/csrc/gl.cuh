// Goldilocks prime field F_p, p = 2^64 - 2^32 + 1, on the 32-bit integer pipe.
//
// The number-theoretic transform of the paper (Def. ntt, Thm. convolution) is a
// DFT over Z/pZ.  The convolutions computed here have integer coefficients at
// most 2^32 - 1 < p, so one 64-bit prime with 2^32 | p - 1 covers every length
// L = 2^k <= 2^32 exactly.  Structure used below:
//   2^64 = 2^32 - 1 (mod p)      ("EPS")
//   2^96 = -1       (mod p)
// Elements are stored canonically in [0, p) between kernels.
#pragma once
#include <stdint.h>

#define GL_P 0xFFFFFFFF00000001ull
#define GL_EPS 0xFFFFFFFFull

#ifdef __CUDACC__
#define GL_HD __host__ __device__ __forceinline__
#else
#define GL_HD inline
#endif

// a + b mod p for canonical a, b; canonical result.
GL_HD uint64_t gl_add_c(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    uint64_t t = s + GL_EPS;  // s - p (mod 2^64)
    // carry out of a + b: the true sum is s + 2^64 >= p, reduce to s + 2^64 - p = t.
    // no carry, but s + EPS wraps: s >= p, reduce to t.
    return ((s < a) | (t < s)) ? t : s;
}

// a - b mod p for canonical a, b; canonical result.
GL_HD uint64_t gl_sub_c(uint64_t a, uint64_t b) {
    uint64_t d = a - b;
    // borrow: d = a - b + 2^64, the answer a - b + p is d - EPS (no wrap).
    return (a < b) ? d - GL_EPS : d;
}

// Reduce the 128-bit value hi * 2^64 + lo modulo p; canonical result.
GL_HD uint64_t gl_reduce128(uint64_t lo, uint64_t hi) {
    uint64_t hh = hi >> 32;            // weight 2^96 = -1
    uint64_t hl = hi & 0xFFFFFFFFull;  // weight 2^64 = EPS
    uint64_t t0 = lo - hh;
    if (lo < hh) t0 -= GL_EPS;         // lo - hh + p
    uint64_t t1 = hl * GL_EPS;         // < 2^64
    uint64_t r = t0 + t1;
    if (r < t1) r += GL_EPS;           // carry 2^64 = EPS; cannot wrap again
    if (r >= GL_P) r -= GL_P;
    return r;
}

// Canonical form of any x < 2^64.
GL_HD uint64_t gl_canon(uint64_t x) { return x >= GL_P ? x - GL_P : x; }

// x * 2^s mod p for canonical x and 0 <= s <= 96; canonical result.  Inside
// fully unrolled transforms s is a compile-time constant, so only one branch
// survives.  These are the twiddles of every sub-transform of length <= 64:
// the root of order 64 is 8 = 2^3, so omega_{2h}^j = 2^(96 j / h).
GL_HD uint64_t gl_shl_c(uint64_t x, int s) {
    if (s == 0) return x;
    if (s == 96) return gl_sub_c(0, x);  // 2^96 = -1
    if (s <= 32) {
        // x 2^s = lo + 2^64 hi, hi < 2^32: 2^64 = EPS, hi * EPS = (hi << 32) - hi
        const uint64_t lo = x << s;
        const uint64_t hi = x >> (64 - s);
        const uint64_t t = (hi << 32) - hi;
        uint64_t r = lo + t;
        if (r < t) r += GL_EPS;
        return gl_canon(r);
    }
    if (s < 64) return gl_reduce128(x << s, x >> (64 - s));
    // 64 <= s < 96, t = s - 64: with A = x_lo 2^t = a0 + 2^32 a1 and
    // B = x_hi 2^t = b0 + 2^32 b1,  x 2^s = 2^32 (a0 - b1) - (a0 + a1 + b0)  (mod p)
    const int t = s - 64;
    const uint64_t A = (x & 0xFFFFFFFFull) << t, B = (x >> 32) << t;
    const uint64_t a0 = A & 0xFFFFFFFFull, a1 = A >> 32, b0 = B & 0xFFFFFFFFull, b1 = B >> 32;
    const uint64_t pos = gl_canon(a0 << 32);
    const uint64_t neg = (b1 << 32) + a0 + a1 + b0;  // < 2^63 + 2^34 < p
    return gl_sub_c(pos, neg);
}

// ---------------------------------------------------------------------------
// Device versions: the same functions written with explicit 32-bit carry
// chains (PTX add.cc / addc / sub.cc / subc / mad.cc).  The transforms are
// bound by the integer ALU pipe, and these sequences issue markedly fewer
// instructions than what the compiler makes of the 64-bit C forms.  Host code
// (and the field self-test) uses the C forms above.
// ---------------------------------------------------------------------------
#if defined(__CUDACC__)
#define GL_SPLIT(x, lo, hi) "mov.b64 {" lo ", " hi "}, " x ";\n\t"

// a - b, canonical a, b (5 instructions)
__device__ __forceinline__ uint64_t gl_sub_ptx(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("{\n\t.reg .u32 al, ah, bl, bh, dl, dh, bw;\n\t"
        GL_SPLIT("%1", "al", "ah") GL_SPLIT("%2", "bl", "bh")
        "sub.cc.u32 dl, al, bl;\n\tsubc.cc.u32 dh, ah, bh;\n\tsubc.u32 bw, 0, 0;\n\t"
        // borrow: d + p = d - EPS; bw = 0xFFFFFFFF exactly when it borrowed
        "sub.cc.u32 dl, dl, bw;\n\tsubc.u32 dh, dh, 0;\n\t"
        "mov.b64 %0, {dl, dh};\n\t}"
        : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// a + b = a - (p - b), canonical a, b (7 instructions): p - b is in (0, p],
// and the subtraction's borrow fix lands in [0, p) either way.
__device__ __forceinline__ uint64_t gl_add_ptx(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("{\n\t.reg .u32 al, ah, bl, bh, nl, nh, dl, dh, bw;\n\t"
        GL_SPLIT("%1", "al", "ah") GL_SPLIT("%2", "bl", "bh")
        "sub.cc.u32 nl, 1, bl;\n\tsubc.u32 nh, 0xFFFFFFFF, bh;\n\t"
        "sub.cc.u32 dl, al, nl;\n\tsubc.cc.u32 dh, ah, nh;\n\tsubc.u32 bw, 0, 0;\n\t"
        "sub.cc.u32 dl, dl, bw;\n\tsubc.u32 dh, dh, 0;\n\t"
        "mov.b64 %0, {dl, dh};\n\t}"
        : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// Canonical residue of r0 + 2^32 r1 + 2^64 r2 + 2^96 r3 (32-bit limbs):
// t = (r1:r0) - r3 (borrow -> + p), u = r2 * EPS = (r2 << 32) - r2 (< p),
// v = t + u (carry -> + EPS, no second carry), then v >= p -> v - p.
__device__ __forceinline__ uint64_t gl_reduce_limbs(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    uint64_t r;
    asm("{\n\t.reg .u32 t0, t1, bw, u0, u1, c, e;\n\t.reg .pred q;\n\t"
        "sub.cc.u32 t0, %1, %4;\n\tsubc.cc.u32 t1, %2, 0;\n\tsubc.u32 bw, 0, 0;\n\t"
        "sub.cc.u32 t0, t0, bw;\n\tsubc.u32 t1, t1, 0;\n\t"
        "sub.cc.u32 u0, 0, %3;\n\tsubc.u32 u1, %3, 0;\n\t"
        "add.cc.u32 t0, t0, u0;\n\taddc.cc.u32 t1, t1, u1;\n\taddc.u32 c, 0, 0;\n\t"
        "sub.u32 e, 0, c;\n\tadd.cc.u32 t0, t0, e;\n\taddc.u32 t1, t1, 0;\n\t"
        "setp.eq.u32 q, t1, 0xFFFFFFFF;\n\tsetp.ne.and.u32 q, t0, 0, q;\n\t"
        "@q sub.u32 t0, t0, 1;\n\t@q mov.u32 t1, 0;\n\t"
        "mov.b64 %0, {t0, t1};\n\t}"
        : "=l"(r) : "r"(r0), "r"(r1), "r"(r2), "r"(r3));
    return r;
}

// Canonical residue of r0 + 2^32 r1 + 2^64 r2 (the shift twiddles with s <= 32,
// where the 2^96 limb is zero): u = r2 * EPS (< p), v = (r1:r0) + u with the
// carry folded back as + EPS, then v >= p -> v - p.
__device__ __forceinline__ uint64_t gl_reduce_limbs3(uint32_t r0, uint32_t r1, uint32_t r2) {
    uint64_t r;
    asm("{\n\t.reg .u32 t0, t1, u0, u1, c, e;\n\t.reg .pred q;\n\t"
        "sub.cc.u32 u0, 0, %3;\n\tsubc.u32 u1, %3, 0;\n\t"
        "add.cc.u32 t0, %1, u0;\n\taddc.cc.u32 t1, %2, u1;\n\taddc.u32 c, 0, 0;\n\t"
        "sub.u32 e, 0, c;\n\tadd.cc.u32 t0, t0, e;\n\taddc.u32 t1, t1, 0;\n\t"
        "setp.eq.u32 q, t1, 0xFFFFFFFF;\n\tsetp.ne.and.u32 q, t0, 0, q;\n\t"
        "@q sub.u32 t0, t0, 1;\n\t@q mov.u32 t1, 0;\n\t"
        "mov.b64 %0, {t0, t1};\n\t}"
        : "=l"(r) : "r"(r0), "r"(r1), "r"(r2));
    return r;
}

// a * b mod p for a, b < 2^64; canonical result.
__device__ __forceinline__ uint64_t gl_mul_ptx(uint64_t a, uint64_t b) {
    uint32_t r0, r1, r2, r3;
    asm("{\n\t.reg .u32 al, ah, bl, bh;\n\t"
        GL_SPLIT("%4", "al", "ah") GL_SPLIT("%5", "bl", "bh")
        "mul.lo.u32 %0, al, bl;\n\tmul.hi.u32 %1, al, bl;\n\t"
        "mul.lo.u32 %2, ah, bh;\n\tmul.hi.u32 %3, ah, bh;\n\t"
        "mad.lo.cc.u32 %1, al, bh, %1;\n\tmadc.hi.cc.u32 %2, al, bh, %2;\n\taddc.u32 %3, %3, 0;\n\t"
        "mad.lo.cc.u32 %1, ah, bl, %1;\n\tmadc.hi.cc.u32 %2, ah, bl, %2;\n\taddc.u32 %3, %3, 0;\n\t}"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "l"(a), "l"(b));
    return gl_reduce_limbs(r0, r1, r2, r3);
}

// x * 2^s mod p, canonical x, 0 <= s <= 96 (compile-time after unrolling).
__device__ __forceinline__ uint64_t gl_shl_ptx(uint64_t x, int s) {
    if (s == 0) return x;
    if (s == 96) return gl_sub_ptx(0, x);
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    if (s < 32) return gl_reduce_limbs3(x0 << s, __funnelshift_l(x0, x1, s), x1 >> (32 - s));
    if (s == 32) return gl_reduce_limbs3(0, x0, x1);
    if (s < 64) {
        const int t = s - 32;
        return gl_reduce_limbs(0, x0 << t, __funnelshift_l(x0, x1, t), x1 >> (32 - t));
    }
    // 64 <= s < 96: x 2^s = 2^32 a0 - (2^32 b1 + a0 + a1 + b0), with
    // x0 2^t = a0 + 2^32 a1, x1 2^t = b0 + 2^32 b1, t = s - 64; both terms < p.
    const int t = s - 64;
    const uint32_t a0 = x0 << t, a1 = t ? x0 >> (32 - t) : 0u;
    const uint32_t b0 = x1 << t, b1 = t ? x1 >> (32 - t) : 0u;
    uint64_t r;
    asm("{\n\t.reg .u32 nl, nh, dl, dh, bw;\n\t"
        "add.cc.u32 nl, %1, %2;\n\taddc.u32 nh, %4, 0;\n\t"
        "add.cc.u32 nl, nl, %3;\n\taddc.u32 nh, nh, 0;\n\t"
        "sub.cc.u32 dl, 0, nl;\n\tsubc.cc.u32 dh, %1, nh;\n\tsubc.u32 bw, 0, 0;\n\t"
        "sub.cc.u32 dl, dl, bw;\n\tsubc.u32 dh, dh, 0;\n\t"
        "mov.b64 %0, {dl, dh};\n\t}"
        : "=l"(r) : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    return r;
}
#endif

// Dispatch: PTX sequences in device code, C forms on the host.
GL_HD uint64_t gl_add(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return gl_add_ptx(a, b);
#else
    return gl_add_c(a, b);
#endif
}
GL_HD uint64_t gl_sub(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return gl_sub_ptx(a, b);
#else
    return gl_sub_c(a, b);
#endif
}
GL_HD uint64_t gl_shl(uint64_t x, int s) {
#if defined(__CUDA_ARCH__)
    return gl_shl_ptx(x, s);
#else
    return gl_shl_c(x, s);
#endif
}

#ifdef __CUDACC__
__device__ __forceinline__ uint64_t gl_mul(uint64_t a, uint64_t b) { return gl_mul_ptx(a, b); }
__device__ __forceinline__ uint64_t gl_mul_c(uint64_t a, uint64_t b) {
    return gl_reduce128(a * b, __umul64hi(a, b));
}
#endif

// Host-side multiply (table construction, plans).
static inline uint64_t gl_mul_host(uint64_t a, uint64_t b) {
    unsigned __int128 x = (unsigned __int128)a * b;
    return gl_reduce128((uint64_t)x, (uint64_t)(x >> 64));
}

static inline uint64_t gl_pow_host(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = gl_mul_host(r, a);
        a = gl_mul_host(a, a);
        e >>= 1;
    }
    return r;
}

// 7 generates F_p^* (p - 1 = 2^32 * 3 * 5 * 17 * 257 * 65537), so 7^((p-1)/2^32)
// has order 2^32; its fifth power g still does and satisfies g^(2^26) = 8, i.e.
// the root of order 64 is 2^3 and every root of order <= 64 is a power of two.
// omega_L = g^(2^32 / L).
static inline uint64_t gl_root_2_32_host(int inverse) {
    uint64_t g = gl_pow_host(gl_pow_host(7, (GL_P - 1) >> 32), 5);
    return inverse ? gl_pow_host(g, GL_P - 2) : g;
}

// L^{-1} mod p for L | p - 1: L * ((p - 1) / L) = -1, so L^{-1} = p - (p - 1) / L.
static inline uint64_t gl_inv_pow2_host(uint64_t L) { return GL_P - (GL_P - 1) / L; }
