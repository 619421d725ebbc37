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
GL_HD uint64_t gl_add(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    uint64_t t = s + GL_EPS;  // s - p (mod 2^64)
    // carry out of a + b: the true sum is s + 2^64 >= p, reduce to s + 2^64 - p = t.
    // no carry, but s + EPS wraps: s >= p, reduce to t.
    return ((s < a) | (t < s)) ? t : s;
}

// a - b mod p for canonical a, b; canonical result.
GL_HD uint64_t gl_sub(uint64_t a, uint64_t b) {
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

#ifdef __CUDACC__
__device__ __forceinline__ uint64_t gl_mul(uint64_t a, uint64_t b) {
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

// 7 generates F_p^* (p - 1 = 2^32 * 3 * 5 * 17 * 257 * 65537).  g32 = 7^((p-1)/2^32)
// has order exactly 2^32; omega_L = g32^(2^32 / L).
static inline uint64_t gl_root_2_32_host(int inverse) {
    uint64_t g = gl_pow_host(7, (GL_P - 1) >> 32);
    return inverse ? gl_pow_host(g, GL_P - 2) : g;
}

// L^{-1} mod p for L | p - 1: L * ((p - 1) / L) = -1, so L^{-1} = p - (p - 1) / L.
static inline uint64_t gl_inv_pow2_host(uint64_t L) { return GL_P - (GL_P - 1) / L; }
