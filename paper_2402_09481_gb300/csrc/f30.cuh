// The prime field F_q, q = 3 * 2^30 + 1, on the 32-bit integer pipe.
//
// This is the field the paper's own implementation uses for inputs below 2^29
// bits (Section "Performance": operations over the field of the prime
// 3 * 2^30 + 1, and a larger field above).  Here it carries every transform of
// length L <= 2^30: the convolution coefficients are counts at most
// K <= L - 1 < q, so the transform result is the exact integer count and its
// parity is bit 0 of the canonical value, as with the 64-bit field.
//
// Elements are 32-bit words, canonical in [0, q) between kernels.  Products use
// Montgomery reduction with R = 2^32 in its subtractive form
//     mont(a, b) = (a b - m q) / 2^32,   m = (a b mod 2^32) q^-1 mod 2^32,
// whose numerator is divisible by 2^32 by construction, so the high words
// subtract exactly and the result lies in (-q, q): one conditional add of q.
// Twiddle tables hold w R mod q, so mont(x, w R) = x w: data stay in normal
// form throughout.  5 generates F_q^*, and g30 = 5^3 = 125 has order 2^30.
#pragma once
#include <stdint.h>

#define F30_Q 3221225473u   // 3 * 2^30 + 1 = 0xC0000001
#define F30_QINV 0x40000001u  // q^-1 mod 2^32
#define F30_R 1073741823u   // 2^32 mod q
#define F30_G30 125u        // 5^3, a root of unity of order 2^30

#ifdef __CUDACC__
#define F30_HD __host__ __device__ __forceinline__
#define F30_CX __host__ __device__ constexpr
#else
#define F30_HD inline
#define F30_CX constexpr
#endif

F30_HD uint32_t f30_add(uint32_t a, uint32_t b) {
    const uint32_t u = F30_Q - b;  // a + b - q = a - u
    const uint32_t r = a - u;
    return a < u ? r + F30_Q : r;
}

F30_HD uint32_t f30_sub(uint32_t a, uint32_t b) {
    const uint32_t r = a - b;
    return a < b ? r + F30_Q : r;
}

// a b 2^-32 mod q for a, b < q.
F30_HD uint32_t f30_mont(uint32_t a, uint32_t b) {
    const uint64_t t = (uint64_t)a * b;
    const uint32_t lo = (uint32_t)t, hi = (uint32_t)(t >> 32);
    const uint32_t m = lo * F30_QINV;
    const uint32_t h2 = (uint32_t)(((uint64_t)m * F30_Q) >> 32);
    const uint32_t r = hi - h2;
    return hi < h2 ? r + F30_Q : r;
}

// Plain modular arithmetic for tables and constants (host and constexpr).
F30_CX uint32_t f30_mulmod(uint32_t a, uint32_t b) {
    return (uint32_t)((uint64_t)a * b % F30_Q);
}
F30_CX uint32_t f30_pow(uint32_t a, uint64_t e) {
    uint32_t r = 1;
    while (e) {
        if (e & 1) r = f30_mulmod(r, a);
        a = f30_mulmod(a, a);
        e >>= 1;
    }
    return r;
}
// Montgomery form w R mod q.
F30_CX uint32_t f30_to_mont(uint32_t w) {
    return (uint32_t)(((uint64_t)w << 32) % F30_Q);
}
// omega_32^j R mod q: the twiddles inside register sub-transforms (length <= 32).
F30_CX uint32_t f30_tw32(int j) {
    return f30_to_mont(f30_pow(f30_pow(F30_G30, 1ull << 25), (uint64_t)j));
}
// Root of order 2^30 (or its inverse).
F30_CX uint32_t f30_root_2_30(bool inverse) {
    return inverse ? f30_pow(F30_G30, (1ull << 30) - 1) : F30_G30;
}
// L^-1 mod q for L = 2^k <= 2^30, in the form the pointwise product takes
// (mont(mont(a, b), c) = a b L^-1 needs c = L^-1 R^2).
F30_CX uint32_t f30_linv_mont2(uint64_t L) {
    return f30_to_mont(f30_to_mont(f30_pow((uint32_t)L, F30_Q - 2)));
}

#ifdef __CUDACC__
// Constant-bank copy of f30_tw32 for the unrolled sub-transforms.
static __constant__ uint32_t kF30Tw32[32] = {
    f30_tw32(0),  f30_tw32(1),  f30_tw32(2),  f30_tw32(3),  f30_tw32(4),  f30_tw32(5),  f30_tw32(6),
    f30_tw32(7),  f30_tw32(8),  f30_tw32(9),  f30_tw32(10), f30_tw32(11), f30_tw32(12), f30_tw32(13),
    f30_tw32(14), f30_tw32(15), f30_tw32(16), f30_tw32(17), f30_tw32(18), f30_tw32(19), f30_tw32(20),
    f30_tw32(21), f30_tw32(22), f30_tw32(23), f30_tw32(24), f30_tw32(25), f30_tw32(26), f30_tw32(27),
    f30_tw32(28), f30_tw32(29), f30_tw32(30), f30_tw32(31)};
#endif
