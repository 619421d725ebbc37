// The prime field F_q, q = 5 * 2^25 + 1, with lazy reduction on the 32-bit
// integer pipe.
//
// Every convolution coefficient of a product of transform length L <= 2^25 is
// a count of at most K <= L < q, so this field gives the exact integer counts
// (Thm. convolution) exactly as the paper's field of 3 * 2^30 + 1 does; its
// point is headroom.  Since 25 q < 2^32, a 32-bit word can hold a value up to
// 25 times the modulus, and the butterflies of a transform need not bring
// their results back to [0, q): a radix-2 butterfly of Cooley-Tukey form
//     (x, y) -> (x + t, x - t + 2q),   t = w y mod q in [0, 2q),
// adds at most 2q to the bound of its inputs and costs two integer adds plus
// the product.  Reductions happen once per on-chip step instead of after
// every add and subtract.
//
// Value ranges (the kernels keep to them):
//   red(x)   any 32-bit x -> [0, 2q)  (x - floor(x mu / 2^32) q, mu = 25)
//   canon(x) any 32-bit x -> [0, q)
//   mont(x, w) = x w 2^-32 mod q in (0, 2q) whenever x w < q 2^32, i.e. for
//            any x when w < q, and for x < 2^31 when w < 2q
//   shoup(x, w, w') = x w mod q in [0, 2q) for any x, w < q,
//            w' = floor(w 2^32 / q) (V. Shoup's precomputed-quotient product)
//   add, sub: [0, 2q) x [0, 2q) -> [0, 2q)
// Root tables hold w 2^32 mod q (Montgomery form, canonical), so mont(x, w R)
// is x w; the constants inside register sub-transforms are plain roots with
// their Shoup quotients.  3 generates F_q^* (q - 1 = 5 * 2^25), so
// g25 = 3^5 = 243 has order 2^25.
#pragma once
#include <stdint.h>

#define F25_Q 167772161u      // 5 * 2^25 + 1
#define F25_QINV 0xF6000001u  // q^-1 mod 2^32
#define F25_R 100663271u      // 2^32 mod q
#define F25_MU 25u            // floor(2^32 / q)
#define F25_G25 243u          // 3^5, a root of unity of order 2^25

#ifdef __CUDACC__
#define F25_HD __host__ __device__ __forceinline__
#define F25_CX __host__ __device__ constexpr
#else
#define F25_HD inline
#define F25_CX constexpr
#endif

F25_HD uint32_t f25_mulhi(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

F25_HD uint32_t f25_umin(uint32_t a, uint32_t b) { return a < b ? a : b; }

// [0, 2q) representative of any 32-bit x: the quotient estimate
// floor(x mu / 2^32) is floor(x / q) or one less.
F25_HD uint32_t f25_red(uint32_t x) { return x - f25_mulhi(x, F25_MU) * F25_Q; }

// Canonical representative of any 32-bit x.
F25_HD uint32_t f25_canon(uint32_t x) {
    const uint32_t r = f25_red(x);
    return f25_umin(r, r - F25_Q);  // r - q wraps above r when r < q
}

// a + b and a - b for a, b in [0, 2q), back in [0, 2q).
F25_HD uint32_t f25_add(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return f25_umin(s, s - 2 * F25_Q);
}
F25_HD uint32_t f25_sub(uint32_t a, uint32_t b) {
    const uint32_t d = a - b + 2 * F25_Q;
    return f25_umin(d, d - 2 * F25_Q);
}

// x w 2^-32 mod q in (0, 2q), for x w < q 2^32 (subtractive Montgomery form:
// with m = (x w mod 2^32) q^-1, x w - m q has a zero low word, so its high
// word is hi(x w) - hi(m q) exactly, in (-q, q)).
F25_HD uint32_t f25_mont(uint32_t x, uint32_t w) {
    const uint32_t lo = x * w, hi = f25_mulhi(x, w);
    const uint32_t m = lo * F25_QINV;
    return hi - f25_mulhi(m, F25_Q) + F25_Q;
}

// x w mod q in [0, 2q) for any x and w < q, wq = floor(w 2^32 / q).
F25_HD uint32_t f25_shoup(uint32_t x, uint32_t w, uint32_t wq) {
    return x * w - f25_mulhi(x, wq) * F25_Q;
}

// Plain modular arithmetic for tables and constants (host and constexpr).
F25_CX uint32_t f25_mulmod(uint32_t a, uint32_t b) { return (uint32_t)((uint64_t)a * b % F25_Q); }
F25_CX uint32_t f25_pow(uint32_t a, uint64_t e) {
    uint32_t r = 1;
    while (e) {
        if (e & 1) r = f25_mulmod(r, a);
        a = f25_mulmod(a, a);
        e >>= 1;
    }
    return r;
}
// Montgomery form w 2^32 mod q.
F25_CX uint32_t f25_to_mont(uint32_t w) { return (uint32_t)(((uint64_t)w << 32) % F25_Q); }
// Shoup quotient floor(w 2^32 / q) of a canonical w.
F25_CX uint32_t f25_shoup_q(uint32_t w) { return (uint32_t)(((uint64_t)w << 32) / F25_Q); }
// omega_32^j (plain, canonical): the roots inside register sub-transforms.
F25_CX uint32_t f25_w32(int j) { return f25_pow(f25_pow(F25_G25, 1ull << 20), (uint64_t)j); }
// Root of order 2^25 (or its inverse).
F25_CX uint32_t f25_root_2_25(bool inverse) {
    return inverse ? f25_pow(F25_G25, (1ull << 25) - 1) : F25_G25;
}
// L^-1 2^64 mod q for L = 2^k <= 2^25: mont(mont(a, b), c) = a b L^-1.
F25_CX uint32_t f25_linv_mont2(uint64_t L) {
    return f25_to_mont(f25_to_mont(f25_pow((uint32_t)(L % F25_Q), F25_Q - 2)));
}
// The Shoup pair of L^-1 2^32 mod q (low word: the root, high word: its
// quotient): shoup(mont(a, b), pair) = a b L^-1.
F25_CX uint64_t f25_linv_shoup(uint64_t L) {
    return (uint64_t)f25_to_mont(f25_pow((uint32_t)(L % F25_Q), F25_Q - 2)) |
           ((uint64_t)f25_shoup_q(f25_to_mont(f25_pow((uint32_t)(L % F25_Q), F25_Q - 2))) << 32);
}

#ifdef __CUDACC__
// Constant-bank copies of omega_32^j and their Shoup quotients.
#define F25_W(j) f25_w32(j)
#define F25_WQ(j) f25_shoup_q(f25_w32(j))
static __constant__ uint32_t kF25W32[32] = {
    F25_W(0),  F25_W(1),  F25_W(2),  F25_W(3),  F25_W(4),  F25_W(5),  F25_W(6),  F25_W(7),
    F25_W(8),  F25_W(9),  F25_W(10), F25_W(11), F25_W(12), F25_W(13), F25_W(14), F25_W(15),
    F25_W(16), F25_W(17), F25_W(18), F25_W(19), F25_W(20), F25_W(21), F25_W(22), F25_W(23),
    F25_W(24), F25_W(25), F25_W(26), F25_W(27), F25_W(28), F25_W(29), F25_W(30), F25_W(31)};
static __constant__ uint32_t kF25W32Q[32] = {
    F25_WQ(0),  F25_WQ(1),  F25_WQ(2),  F25_WQ(3),  F25_WQ(4),  F25_WQ(5),  F25_WQ(6),  F25_WQ(7),
    F25_WQ(8),  F25_WQ(9),  F25_WQ(10), F25_WQ(11), F25_WQ(12), F25_WQ(13), F25_WQ(14), F25_WQ(15),
    F25_WQ(16), F25_WQ(17), F25_WQ(18), F25_WQ(19), F25_WQ(20), F25_WQ(21), F25_WQ(22), F25_WQ(23),
    F25_WQ(24), F25_WQ(25), F25_WQ(26), F25_WQ(27), F25_WQ(28), F25_WQ(29), F25_WQ(30), F25_WQ(31)};
#undef F25_W
#undef F25_WQ
#endif
