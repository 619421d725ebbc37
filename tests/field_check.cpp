// CPU check of the Goldilocks host/device arithmetic against 128-bit integers.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "gl.cuh"

typedef unsigned __int128 u128;
static const u128 P = ((u128)1 << 64) - ((u128)1 << 32) + 1;

static uint64_t st = 0x2402094810ull;
static uint64_t rnd() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static uint64_t canon_sample(int k) {
    static const uint64_t edge[] = {0, 1, 2, 0xFFFFFFFFull, 0x100000000ull, 0xFFFFFFFF00000000ull,
                                    GL_P - 1, GL_P - 2, 0x7FFFFFFFFFFFFFFFull, 0x8000000000000000ull};
    if (k < 10) return edge[k];
    uint64_t v = rnd();
    return v >= GL_P ? v - GL_P : v;
}
static int fail(const char *what, uint64_t a, uint64_t b, uint64_t got, uint64_t want) {
    printf("FAIL %s a=%016llx b=%016llx got=%016llx want=%016llx\n", what, (unsigned long long)a,
           (unsigned long long)b, (unsigned long long)got, (unsigned long long)want);
    return 1;
}

int main() {
    int bad = 0;
    for (int i = 0; i < 200000 && !bad; ++i) {
        const uint64_t a = canon_sample(i % 10 == i ? i : (i < 100 ? i % 10 : 10));
        const uint64_t b = canon_sample(i < 100 ? (i / 10) : 10);
        const uint64_t add = (uint64_t)(((u128)a + b) % P);
        const uint64_t sub = (uint64_t)(((u128)a + P - b) % P);
        const uint64_t mul = (uint64_t)(((u128)a * b) % P);
        if (gl_add(a, b) != add) bad |= fail("add", a, b, gl_add(a, b), add);
        if (gl_sub(a, b) != sub) bad |= fail("sub", a, b, gl_sub(a, b), sub);
        if (gl_mul_host(a, b) != mul) bad |= fail("mul", a, b, gl_mul_host(a, b), mul);
        for (int s = 0; s <= 96 && !bad; ++s) {
            u128 w = 1;
            for (int k = 0; k < s; ++k) w = (w * 2) % P;
            const uint64_t want = (uint64_t)((u128)a * w % P);
            const uint64_t got = gl_shl(a, s);
            if (got != want) bad |= fail("shl", a, (uint64_t)s, got, want);
        }
        // full 128-bit reduction of arbitrary inputs
        const uint64_t lo = rnd(), hi = rnd();
        const uint64_t want = (uint64_t)((((u128)hi << 64) | lo) % P);
        if (gl_reduce128(lo, hi) != want) bad |= fail("reduce128", lo, hi, gl_reduce128(lo, hi), want);
    }
    // root structure: g of order 2^32 with g^(2^26) = 8
    const uint64_t g = gl_root_2_32_host(0), gi = gl_root_2_32_host(1);
    if (gl_pow_host(g, 1ull << 26) != 8) bad |= fail("omega64", g, 0, gl_pow_host(g, 1ull << 26), 8);
    if (gl_pow_host(g, 1ull << 31) != GL_P - 1) bad |= fail("order", g, 0, 0, 0);
    if (gl_mul_host(g, gi) != 1) bad |= fail("inverse", g, gi, gl_mul_host(g, gi), 1);
    for (int k = 1; k <= 32; ++k) {
        const uint64_t L = 1ull << k;
        if (gl_mul_host(gl_inv_pow2_host(L), L % GL_P) != 1) bad |= fail("Linv", L, 0, 0, 1);
    }
    printf(bad ? "field_check: FAILED\n" : "field_check: ok\n");
    return bad;
}
