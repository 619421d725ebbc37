// CPU check of the 32-bit field routines (q = 3 * 2^30 + 1) against plain
// 64-bit modular arithmetic and the field's defining properties.
#include <stdint.h>
#include <stdio.h>

#include "f30.cuh"

static const uint64_t Q = 3ull * (1ull << 30) + 1;

static uint64_t st = 0x3000000001ull;
static uint64_t rnd() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static uint64_t pw(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    a %= Q;
    while (e) {
        if (e & 1) r = r * a % Q;
        a = a * a % Q;
        e >>= 1;
    }
    return r;
}
static int fail(const char *what, uint64_t a, uint64_t b, uint64_t got, uint64_t want) {
    printf("FAIL %s a=%llu b=%llu got=%llu want=%llu\n", what, (unsigned long long)a, (unsigned long long)b,
           (unsigned long long)got, (unsigned long long)want);
    return 1;
}

int main() {
    int bad = 0;
    // q is prime (trial division) and 5 generates F_q^* (q - 1 = 3 * 2^30)
    for (uint64_t d = 2; d * d <= Q; ++d)
        if (Q % d == 0) bad |= fail("prime", Q, d, 0, 1);
    if (pw(5, (Q - 1) / 2) == 1 || pw(5, (Q - 1) / 3) == 1) bad |= fail("generator", 5, 0, 0, 1);
    // g30 = 125 has order exactly 2^30
    if (F30_G30 != pw(5, 3) || pw(F30_G30, 1ull << 30) != 1 || pw(F30_G30, 1ull << 29) != Q - 1)
        bad |= fail("g30", F30_G30, 0, 0, 1);
    if ((uint64_t)F30_Q != Q || (uint32_t)(F30_QINV * F30_Q) != 1u || F30_R != (1ull << 32) % Q)
        bad |= fail("constants", F30_Q, F30_QINV, 0, 0);
    const uint64_t rinv = pw(1ull << 32, Q - 2);
    const uint64_t edge[] = {0, 1, 2, Q - 1, Q - 2, 1ull << 31, (1ull << 31) - 1, (1ull << 32) % Q};
    for (int i = 0; i < 400000 && !bad; ++i) {
        const uint64_t a = i < 64 ? edge[i % 8] : rnd() % Q, b = i < 64 ? edge[i / 8] : rnd() % Q;
        if (f30_add((uint32_t)a, (uint32_t)b) != (a + b) % Q)
            bad |= fail("add", a, b, f30_add((uint32_t)a, (uint32_t)b), (a + b) % Q);
        if (f30_sub((uint32_t)a, (uint32_t)b) != (a + Q - b) % Q)
            bad |= fail("sub", a, b, f30_sub((uint32_t)a, (uint32_t)b), (a + Q - b) % Q);
        const uint64_t mont = a * b % Q * rinv % Q;
        if (f30_mont((uint32_t)a, (uint32_t)b) != mont) bad |= fail("mont", a, b, f30_mont((uint32_t)a, (uint32_t)b), mont);
        // Montgomery twiddles: mont(x, w R) = x w
        const uint64_t w = rnd() % Q;
        if (f30_mont((uint32_t)a, f30_to_mont((uint32_t)w)) != a * w % Q) bad |= fail("to_mont", a, w, 0, a * w % Q);
    }
    // sub-transform twiddles omega_32^j R, omega_32 of order 32
    const uint64_t w32 = pw(F30_G30, 1ull << 25);
    if (pw(w32, 16) != Q - 1) bad |= fail("omega_32", w32, 16, pw(w32, 16), Q - 1);
    for (int j = 0; j < 32; ++j)
        if (f30_tw32(j) != pw(w32, j) * ((1ull << 32) % Q) % Q) bad |= fail("tw32", j, 0, f30_tw32(j), 0);
    // L^-1 R^2 for the pointwise product: mont(mont(a, b), c) = a b / L
    for (int lg = 0; lg <= 30; ++lg) {
        const uint64_t L = 1ull << lg, a = rnd() % Q, b = rnd() % Q;
        const uint32_t c = f30_linv_mont2(L);
        const uint64_t want = a * b % Q * pw(L, Q - 2) % Q;
        if (f30_mont(f30_mont((uint32_t)a, (uint32_t)b), c) != want) bad |= fail("linv", L, a, 0, want);
    }
    if (f30_mulmod(f30_root_2_30(true), f30_root_2_30(false)) != 1) bad |= fail("inverse root", 0, 0, 0, 1);
    if (!bad) printf("field30_check: ok\n");
    return bad;
}
