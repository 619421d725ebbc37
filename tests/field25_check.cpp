// CPU check of the lazily reduced field routines (q = 5 * 2^25 + 1) against
// plain 64-bit modular arithmetic, the field's defining properties and the
// value ranges the transform kernels rely on.
#include <stdint.h>
#include <stdio.h>

#include "f25.cuh"

static const uint64_t Q = 5ull * (1ull << 25) + 1;

static uint64_t st = 0x2500000001ull;
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
    // q is prime (trial division), 3 generates F_q^* (q - 1 = 5 * 2^25), and
    // 25 q < 2^32 < 26 q (the headroom of the lazy butterflies)
    for (uint64_t d = 2; d * d <= Q; ++d)
        if (Q % d == 0) bad |= fail("prime", Q, d, 0, 1);
    if (pw(3, (Q - 1) / 2) == 1 || pw(3, (Q - 1) / 5) == 1) bad |= fail("generator", 3, 0, 0, 1);
    if (!(25 * Q < (1ull << 32) && 26 * Q > (1ull << 32))) bad |= fail("headroom", Q, 0, 0, 0);
    if (F25_G25 != pw(3, 5) || pw(F25_G25, 1ull << 25) != 1 || pw(F25_G25, 1ull << 24) != Q - 1)
        bad |= fail("g25", F25_G25, 0, 0, 1);
    if ((uint64_t)F25_Q != Q || (uint32_t)(F25_QINV * F25_Q) != 1u || F25_R != (1ull << 32) % Q ||
        F25_MU != (1ull << 32) / Q)
        bad |= fail("constants", F25_Q, F25_QINV, 0, 0);
    const uint64_t rinv = pw(1ull << 32, Q - 2);
    const uint64_t edge[] = {0, 1, 2, Q - 1, Q, 2 * Q - 1, 12 * Q, 25 * Q, (1ull << 31) - 1, (1ull << 32) - 1};
    for (int i = 0; i < 2000000 && !bad; ++i) {
        const uint64_t x = i < 100 ? edge[i % 10] : rnd() >> 32;  // any 32-bit word
        const uint64_t c = i < 100 ? edge[i / 10] % Q : rnd() % Q;  // canonical
        const uint64_t e = i < 100 ? edge[i % 10] % (2 * Q) : rnd() % (2 * Q), f = rnd() % (2 * Q);
        const uint64_t r = f25_red((uint32_t)x);
        if (r >= 2 * Q || r % Q != x % Q) bad |= fail("red", x, 0, r, x % Q);
        if (f25_canon((uint32_t)x) != x % Q) bad |= fail("canon", x, 0, f25_canon((uint32_t)x), x % Q);
        const uint64_t ad = f25_add((uint32_t)e, (uint32_t)f), sb = f25_sub((uint32_t)e, (uint32_t)f);
        if (ad >= 2 * Q || ad % Q != (e + f) % Q) bad |= fail("add", e, f, ad, (e + f) % Q);
        if (sb >= 2 * Q || sb % Q != (e % Q + Q - f % Q) % Q) bad |= fail("sub", e, f, sb, 0);
        // Montgomery: any x with a canonical root, x < 2^31 with a root in [0, 2q)
        const uint64_t mo = f25_mont((uint32_t)x, (uint32_t)c), mw = x % Q * c % Q * rinv % Q;
        if (mo == 0 || mo >= 2 * Q || mo % Q != mw) bad |= fail("mont", x, c, mo, mw);
        const uint64_t x31 = x >> 1;
        const uint64_t m2 = f25_mont((uint32_t)x31, (uint32_t)f), m2w = x31 % Q * (f % Q) % Q * rinv % Q;
        if (m2 >= 2 * Q || m2 % Q != m2w) bad |= fail("mont2q", x31, f, m2, m2w);
        // Shoup product with a canonical root
        const uint64_t sh = f25_shoup((uint32_t)x, (uint32_t)c, f25_shoup_q((uint32_t)c));
        if (sh >= 2 * Q || sh % Q != x % Q * c % Q) bad |= fail("shoup", x, c, sh, x % Q * c % Q);
        // Montgomery twiddles: mont(x, w R) = x w
        if (f25_mont((uint32_t)x, f25_to_mont((uint32_t)c)) % Q != x % Q * c % Q) bad |= fail("to_mont", x, c, 0, 0);
    }
    // sub-transform roots omega_32^j, omega_32 of order 32
    const uint64_t w32 = pw(F25_G25, 1ull << 20);
    if (pw(w32, 16) != Q - 1) bad |= fail("omega_32", w32, 16, pw(w32, 16), Q - 1);
    for (int j = 0; j < 32; ++j)
        if (f25_w32(j) != pw(w32, j)) bad |= fail("w32", j, 0, f25_w32(j), pw(w32, j));
    // L^-1 R^2 for the pointwise product: mont(mont(a, b), c) = a b / L
    for (int lg = 0; lg <= 25; ++lg) {
        const uint64_t L = 1ull << lg, a = rnd() % (2 * Q), b = rnd() % (12 * Q);
        const uint32_t c = f25_linv_mont2(L);
        const uint64_t want = a % Q * (b % Q) % Q * pw(L, Q - 2) % Q;
        const uint32_t got = f25_mont(f25_mont((uint32_t)a, (uint32_t)b), c);
        if (got >= 2 * Q || got % Q != want) bad |= fail("linv", L, a, got, want);
    }
    if (f25_mulmod(f25_root_2_25(true), f25_root_2_25(false)) != 1) bad |= fail("inverse root", 0, 0, 0, 1);
    if (!bad) printf("field25_check: ok\n");
    return bad;
}
