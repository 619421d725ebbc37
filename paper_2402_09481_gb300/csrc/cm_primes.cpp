// Primes with 2 as a primitive root (the set N_A of the footnote to Def. ext-circ).
//
// The Circulant seed length and the Dodis et al. input length must be such a
// prime P.  P is prime by deterministic Miller-Rabin (the first twelve prime
// bases decide every P < 3.3 * 10^24); 2 is a primitive root iff
// 2^((P-1)/q) != 1 (mod P) for every prime q | P - 1, with q found by trial
// division (P - 1 <= 2^64 needs at most 2^32 trial divisors; the lengths used
// here stay below 2^33, i.e. below ~10^5 divisors).
#include <stdint.h>

#include <mutex>
#include <unordered_map>

#include "cm.h"

namespace cm {

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t n) {
    return (uint64_t)((unsigned __int128)a * b % n);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t n) {
    uint64_t r = 1 % n;
    a %= n;
    while (e) {
        if (e & 1) r = mulmod(r, a, n);
        a = mulmod(a, a, n);
        e >>= 1;
    }
    return r;
}

static bool is_prime_u64(uint64_t n) {
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t p : bases) {
        if (n % p == 0) return n == p;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    for (uint64_t a : bases) {
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

static bool na_uncached(uint64_t P) {
    if (P < 3 || !is_prime_u64(P)) return false;
    uint64_t r = P - 1;
    for (uint64_t q = 2; q <= r / q; q += (q == 2 ? 1 : 2)) {
        if (r % q == 0) {
            if (powmod(2, (P - 1) / q, P) == 1) return false;
            while (r % q == 0) r /= q;
        }
    }
    if (r > 1 && powmod(2, (P - 1) / r, P) == 1) return false;
    return true;
}

bool is_prime(uint64_t n) { return is_prime_u64(n); }

bool is_na_prime(uint64_t P) {
    static std::mutex mu;
    static std::unordered_map<uint64_t, bool> cache;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(P);
        if (it != cache.end()) return it->second;
    }
    const bool v = na_uncached(P);
    std::lock_guard<std::mutex> g(mu);
    if (cache.size() > 4096) cache.clear();
    cache[P] = v;
    return v;
}

}  // namespace cm

extern "C" int cm_is_na_prime(uint64_t P) { return cm::is_na_prime(P) ? 1 : 0; }

extern "C" uint64_t cm_next_na_prime(uint64_t n) {
    uint64_t P = n < 3 ? 3 : n;
    for (; P < (1ull << 63); ++P)
        if (cm::na_uncached(P)) return P;
    return 0;
}

extern "C" uint64_t cm_prev_na_prime(uint64_t n) {
    for (uint64_t P = n; P >= 3; --P)
        if (cm::na_uncached(P)) return P;
    return 0;
}
