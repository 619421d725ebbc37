// Output-length bounds and N_A length planning (host arithmetic).
//
// Each bound is one of the paper's theorems (Section "Library in detail",
// summarised by Fig. Table) evaluated in double precision; the floor is taken
// last.  The Markov-model bounds for Dodis et al. and Trevisan come from
// Thm. Markov2 applied to the classical two-source bound (final error
// eps = sqrt(3 eps0 2^(m-2)), entropies lowered by log2(1/eps0)); the
// paper prints them in closed form and the closed forms are used here.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "cm.h"
#include "cm_params.h"

namespace cm {
bool is_prime(uint64_t n);
bool is_na_prime(uint64_t P);
}  // namespace cm

namespace {

const double kE = 2.718281828459045;  // exp(1)

bool valid_eps(double le) { return isfinite(le) && le < 0.0; }
bool valid_entropy(double k) { return isfinite(k) && k >= 0.0; }

int64_t floor_len(double v) {
    if (!(v >= 1.0)) return 0;
    if (v >= 9.2e18) return INT64_MAX;
    return (int64_t)floor(v);
}

// Largest integer m >= 1 with a*m + b*log2(m) <= rhs (a > 0, b >= 0, so the
// left side increases with m); 0 if m = 1 fails.  Doubling, then bisection.
int64_t largest_implicit(double a, double b, double rhs) {
    auto ok = [&](uint64_t m) { return a * (double)m + b * log2((double)m) <= rhs; };
    if (!ok(1)) return 0;
    uint64_t good = 1, bad = 2;
    while (ok(bad)) {
        good = bad;
        if (bad >= (1ull << 61)) return (int64_t)good;
        bad <<= 1;
    }
    while (bad - good > 1) {
        const uint64_t mid = good + (bad - good) / 2;
        if (ok(mid))
            good = mid;
        else
            bad = mid;
    }
    return (int64_t)good;
}

// Seed length the kind takes for an input of n1 bits (Toeplitz depends on m
// and is not bounded here).
uint64_t fixed_seed_len(int kind, uint64_t n1, uint64_t d) {
    switch (kind) {
        case CM_CIRCULANT: return n1 + 1;
        case CM_DODIS: return n1;
        case CM_PARAM_TREVISAN: return d;
        default: return UINT64_MAX;
    }
}

// The bound proper; arguments already validated.
int64_t bound(int kind, int model, int adversary, uint64_t n1, uint64_t d, double k1, double k2,
              double le) {
    const bool seeded = model == CM_MODEL_SEEDED;
    const bool quantum = adversary == CM_ADV_QUANTUM;
    const double n = (double)n1;
    const double l43 = log2(4.0 / 3.0);
    const double le3 = le - log2(3.0);  // Thm. Markov1: eps0 = eps / 3
    switch (kind) {
        case CM_TOEPLITZ:
            if (seeded) return floor_len(k1 + 2.0 * le);
            return floor_len(0.5 * (k1 + k2 - n + 1.0 + 2.0 * le));
        case CM_CIRCULANT:
            if (seeded) return floor_len(k1 + 2.0 * le);
            return floor_len(k1 + k2 - (n + 1.0) + 2.0 * le);
        case CM_DODIS: {
            const double kk2 = seeded ? n : k2;
            const int64_t q = floor_len((k1 + kk2 - n + 8.0 * le + 4.0 * l43 + 1.0) / 5.0);
            if (quantum) return q;
            if (seeded || model == CM_MODEL_PRODUCT) return floor_len(k1 + kk2 - n + 1.0 + 2.0 * le);
            const int64_t c = floor_len(k1 + kk2 - n + 1.0 + 4.0 * le3);
            return c > q ? c : q;
        }
        default: {  // Trevisan
            if (seeded) return largest_implicit(1.0, 4.0, k1 + 4.0 * le - 6.0);
            const double dd = (double)d;
            const int64_t q = largest_implicit(10.0, 4.0, k1 + 4.0 * (k2 - dd) + 18.0 * le + 9.0 * l43 - 6.0);
            if (quantum) return q;
            if (model == CM_MODEL_PRODUCT)
                return largest_implicit(1.0, 4.0, k1 + 4.0 * k2 - 4.0 * dd + 4.0 * le - 6.0);
            const int64_t c = largest_implicit(1.0, 4.0, k1 + 4.0 * (k2 - dd) + 9.0 * le3 - 6.0);
            return c > q ? c : q;
        }
    }
}

bool valid_enums(int kind, int model, int adversary) {
    return kind >= CM_TOEPLITZ && kind <= CM_PARAM_TREVISAN && model >= CM_MODEL_SEEDED &&
           model <= CM_MODEL_MARKOV && (adversary == CM_ADV_CLASSICAL || adversary == CM_ADV_QUANTUM);
}

}  // namespace

extern "C" cm_status cm_output_length(int kind, int model, int adversary, uint64_t n1, uint64_t d, double k1,
                                      double k2, double log2_eps, int64_t *m) {
    if (!m || !valid_enums(kind, model, adversary) || n1 == 0 || !valid_eps(log2_eps)) return CM_EINVAL;
    if (!valid_entropy(k1) || k1 > (double)n1) return CM_EINVAL;
    if (kind == CM_CIRCULANT && !cm::is_na_prime(n1 + 1)) return CM_EINVAL;
    if (kind == CM_DODIS && !cm::is_na_prime(n1)) return CM_EINVAL;
    if (model != CM_MODEL_SEEDED) {
        if (kind == CM_PARAM_TREVISAN && d == 0) return CM_EINVAL;
        if (!valid_entropy(k2) || k2 > (double)fixed_seed_len(kind, n1, d)) return CM_EINVAL;
    }
    *m = bound(kind, model, adversary, n1, d, k1, k2, log2_eps);
    return CM_OK;
}

extern "C" cm_status cm_trevisan_seed_length(uint64_t n1, uint64_t m, double log2_eps, uint64_t *t, uint64_t *a,
                                             uint64_t *d) {
    if (n1 == 0 || m == 0 || !valid_eps(log2_eps)) return CM_EINVAL;
    // q = 2 ceil(log2 n1 + 2 log2(2m/eps)), log2(2m/eps) = 1 + log2 m - log2 eps
    const double inner = log2((double)n1) + 2.0 * (1.0 + log2((double)m) - log2_eps);
    if (!(inner < 1e15)) return CM_EINVAL;
    uint64_t tt = 2 * (uint64_t)ceil(inner);
    while (!cm::is_prime(tt)) ++tt;
    uint64_t aa = 1;
    if ((double)m > 2.0 * kE) {
        const double r = (log2((double)m - 2.0 * kE) - log2((double)tt - 2.0 * kE)) /
                         (log2(2.0 * kE) - log2(2.0 * kE - 1.0));
        const double c = ceil(r);
        if (c > 1.0) aa = (uint64_t)c;
    }
    if (t) *t = tt;
    if (a) *a = aa;
    if (d) *d = aa * tt * tt;
    return CM_OK;
}

extern "C" uint64_t cm_closest_na_prime(uint64_t n) {
    const uint64_t up = cm_next_na_prime(n);
    const uint64_t down = cm_prev_na_prime(n);
    if (!down) return up;
    if (!up) return down;
    return (up - n <= n - down) ? up : down;
}

extern "C" cm_status cm_plan_params(int kind, int model, int adversary, uint64_t n_raw, double k1,
                                    double seed_rate, double log2_eps, int adjust, cm_param_plan *out) {
    if (!out || !valid_enums(kind, model, adversary) || n_raw == 0 || !valid_eps(log2_eps)) return CM_EINVAL;
    if (adjust < CM_ADJUST_UP || adjust > CM_ADJUST_CLOSEST) return CM_EINVAL;
    if (!valid_entropy(k1) || k1 > (double)n_raw) return CM_EINVAL;
    const bool seeded = model == CM_MODEL_SEEDED;
    if (!seeded && !(seed_rate > 0.0 && seed_rate <= 1.0)) return CM_EINVAL;
    if (kind == CM_PARAM_TREVISAN && !seeded) return CM_EINVAL;
    cm_param_plan p;
    memset(&p, 0, sizeof(p));
    p.n1 = n_raw;
    p.k1 = k1;
    if (kind == CM_CIRCULANT || kind == CM_DODIS) {
        // the length that must be in N_A: the seed (n_raw + 1) or the common length
        const uint64_t want = kind == CM_CIRCULANT ? n_raw + 1 : n_raw;
        const uint64_t P = adjust == CM_ADJUST_UP     ? cm_next_na_prime(want)
                           : adjust == CM_ADJUST_DOWN ? cm_prev_na_prime(want)
                                                      : cm_closest_na_prime(want);
        if (P == 0 || (kind == CM_CIRCULANT && P < 3)) return CM_EINVAL;
        if (P >= want) {
            p.pad_input = P - want;
        } else {
            p.cut_input = want - P;
            p.k1 = k1 - (double)p.cut_input;
            if (p.k1 < 0.0) p.k1 = 0.0;
        }
        p.n1 = kind == CM_CIRCULANT ? P - 1 : P;
        p.n2 = P;
        p.k2 = seeded ? (double)P : seed_rate * (double)P;
        const cm_status s = cm_output_length(kind, model, adversary, p.n1, 0, p.k1, p.k2, log2_eps, &p.m);
        if (s != CM_OK) return s;
    } else if (kind == CM_TOEPLITZ) {
        if (seeded) {
            p.m = bound(kind, model, adversary, p.n1, 0, k1, 0.0, log2_eps);
        } else {
            // m <= k1 + (r - 1)(n1 + m - 1) + 2 log2 eps, linear in m
            const double r = seed_rate, n = (double)p.n1;
            auto ok = [&](int64_t m) { return (double)m <= k1 + (r - 1.0) * (n + (double)m - 1.0) + 2.0 * log2_eps; };
            int64_t m = floor_len((k1 + (r - 1.0) * (n - 1.0) + 2.0 * log2_eps) / (2.0 - r));
            while (m > 0 && !ok(m)) --m;
            while (ok(m + 1)) ++m;
            p.m = m;
        }
        p.n2 = p.m > 0 ? p.n1 + (uint64_t)p.m - 1 : 0;
        p.k2 = seeded ? (double)p.n2 : seed_rate * (double)p.n2;
    } else {  // Trevisan, seeded
        p.m = bound(kind, model, adversary, p.n1, 0, k1, 0.0, log2_eps);
        if (p.m > 0) {
            const cm_status s = cm_trevisan_seed_length(p.n1, (uint64_t)p.m, log2_eps, nullptr, nullptr, &p.n2);
            if (s != CM_OK) return s;
        }
        p.k2 = (double)p.n2;
    }
    *out = p;
    return CM_OK;
}
