// Bit-packed NTT extractor on the host CPU: the CPU baseline the GPU path is
// timed against.
//
// It computes what the GPU path computes, the Toeplitz, Circulant and Dodis et
// al. extractors as an exact integer cyclic convolution (Thm. convolution) by a
// number-theoretic transform (Def. ntt), reduced mod 2, written as the paper's
// own implementation is described (Section "Performance": a C++ NTT over the
// field of 3 * 2^30 + 1, one transform per extraction) and made competent for
// a multicore host: radix-2 decimation in frequency forward (natural order in,
// bit-reversed out) and its exact inverse by decimation in time (bit-reversed
// in, natural out), so no reordering pass is needed; Shoup products with
// precomputed quotients; the first stages breadth-first over all threads, the
// rest depth-first on blocks of 2^13 elements that stay in cache; bits
// unpacked straight into the transform arrays and the window's parities packed
// straight into output words.  It shares no code with the GPU library.
//
// Build: g++ -O3 -std=c++20 -pthread -shared -fPIC (cpu_ntt/__init__.py).
#include <stdint.h>
#include <string.h>

#include <barrier>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using u64 = uint64_t;
using u128 = unsigned __int128;

constexpr u64 kP = 3221225473ull;  // 3 * 2^30 + 1
constexpr u64 kGen = 5;            // generates the multiplicative group
constexpr int kMaxLg = 30;         // 2^30 divides kP - 1
constexpr int kBlockLg = 13;       // depth-first blocks of 2^13 elements (64 KiB)

u64 mulmod(u64 a, u64 b) { return (u64)((u128)a * b % kP); }
u64 powmod(u64 a, u64 e) {
    u64 r = 1;
    for (; e; e >>= 1, a = mulmod(a, a))
        if (e & 1) r = mulmod(r, a);
    return r;
}

// A root with its Shoup quotient floor(w 2^64 / p): x w mod p in [0, 2p) for
// any 64-bit x, by one high and two low products and no division.
struct Root {
    u64 w, q;
};
Root root_of(u64 w) { return {w, (u64)(((u128)w << 64) / kP)}; }
inline u64 shoup(u64 x, const Root &r) { return x * r.w - (u64)(((u128)x * r.q) >> 64) * kP; }
inline u64 fold(u64 x) { return x >= 2 * kP ? x - 2 * kP : x; }  // [0, 4p) -> [0, 2p)

// Roots of a transform of length 2^lg: the stage of half-size h uses
// omega_(2h)^j, j < h, stored at [h + j] (h = 1 .. 2^(lg-1)); fwd for the
// forward transform, inv (omega^-1) for the inverse.
struct Tables {
    int lg = -1;
    std::vector<Root> fwd, inv;
};

Tables &tables_for(int lg) {
    static std::mutex mu;
    static Tables cache[kMaxLg + 1];
    std::lock_guard<std::mutex> g(mu);
    Tables &t = cache[lg];
    if (t.lg == lg) return t;
    const u64 L = 1ull << lg;
    t.fwd.assign(L, Root{0, 0});
    t.inv.assign(L, Root{0, 0});
    if (L >= 2) {
        // the top stage (h = L / 2) directly, lower stages by striding it:
        // omega_(2h)^j = omega_L^(j L / (2h))
        const u64 h = L / 2;
        const u64 w = powmod(kGen, (kP - 1) >> lg), wi = powmod(w, kP - 2);
        u64 a = 1, b = 1;
        for (u64 j = 0; j < h; ++j) {
            t.fwd[h + j] = root_of(a);
            t.inv[h + j] = root_of(b);
            a = mulmod(a, w);
            b = mulmod(b, wi);
        }
        for (u64 hh = h / 2; hh >= 1; hh /= 2)
            for (u64 j = 0; j < hh; ++j) {
                t.fwd[hh + j] = t.fwd[h + j * (h / hh)];
                t.inv[hh + j] = t.inv[h + j * (h / hh)];
            }
    }
    t.lg = lg;
    return t;
}

// Butterflies of one forward stage (half-size h = 2^lh) with indices
// [b0, b1) of the L / 2 of the stage; values in [0, 2p) stay there.
inline void dif_range(u64 *a, int lh, const Root *tw, u64 b0, u64 b1) {
    const u64 h = 1ull << lh;
    for (u64 b = b0; b < b1; ++b) {
        const u64 j = b & (h - 1);
        u64 *x = a + ((b >> lh) << (lh + 1)) + j;
        const u64 u = x[0], v = x[h];
        x[0] = fold(u + v);
        x[h] = shoup(u - v + 2 * kP, tw[h + j]);
    }
}
inline void dit_range(u64 *a, int lh, const Root *tw, u64 b0, u64 b1) {
    const u64 h = 1ull << lh;
    for (u64 b = b0; b < b1; ++b) {
        const u64 j = b & (h - 1);
        u64 *x = a + ((b >> lh) << (lh + 1)) + j;
        const u64 u = x[0], t = shoup(x[h], tw[h + j]);
        x[0] = fold(u + t);
        x[h] = fold(u - t + 2 * kP);
    }
}
// All stages of half-size < 2^top on one block of 2^top elements.
inline void dif_block(u64 *a, int top, const Root *tw) {
    for (int lh = top - 1; lh >= 0; --lh) dif_range(a, lh, tw, 0, 1ull << (top - 1));
}
inline void dit_block(u64 *a, int top, const Root *tw) {
    for (int lh = 0; lh < top; ++lh) dit_range(a, lh, tw, 0, 1ull << (top - 1));
}
// Canonical value of x in [0, 2p); a b mod p for a, b in [0, 2p) by Barrett's
// method (a b < 2^64 once both are canonical; mu = floor(2^64 / p)).
inline u64 canon(u64 x) { return x >= kP ? x - kP : x; }
constexpr u64 kMu = (u64)(((u128)1 << 64) / kP);
inline u64 mulmod_b(u64 a, u64 b) {
    const u64 ab = canon(a) * canon(b);
    const u64 r = ab - (u64)(((u128)ab * kMu) >> 64) * kP;
    return canon(r);
}

struct Job {
    int kind;
    const u64 *x, *y;
    u64 n, m, *z;
    u64 K, L, N2;  // terms of a, transform length, length of b
    int lg;
    std::vector<u64> A, B;
};

inline u64 bit(const u64 *s, u64 i) { return (s[i >> 6] >> (i & 63)) & 1ull; }

// The operand maps (the middle product z_i = sum_{t<K} a_t b_{t+i} read off
// positions K - 1 .. K + m - 2 of the cyclic convolution of rev(a) and b).
inline u64 a_rev(const Job &j, u64 u) {
    if (u >= j.K) return 0;
    switch (j.kind) {
        case 0: return bit(j.x, u);                                     // Toeplitz: rev(a)_u = x_u
        case 1: return (j.K - 1 - u < j.n) ? bit(j.x, j.K - 1 - u) : 0;  // Circulant: x' = [x, 0]
        default: return bit(j.x, j.K - 1 - u);                           // Dodis et al.
    }
}
inline u64 b_at(const Job &j, u64 k) {
    if (k >= j.N2) return 0;
    switch (j.kind) {
        case 0: {  // y[(k - n + 1) mod (n + m - 1)] = y[(k + m) mod (n + m - 1)]
            const u64 N = j.n + j.m - 1;
            u64 i = k + j.m % N;
            if (i >= N) i -= N;
            return bit(j.y, i);
        }
        default: return bit(j.y, k % j.K);  // y[k mod P]
    }
}

void run(Job &j, int threads) {
    Tables &tb = tables_for(j.lg);
    const u64 L = j.L, half = L / 2;
    const int top = j.lg < kBlockLg ? j.lg : kBlockLg;
    const u64 nblk = L >> top;
    std::barrier<> bar(threads);
    auto part = [&](u64 total, int t, u64 &b0, u64 &b1) {
        b0 = total * (u64)t / threads;
        b1 = total * (u64)(t + 1) / threads;
    };
    const u64 linv = powmod(L % kP, kP - 2);
    const Root lr = root_of(linv);
    auto worker = [&](int t) {
        u64 b0, b1;
        // unpack both operands
        part(L, t, b0, b1);
        for (u64 u = b0; u < b1; ++u) {
            j.A[u] = a_rev(j, u);
            j.B[u] = b_at(j, u);
        }
        bar.arrive_and_wait();
        // forward transforms: breadth-first stages, then depth-first blocks
        for (u64 *arr : {j.A.data(), j.B.data()}) {
            for (int lh = j.lg - 1; lh >= top; --lh) {
                part(half, t, b0, b1);
                dif_range(arr, lh, tb.fwd.data(), b0, b1);
                bar.arrive_and_wait();
            }
            part(nblk, t, b0, b1);
            for (u64 b = b0; b < b1; ++b) dif_block(arr + (b << top), top, tb.fwd.data());
            bar.arrive_and_wait();
        }
        // pointwise product times L^-1 (bit-reversed order on both sides)
        part(L, t, b0, b1);
        for (u64 u = b0; u < b1; ++u) j.A[u] = shoup(mulmod_b(j.A[u], j.B[u]), lr);
        bar.arrive_and_wait();
        // inverse: depth-first blocks, then breadth-first stages
        part(nblk, t, b0, b1);
        for (u64 b = b0; b < b1; ++b) dit_block(j.A.data() + (b << top), top, tb.inv.data());
        bar.arrive_and_wait();
        for (int lh = top; lh < j.lg; ++lh) {
            part(half, t, b0, b1);
            dit_range(j.A.data(), lh, tb.inv.data(), b0, b1);
            bar.arrive_and_wait();
        }
        // parities of positions K - 1 .. K + m - 2, 64 outputs a word
        const u64 words = (j.m + 63) / 64;
        part(words, t, b0, b1);
        for (u64 w = b0; w < b1; ++w) {
            u64 acc = 0;
            const u64 i0 = w * 64, cnt = j.m - i0 < 64 ? j.m - i0 : 64;
            for (u64 i = 0; i < cnt; ++i) acc |= (canon(j.A[j.K - 1 + i0 + i]) & 1ull) << i;
            j.z[w] = acc;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(worker, t);
    worker(0);
    for (auto &th : pool) th.join();
}

bool is_prime(u64 n) {
    if (n < 2) return false;
    for (u64 d = 2; d * d <= n; ++d)
        if (n % d == 0) return false;
    return true;
}

}  // namespace

extern "C" {

// Extraction of `kind` (0 Toeplitz, 1 Circulant, 2 Dodis et al.) with the
// lengths of the GPU library's single calls: x of n bits, y of n + m - 1
// (Toeplitz), n + 1 (Circulant, n + 1 prime) or n (Dodis et al., n prime)
// bits, z of m bits (ceil(m / 64) words written; bits past m are 0), packed
// LSB-first in 64-bit words, host memory.  threads >= 1 host threads.  Returns
// 0, or -1 for invalid lengths or a transform longer than 2^30 (this field's
// limit; the GPU library blocks longer products).  Primality is checked, not
// primitive root 2 (the extraction is defined either way).
int cpu_ntt_extract(int kind, const uint64_t *x, uint64_t n, const uint64_t *y, uint64_t m, uint64_t *z,
                    int threads) {
    if (!x || !y || !z || n == 0 || m == 0 || threads < 1 || kind < 0 || kind > 2) return -1;
    Job j;
    j.kind = kind;
    j.x = x;
    j.y = y;
    j.n = n;
    j.m = m;
    j.z = z;
    if (kind == 0) {
        j.K = n;
    } else {
        j.K = kind == 1 ? n + 1 : n;
        if (m > n || !is_prime(j.K)) return -1;
    }
    j.N2 = j.K + m - 1;
    j.lg = 1;
    while ((1ull << j.lg) < j.N2) ++j.lg;
    if (j.lg > kMaxLg) return -1;
    j.L = 1ull << j.lg;
    j.A.assign(j.L, 0);
    j.B.assign(j.L, 0);
    run(j, threads);
    return 0;
}

// Builds (and caches) the root tables of a transform of length 2^lg, so that
// a timed call does not include them.
void cpu_ntt_prepare(int lg) {
    if (lg >= 1 && lg <= kMaxLg) tables_for(lg);
}

}  // extern "C"
