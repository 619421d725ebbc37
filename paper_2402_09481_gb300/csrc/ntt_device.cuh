// Device building blocks of the GF(2) extractor path: bit maps, on-chip NTT
// networks over shared memory, and the Goldilocks twiddle lookups.
//
// Every extraction is one GF(2) "middle product"
//     z_i = sum_{t<K} a_t b_{t+i}  (mod 2),  i < m,  |b| = K + m - 1,
// read off positions K-1 .. K+m-2 of the length-L cyclic convolution of
// rev(a) and b (Thm. convolution), L a power of two >= K + m - 1.  The NTT is
// the DFT over F_p of Def. ntt.  The three extractors differ only in how a and b
// are read out of the packed input bits (see BitMap).
#pragma once
#include <stdint.h>
#include "gl.cuh"

namespace cm {

constexpr int kThreads = 512;     // threads per CTA for every NTT kernel
constexpr int kMidLgMax = 13;     // fused on-chip block: 2 operands x 2^13 x 8 B
constexpr int kTileLg = 14;       // column-pass tile: 2^14 elements (128 KiB)
constexpr int kSmallLg = 13;      // root table omega_{2^13}^e, e < 2^12

// Shared-memory index with one pad word per 32 (breaks power-of-two strides).
__device__ __forceinline__ int sp(int i) { return i + (i >> 5); }
__host__ __device__ constexpr int sp_size(int n) { return n + (n >> 5) + 1; }

struct RootTables {
    const uint64_t *small_fwd;   // omega_{8192}^e,  e < 4096
    const uint64_t *small_inv;   // omega_{8192}^-e
    const uint64_t *big_lo_fwd;  // g^e,            e < 2^16, g of order 2^32
    const uint64_t *big_hi_fwd;  // g^(2^16 e),     e < 2^16
    const uint64_t *big_lo_inv;
    const uint64_t *big_hi_inv;
};

// g^(E) for E < 2^32, g the fixed root of order 2^32.
__device__ __forceinline__ uint64_t big_root(const uint64_t *lo, const uint64_t *hi, uint32_t E) {
    return gl_mul(__ldg(hi + (E >> 16)), __ldg(lo + (E & 0xFFFFu)));
}

// ---------------------------------------------------------------------------
// Packed-bit operand maps.  Bit i of a bit string is word i >> 6, position i & 63.
// value(k), k in [0, L): 0 beyond len; otherwise the source bit at idx(k):
//   kModForward: idx = (k + off) mod srclen   (b of every extractor)
//   kReverse:    idx = off - k, 0 if idx >= srclen (rev(a) for Circulant/Dodis;
//                the Circulant pad bit x'_{P-1} = 0 falls out at k = 0)
//   kIdentity:   idx = k                      (rev(a) = x for Toeplitz)
// ---------------------------------------------------------------------------
enum MapMode : int { kIdentity = 0, kModForward = 1, kReverse = 2 };

struct BitMap {
    const uint64_t *src;
    uint64_t len;     // number of non-zero-padded positions
    uint64_t srclen;  // bits in src
    uint64_t off;
    int mode;

    __device__ __forceinline__ uint64_t get(uint64_t k) const {
        if (k >= len) return 0;
        uint64_t idx;
        if (mode == kIdentity) {
            idx = k;
        } else if (mode == kModForward) {
            idx = k + off;
            if (idx >= srclen) idx -= srclen;
        } else {
            idx = off - k;
            if (idx >= srclen) return 0;
        }
        return (__ldg(src + (idx >> 6)) >> (idx & 63)) & 1ull;
    }
};

// ---------------------------------------------------------------------------
// Radix-2 decimation-in-frequency network on NCOL interleaved columns of length
// R = 2^LOGR stored in shared memory (element (i, c) at sp(i * NCOL + c)),
// natural order in, bit-reversed order out.  Stages are grouped: each thread
// loads 2^Q elements of one column, runs Q stages in registers and writes back.
// Stage s pairs i and i + h, h = R >> (s + 1), as (a, b) -> (a + b, (a - b) w),
// w = omega_{2h}^(i mod h) = omega_R^((i mod h) 2^s).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ntt_nsteps(int logr) { return (logr + 3) / 4; }
__host__ __device__ constexpr int ntt_q(int logr, int step) {
    // split logr into ntt_nsteps(logr) parts, larger parts first
    return logr / ntt_nsteps(logr) + (step < logr % ntt_nsteps(logr) ? 1 : 0);
}
__host__ __device__ constexpr int ntt_s0(int logr, int step) {
    return step == 0 ? 0 : ntt_s0(logr, step - 1) + ntt_q(logr, step - 1);
}

template <int LOGR, int S0, int Q, int NCOL_LG, int NBUF>
__device__ __forceinline__ void dif_step(uint64_t *s0, uint64_t *s1, const uint64_t *__restrict__ tw) {
    constexpr int R = 1 << LOGR;
    constexpr int HL = R >> (S0 + Q);
    constexpr int NG = R >> Q;
    constexpr int TWS_LG = kSmallLg - LOGR;  // omega_R = omega_8192^(2^TWS_LG)
    constexpr int ITEMS = NG << NCOL_LG;
    for (int item = threadIdx.x; item < ITEMS * NBUF; item += kThreads) {
        const int bi = item / ITEMS;
        const int it = item - bi * ITEMS;
        uint64_t *s = (NBUF == 2 && bi) ? s1 : s0;
        const int c = it & ((1 << NCOL_LG) - 1);
        const int g = it >> NCOL_LG;
        const int blk = g / HL, off = g - blk * HL;
        const int base = blk * (R >> S0) + off;
        uint64_t v[1 << Q];
#pragma unroll
        for (int t = 0; t < (1 << Q); ++t) v[t] = s[sp(((base + t * HL) << NCOL_LG) + c)];
#pragma unroll
        for (int st = 0; st < Q; ++st) {
            const int span = 1 << (Q - 1 - st);
            const int h = R >> (S0 + st + 1);
#pragma unroll
            for (int t = 0; t < (1 << Q); ++t) {
                if (t & span) continue;
                const int pos = (off + t * HL) & (h - 1);
                const uint64_t w = __ldg(tw + ((pos << (S0 + st)) << TWS_LG));
                const uint64_t a = v[t], b = v[t + span];
                v[t] = gl_add(a, b);
                v[t + span] = gl_mul(gl_sub(a, b), w);
            }
        }
#pragma unroll
        for (int t = 0; t < (1 << Q); ++t) s[sp(((base + t * HL) << NCOL_LG) + c)] = v[t];
    }
}

// Inverse of dif_step (up to a factor 2 per stage) with inverse roots:
// (A, B) -> (A + B w^-1, A - B w^-1), stages in reverse order.
template <int LOGR, int S0, int Q, int NCOL_LG, int NBUF>
__device__ __forceinline__ void dit_step(uint64_t *s0, uint64_t *s1, const uint64_t *__restrict__ twi) {
    constexpr int R = 1 << LOGR;
    constexpr int HL = R >> (S0 + Q);
    constexpr int NG = R >> Q;
    constexpr int TWS_LG = kSmallLg - LOGR;
    constexpr int ITEMS = NG << NCOL_LG;
    for (int item = threadIdx.x; item < ITEMS * NBUF; item += kThreads) {
        const int bi = item / ITEMS;
        const int it = item - bi * ITEMS;
        uint64_t *s = (NBUF == 2 && bi) ? s1 : s0;
        const int c = it & ((1 << NCOL_LG) - 1);
        const int g = it >> NCOL_LG;
        const int blk = g / HL, off = g - blk * HL;
        const int base = blk * (R >> S0) + off;
        uint64_t v[1 << Q];
#pragma unroll
        for (int t = 0; t < (1 << Q); ++t) v[t] = s[sp(((base + t * HL) << NCOL_LG) + c)];
#pragma unroll
        for (int st = Q - 1; st >= 0; --st) {
            const int span = 1 << (Q - 1 - st);
            const int h = R >> (S0 + st + 1);
#pragma unroll
            for (int t = 0; t < (1 << Q); ++t) {
                if (t & span) continue;
                const int pos = (off + t * HL) & (h - 1);
                const uint64_t w = __ldg(twi + ((pos << (S0 + st)) << TWS_LG));
                const uint64_t a = v[t], b = gl_mul(v[t + span], w);
                v[t] = gl_add(a, b);
                v[t + span] = gl_sub(a, b);
            }
        }
#pragma unroll
        for (int t = 0; t < (1 << Q); ++t) s[sp(((base + t * HL) << NCOL_LG) + c)] = v[t];
    }
}

template <int LOGR, int STEP, int NCOL_LG, int NBUF>
__device__ __forceinline__ void dif_from(uint64_t *s0, uint64_t *s1, const uint64_t *tw) {
    if constexpr (STEP < ntt_nsteps(LOGR)) {
        dif_step<LOGR, ntt_s0(LOGR, STEP), ntt_q(LOGR, STEP), NCOL_LG, NBUF>(s0, s1, tw);
        __syncthreads();
        dif_from<LOGR, STEP + 1, NCOL_LG, NBUF>(s0, s1, tw);
    }
}

template <int LOGR, int STEP, int NCOL_LG, int NBUF>
__device__ __forceinline__ void dit_from(uint64_t *s0, uint64_t *s1, const uint64_t *twi) {
    if constexpr (STEP >= 0) {
        dit_step<LOGR, ntt_s0(LOGR, STEP), ntt_q(LOGR, STEP), NCOL_LG, NBUF>(s0, s1, twi);
        __syncthreads();
        dit_from<LOGR, STEP - 1, NCOL_LG, NBUF>(s0, s1, twi);
    }
}

// Full DIF over LOGR (natural -> bit-reversed); ends with a barrier.
template <int LOGR, int NCOL_LG, int NBUF>
__device__ __forceinline__ void ntt_dif(uint64_t *s0, uint64_t *s1, const uint64_t *tw) {
    if constexpr (LOGR > 0) dif_from<LOGR, 0, NCOL_LG, NBUF>(s0, s1, tw);
}
// Full DIT over LOGR (bit-reversed -> natural); ends with a barrier.
template <int LOGR, int NCOL_LG, int NBUF>
__device__ __forceinline__ void ntt_dit(uint64_t *s0, uint64_t *s1, const uint64_t *twi) {
    if constexpr (LOGR > 0) dit_from<LOGR, ntt_nsteps(LOGR) - 1, NCOL_LG, NBUF>(s0, s1, twi);
}

__device__ __forceinline__ int bitrev(int k, int lg) {
    return lg == 0 ? 0 : (int)(__brev((unsigned)k) >> (32 - lg));
}

}  // namespace cm
