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
#include "f25.cuh"
#include "f30.cuh"
#include "gl.cuh"

namespace cm {

constexpr int kThreads = 512;     // threads per CTA for every NTT kernel
constexpr int kMidLgMax = 13;     // fused on-chip block: 2 operands x 2^13 x 8 B
constexpr int kTileLg = 14;       // column-pass tile: 2^14 elements (128 KiB)
constexpr int kSmallLg = 13;      // root table omega_{2^13}^e, e < 2^13

// Shared-memory index with one pad word per 32 (breaks power-of-two strides).
__device__ __forceinline__ int sp(int i) { return i + (i >> 5); }

// Position of root e in a shared-memory root table.  Lookups index the table
// with power-of-two strides (e = i2 k1 2^off for consecutive i2), which would
// send up to 16 lanes to one bank; XOR-ing the bank-pair bits (e & 15) with
// higher bits spreads them.  A bijection inside every aligned group of 16.
__device__ __forceinline__ int tw_swz(int e) { return e ^ (((e >> 5) ^ (e >> 9)) & 15); }
__host__ __device__ constexpr int sp_size(int n) { return n + (n >> 5) + 1; }

// Resident root tables of one field (element type T).  Goldilocks: g of order
// 2^32, 2^16-entry halves; F30: g of order 2^30, 2^15-entry halves, entries in
// Montgomery form; F25: g of order 2^25, halves of 2^13 (low) and 2^12 (high)
// entries, Montgomery form.
template <class T>
struct RootTablesT {
    const T *small;       // omega_{8192}^e,  e < 8192
    const T *big_lo_fwd;  // g^e,             e < 2^kBigLg
    const T *big_hi_fwd;  // g^(2^kBigLg e),  e < 2^kBigLg
    const T *big_lo_inv;
    const T *big_hi_inv;
    // 32-bit fields only (null for Goldilocks): the length-16 DFT of 8 input
    // bits, bits16[k * 256 + p] = sum over the set bits j of p of
    // omega_16^(j k), canonical, for the first forward step on 0/1 inputs
    // (fwd_step_f, fwd_step25).
    const T *bits16;
    // F25 only: the per-step root tables of every on-chip length 2^l
    // (l = 1 .. 13) at word 2^l (ntt25.cuh).
    const T *steps;
};
using RootTables = RootTablesT<uint64_t>;
using RootTables30 = RootTablesT<uint32_t>;
using RootTables25 = RootTablesT<uint32_t>;

// ---------------------------------------------------------------------------
// Field policies.  Every transform below is written once over a policy F:
//   FieldGL  -- Goldilocks p = 2^64 - 2^32 + 1, 64-bit words, every L <= 2^32;
//              the root of order 64 is 8 = 2^3, so register sub-transforms
//              twiddle by shifts;
//   FieldF30 -- q = 3 * 2^30 + 1 (the paper's small field), 32-bit words,
//              L <= 2^30; Montgomery products with constant twiddles;
//   FieldF25 -- q = 5 * 2^25 + 1, 32-bit words, L <= 2^25, lazy reduction
//              (f25.cuh): values between steps are any representative below
//              12 q (< 2^31), every on-chip step brings its inputs to [0, 2q)
//              (by its twiddle product or red) and its butterflies skip the
//              compare-and-select of a canonical field.
// Every policy has red (to the representative the next DFT accepts) and canon
// (to [0, q), before a parity is read); both are the identity for the
// canonical fields.
// ---------------------------------------------------------------------------
struct FieldGL {
    using T = uint64_t;
    static constexpr bool kLazy = false;
    static constexpr int kAdicity = 32;
    static constexpr int kBigLg = 16;
    // columns of a column-pass tile of 2^LOGR rows: 2^14 elements (32-byte rows
    // for LOGR = 12)
    static constexpr int ncol_lg(int logr) { return kTileLg - logr; }
    __device__ static __forceinline__ T add(T a, T b) { return gl_add(a, b); }
    __device__ static __forceinline__ T sub(T a, T b) { return gl_sub(a, b); }
    __device__ static __forceinline__ T twmul(T x, T w) { return gl_mul(x, w); }
    // x omega_{2h}^pos, h = 2^lh <= 16: omega_{2h} = 2^(96 / h)
    __device__ static __forceinline__ T rot(T x, int lh, int pos) { return gl_shl(x, (96 >> lh) * pos); }
    __device__ static __forceinline__ T prod(T a, T b, T linv) { return gl_mul(gl_mul(a, b), linv); }
    __device__ static __forceinline__ T red(T x) { return x; }
    __device__ static __forceinline__ T canon(T x) { return x; }
};

struct FieldF30 {
    using T = uint32_t;
    static constexpr bool kLazy = false;
    static constexpr int kAdicity = 30;
    static constexpr int kBigLg = 15;
    // 2^14-element tiles (64 KiB), so that two CTAs fit on an SM
    static constexpr int ncol_lg(int logr) { return kTileLg - logr; }
    __device__ static __forceinline__ T add(T a, T b) { return f30_add(a, b); }
    __device__ static __forceinline__ T sub(T a, T b) { return f30_sub(a, b); }
    __device__ static __forceinline__ T twmul(T x, T w) { return f30_mont(x, w); }
    __device__ static __forceinline__ T rot(T x, int lh, int pos) {
        return pos == 0 ? x : f30_mont(x, kF30Tw32[(16 >> lh) * pos]);
    }
    __device__ static __forceinline__ T prod(T a, T b, T linv) { return f30_mont(f30_mont(a, b), linv); }
    __device__ static __forceinline__ T red(T x) { return x; }
    __device__ static __forceinline__ T canon(T x) { return x; }
};

struct FieldF25 {
    using T = uint32_t;
    static constexpr bool kLazy = true;
    static constexpr int kAdicity = 25;
    static constexpr int kBigLg = 13;
    static constexpr int ncol_lg(int logr) { return kTileLg - logr; }
    // a, b in [0, 2q) -> [0, 2q)
    __device__ static __forceinline__ T add(T a, T b) { return f25_add(a, b); }
    __device__ static __forceinline__ T sub(T a, T b) { return f25_sub(a, b); }
    // x w for any x < 2^31 and a table root w < 2q (canonical roots: any x) -> (0, 2q)
    __device__ static __forceinline__ T twmul(T x, T w) { return f25_mont(x, w); }
    // x omega_{2h}^pos, h = 2^lh <= 16 (Shoup product with a constant root) -> [0, 2q)
    __device__ static __forceinline__ T rot(T x, int lh, int pos) {
        return pos == 0 ? f25_red(x) : f25_shoup(x, kF25W32[(16 >> lh) * pos], kF25W32Q[(16 >> lh) * pos]);
    }
    // a b L^-1 for any a, b -> (0, 2q); linv = L^-1 2^64 mod q
    __device__ static __forceinline__ T prod(T a, T b, T linv) {
        return f25_mont(f25_mont(f25_red(a), f25_red(b)), linv);
    }
    __device__ static __forceinline__ T red(T x) { return f25_red(x); }
    __device__ static __forceinline__ T canon(T x) { return f25_canon(x); }
};

// 16 bytes as 2 x 64-bit or 4 x 32-bit elements, and back.
__device__ __forceinline__ void unpack16(uint4 v, uint64_t (&o)[2]) {
    o[0] = ((uint64_t)v.y << 32) | v.x;
    o[1] = ((uint64_t)v.w << 32) | v.z;
}
__device__ __forceinline__ void unpack16(uint4 v, uint32_t (&o)[4]) {
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
__device__ __forceinline__ uint4 pack16(const uint64_t (&o)[2]) {
    return make_uint4((uint32_t)o[0], (uint32_t)(o[0] >> 32), (uint32_t)o[1], (uint32_t)(o[1] >> 32));
}
__device__ __forceinline__ uint4 pack16(const uint32_t (&o)[4]) { return make_uint4(o[0], o[1], o[2], o[3]); }

// g^E for E < 2^kAdicity, g the field's fixed root of maximal 2-power order.
template <class F>
__device__ __forceinline__ typename F::T big_root_f(const typename F::T *lo, const typename F::T *hi, uint32_t E) {
    return F::twmul(__ldg(hi + (E >> F::kBigLg)), __ldg(lo + (E & ((1u << F::kBigLg) - 1))));
}
__device__ __forceinline__ uint64_t big_root(const uint64_t *lo, const uint64_t *hi, uint32_t E) {
    return big_root_f<FieldGL>(lo, hi, E);
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
            idx = k + off;  // k + off < 3 srclen for every plan and block
            if (idx >= srclen) idx -= srclen;
            if (idx >= srclen) idx -= srclen;
            if (idx >= srclen) return 0;  // unreachable; keeps every read in bounds
        } else {
            idx = off - k;
            if (idx >= srclen) return 0;
        }
        return (__ldg(src + (idx >> 6)) >> (idx & 63)) & 1ull;
    }

    // Values of the CNT <= 32 consecutive positions k .. k + CNT - 1 as bits
    // 0 .. CNT - 1, from one or two word loads when the run maps to a run of
    // source bits (no cut at len, no wrap, no pad bit); else position by position.
    template <int CNT>
    __device__ __forceinline__ uint32_t get_run(uint64_t k) const {
        constexpr uint64_t mask = (1ull << CNT) - 1;
        if (k + CNT <= len) {
            uint64_t lo;   // lowest source index of the run
            bool fast;
            if (mode == kIdentity) {
                lo = k;
                fast = true;
            } else if (mode == kModForward) {
                lo = k + off;
                if (lo >= srclen) lo -= srclen;
                if (lo >= srclen) lo -= srclen;
                fast = lo + CNT <= srclen;
            } else {
                const uint64_t hi = off - k;  // decreasing: hi, hi - 1, ..., hi - CNT + 1
                fast = hi < srclen && hi >= CNT - 1;
                lo = hi - (CNT - 1);
            }
            if (fast) {
                const uint64_t w = lo >> 6;
                const int sh = (int)(lo & 63);
                uint64_t r = __ldg(src + w) >> sh;
                if (sh + CNT > 64) r |= __ldg(src + w + 1) << (64 - sh);
                r &= mask;
                if (mode == kReverse) r = __brev((uint32_t)r) >> (32 - CNT);
                return (uint32_t)r;
            }
        }
        uint32_t r = 0;
#pragma unroll
        for (int j = 0; j < CNT; ++j) r |= (uint32_t)get(k + j) << j;
        return r;
    }
};

// ---------------------------------------------------------------------------
// On-chip transforms: mixed-radix decimation in frequency over shared memory.
//
// A length-R column (R = 2^LOGR) of NCOL interleaved columns lives in shared
// memory, element (i, c) at sp(i * NCOL + c).  The transform is a sequence of
// steps of radix RD_j = 2^q_j <= 32 (the four-step split of Def. ntt applied
// recursively): step j views each sub-block of N_j contiguous rows as an
// RD_j x M_j matrix (M_j = N_j / RD_j), transforms every column i2 in registers,
// multiplies output k1 by omega_{N_j}^(i2 k1) and writes it to row k1 M_j + i2,
// so that each output row k1 becomes a sub-block of the next step.  The
// in-register sub-transforms have length <= 32, so all their twiddles are
// powers of two (omega_64 = 8) and cost shifts, not multiplies; one general
// multiply per element per step remains.  The result sits in digit-reversed
// order (position -> frequency: pos_to_freq).  The inverse applies the exact
// inverse of each step in reverse order, mapping that order back to natural.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ constexpr int st_n(int logr) { return (logr + 4) / 5; }
__host__ __device__ __forceinline__ constexpr int st_q(int logr, int j) {
    return logr / st_n(logr) + (j < logr % st_n(logr) ? 1 : 0);
}
__host__ __device__ __forceinline__ constexpr int st_off(int logr, int j) {
    int o = 0;
    for (int i = 0; i < j; ++i) o += st_q(logr, i);
    return o;
}

__device__ __forceinline__ int bitrev_c(int k, int lg) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b)
        if (b < lg) r |= ((k >> b) & 1) << (lg - 1 - b);
    return r;
}

// In-register DFT of length 2^LQ <= 32 over F25 with lazy reduction: natural
// order in, v[bitrev(k)] = X[k] out, like dft_reg_f.  Cooley-Tukey butterflies
// on natural-order input: stage s (half-length len = RD / 2^(s+1)) splits each
// residue of the input polynomial modulo X^(2 len) - zeta^2 into the residues
// modulo X^len - zeta and X^len + zeta, (lo, hi) -> (lo + zeta hi, lo - zeta hi),
// where block b of the stage has zeta = omega_(2^(s+1))^bitrev_s(b); after the
// last stage position b holds the residue modulo X - omega^bitrev(b), i.e.
// X[bitrev(b)].  Inputs in [0, 2q).  A block with zeta != 1 brings
// t = zeta hi to [0, 2q) by the Shoup product and adds 2q to the bound of its
// inputs.  Block 0 (zeta = 1) adds hi unreduced, (lo + hi, lo - hi + B q) for
// inputs below B q, doubling the bound, as long as a doubled bound plus 2q per
// remaining stage stays within 24 q; otherwise it reduces hi (red) and adds 2q.
// Outputs below (f25_dft_bound(LQ)) q: 4, 8, 16, 18, 20 for LQ = 1 .. 5.
// block 0's input bound at stage s (in units of q; 2 at stage 0)
__host__ __device__ __forceinline__ constexpr int f25_b0_bound(int lq, int s) {
    int b = 2;
    for (int j = 0; j < s; ++j) b = (2 * b + 2 * (lq - 1 - j) <= 24) ? 2 * b : b + 2;
    return b;
}
__host__ __device__ __forceinline__ constexpr bool f25_b0_reduces(int lq, int s) {
    return s > 0 && 2 * f25_b0_bound(lq, s) + 2 * (lq - 1 - s) > 24;
}
__host__ __device__ constexpr int f25_dft_bound(int lq) { return f25_b0_bound(lq, lq); }
template <int LQ>
__device__ __forceinline__ void dft_reg_f25(uint32_t *v) {
    constexpr int RD = 1 << LQ;
    static_assert(LQ >= 1 && LQ <= 5, "register sub-transforms of length 2 .. 32");
    static_assert(f25_dft_bound(LQ) <= 24 && (uint64_t)f25_dft_bound(LQ) * F25_Q < (1ull << 32), "headroom");
#pragma unroll
    for (int s = 0; s < LQ; ++s) {
        const int len = RD >> (s + 1);
#pragma unroll
        for (int b = 0; b < (1 << s); ++b) {
            const int e = (32 >> (s + 1)) * bitrev_c(b, s);  // zeta = omega_32^e
#pragma unroll
            for (int j = 0; j < len; ++j) {
                const int i0 = b * 2 * len + j, i1 = i0 + len;
                const uint32_t x = v[i0], y = v[i1];
                uint32_t t, add;
                if (b == 0 && !f25_b0_reduces(LQ, s)) {
                    t = y;  // zeta = 1, unreduced: both inputs below B q
                    add = (uint32_t)f25_b0_bound(LQ, s) * F25_Q;
                } else {
                    t = b == 0 ? f25_red(y) : f25_shoup(y, kF25W32[e], kF25W32Q[e]);
                    add = 2 * F25_Q;
                }
                v[i0] = x + t;
                v[i1] = x - t + add;
            }
        }
    }
}

// In-register DFT of length 2^LQ <= 32 (Goldilocks: omega = 2^(192 / 2^LQ)):
// natural order in, v[bitrev(k)] = X[k] out.
template <class F, int LQ>
__device__ __forceinline__ void dft_reg_f(typename F::T *v) {
    if constexpr (F::kLazy) {
        dft_reg_f25<LQ>(v);
        return;
    }
    constexpr int RD = 1 << LQ;
    // one flat loop with a constant trip count, so that every index and shift
    // below is a compile-time constant after unrolling
#pragma unroll
    for (int j = 0; j < LQ * (RD / 2); ++j) {
        const int lh = LQ - 1 - j / (RD / 2);  // stage with half-size h = 2^lh
        const int h = 1 << lh;
        const int b = j % (RD / 2);
        const int pos = b % h, blk = (b / h) * 2 * h;
        const typename F::T a = v[blk + pos], c = v[blk + pos + h];
        v[blk + pos] = F::add(a, c);
        v[blk + pos + h] = F::rot(F::sub(a, c), lh, pos);
    }
}
template <int LQ>
__device__ __forceinline__ void dft_reg(uint64_t *v) { dft_reg_f<FieldGL, LQ>(v); }

// Forward step J over NBUF buffers; tw[e] = omega_R^e, e < R.
//
// BITS0: every input of step 0 is 0 or 1 and step 0 has radix 16 (32-bit
// field).  Its DFTs then come from a table instead of 32 butterflies each: for
// input bits b_0 .. b_15, since omega_16^8 = -1,
//   X_k = sum_i b_i omega_16^(i k) = T_k(b_0 .. b_7) + (-1)^k T_k(b_8 .. b_15),
//   T_k(p) = tab[k * 256 + p] (RootTablesT::bits16, copied to shared memory),
// the same canonical values the butterflies give.
template <class F, int LOGR, int J, int NCOL_LG, int NBUF, bool BITS0 = false>
__device__ __forceinline__ void fwd_step_f(typename F::T *s0, typename F::T *s1, const typename F::T *tw,
                                           const typename F::T *tab = nullptr) {
    using T = typename F::T;
    constexpr int OFF = st_off(LOGR, J), LQ = st_q(LOGR, J), RD = 1 << LQ;
    constexpr int LN = LOGR - OFF, LM = LN - LQ;
    constexpr int ITEMS = (1 << (LOGR - LQ)) << NCOL_LG;
    for (int item = threadIdx.x; item < ITEMS * NBUF; item += kThreads) {
        const int bi = item / ITEMS;
        const int it = item - bi * ITEMS;
        T *s = (NBUF == 2 && bi) ? s1 : s0;
        const int c = it & ((1 << NCOL_LG) - 1);
        const int rest = it >> NCOL_LG;
        const int i2 = rest & ((1 << LM) - 1);
        const int row0 = ((rest >> LM) << LN) + i2;
        T v[RD];
        if constexpr (BITS0 && J == 0) {
            static_assert(RD == 16 && sizeof(T) == 4, "the bit table holds radix-16 DFTs of the 32-bit field");
            uint32_t p = 0;
#pragma unroll
            for (int i1 = 0; i1 < RD; ++i1) p |= (uint32_t)s[sp(((row0 + (i1 << LM)) << NCOL_LG) + c)] << i1;
            const T *tlo = tab + (p & 255u), *thi = tab + (p >> 8);
#pragma unroll
            for (int k = 0; k < RD; ++k) {
                const T a = tlo[k << 8], b = thi[k << 8];
                v[bitrev_c(k, LQ)] = (k & 1) ? F::sub(a, b) : F::add(a, b);
            }
        } else {
#pragma unroll
            for (int i1 = 0; i1 < RD; ++i1) v[i1] = s[sp(((row0 + (i1 << LM)) << NCOL_LG) + c)];
            dft_reg_f<F, LQ>(v);
        }
#pragma unroll
        for (int k1 = 0; k1 < RD; ++k1) {
            T x = v[bitrev_c(k1, LQ)];
            if (LM > 0 && k1 > 0 && i2 > 0) {
                x = F::twmul(x, tw[tw_swz((i2 * k1) << OFF)]);
            } else {
                x = F::red(x);
            }
            s[sp(((row0 + (k1 << LM)) << NCOL_LG) + c)] = x;
        }
    }
}
template <int LOGR, int J, int NCOL_LG, int NBUF>
__device__ __forceinline__ void fwd_step(uint64_t *s0, uint64_t *s1, const uint64_t *tw) {
    fwd_step_f<FieldGL, LOGR, J, NCOL_LG, NBUF>(s0, s1, tw);
}

// Exact inverse of fwd_step J (up to the factor RD), inverse roots.
template <class F, int LOGR, int J, int NCOL_LG, int NBUF>
__device__ __forceinline__ void inv_step_f(typename F::T *s0, typename F::T *s1, const typename F::T *tw) {
    using T = typename F::T;
    constexpr int R = 1 << LOGR;
    constexpr int OFF = st_off(LOGR, J), LQ = st_q(LOGR, J), RD = 1 << LQ;
    constexpr int LN = LOGR - OFF, LM = LN - LQ;
    constexpr int ITEMS = (1 << (LOGR - LQ)) << NCOL_LG;
    for (int item = threadIdx.x; item < ITEMS * NBUF; item += kThreads) {
        const int bi = item / ITEMS;
        const int it = item - bi * ITEMS;
        T *s = (NBUF == 2 && bi) ? s1 : s0;
        const int c = it & ((1 << NCOL_LG) - 1);
        const int rest = it >> NCOL_LG;
        const int i2 = rest & ((1 << LM) - 1);
        const int row0 = ((rest >> LM) << LN) + i2;
        T v[RD];
#pragma unroll
        for (int k1 = 0; k1 < RD; ++k1) {
            T x = s[sp(((row0 + (k1 << LM)) << NCOL_LG) + c)];
            if (LM > 0 && k1 > 0 && i2 > 0) {
                x = F::twmul(x, tw[tw_swz((R - ((i2 * k1) << OFF)) & (R - 1))]);
            } else {
                x = F::red(x);
            }
            v[k1] = x;
        }
        dft_reg_f<F, LQ>(v);
        // inverse DFT output i1 is the forward output at frequency -i1 mod RD
#pragma unroll
        for (int i1 = 0; i1 < RD; ++i1)
            s[sp(((row0 + (i1 << LM)) << NCOL_LG) + c)] = v[bitrev_c((RD - i1) & (RD - 1), LQ)];
    }
}
template <int LOGR, int J, int NCOL_LG, int NBUF>
__device__ __forceinline__ void inv_step(uint64_t *s0, uint64_t *s1, const uint64_t *tw) {
    inv_step_f<FieldGL, LOGR, J, NCOL_LG, NBUF>(s0, s1, tw);
}

template <class F, int LOGR, int J, int NCOL_LG, int NBUF, bool BITS0 = false>
__device__ __forceinline__ void fwd_from(typename F::T *s0, typename F::T *s1, const typename F::T *tw,
                                         const typename F::T *tab = nullptr) {
    if constexpr (J < st_n(LOGR)) {
        fwd_step_f<F, LOGR, J, NCOL_LG, NBUF, BITS0>(s0, s1, tw, tab);
        __syncthreads();
        fwd_from<F, LOGR, J + 1, NCOL_LG, NBUF, BITS0>(s0, s1, tw, tab);
    }
}
template <class F, int LOGR, int J, int NCOL_LG, int NBUF>
__device__ __forceinline__ void inv_from(typename F::T *s0, typename F::T *s1, const typename F::T *tw) {
    if constexpr (J >= 0) {
        inv_step_f<F, LOGR, J, NCOL_LG, NBUF>(s0, s1, tw);
        __syncthreads();
        inv_from<F, LOGR, J - 1, NCOL_LG, NBUF>(s0, s1, tw);
    }
}

// Forward transform of every column (natural -> digit-reversed); ends with a barrier.
template <class F, int LOGR, int NCOL_LG, int NBUF, bool BITS0 = false>
__device__ __forceinline__ void ntt_fwd_f(typename F::T *s0, typename F::T *s1, const typename F::T *tw,
                                          const typename F::T *tab = nullptr) {
    if constexpr (LOGR > 0) fwd_from<F, LOGR, 0, NCOL_LG, NBUF, BITS0>(s0, s1, tw, tab);
}
// Inverse of ntt_fwd up to the factor R (digit-reversed -> natural); ends with a barrier.
template <class F, int LOGR, int NCOL_LG, int NBUF>
__device__ __forceinline__ void ntt_inv_f(typename F::T *s0, typename F::T *s1, const typename F::T *tw) {
    if constexpr (LOGR > 0) inv_from<F, LOGR, st_n(LOGR) - 1, NCOL_LG, NBUF>(s0, s1, tw);
}
template <int LOGR, int NCOL_LG, int NBUF>
__device__ __forceinline__ void ntt_fwd(uint64_t *s0, uint64_t *s1, const uint64_t *tw) {
    ntt_fwd_f<FieldGL, LOGR, NCOL_LG, NBUF>(s0, s1, tw);
}
template <int LOGR, int NCOL_LG, int NBUF>
__device__ __forceinline__ void ntt_inv(uint64_t *s0, uint64_t *s1, const uint64_t *tw) {
    ntt_inv_f<FieldGL, LOGR, NCOL_LG, NBUF>(s0, s1, tw);
}

// How a fused middle row treats a product that is one of several summed in
// the transform domain (a sum group of input blocks): the scaled pointwise
// products are added up before the inverse row transform (which is linear), so
// only the group's last product pays for it.
enum MidSum : int {
    kMidAlone = 0,  // inverse row transform of this product
    kMidFirst = 1,  // store the product to the row's accumulator, no inverse
    kMidInner = 2,  // add the product into the accumulator, no inverse
    kMidLast = 3,   // inverse row transform of accumulator + product
};

// One fused middle row of B = 2^13 elements (steps of radix 32, 16, 16): forward
// transforms of both operands, the pointwise product scaled by linv, and the
// inverse transform of the product, left in sA in natural order.  The last
// forward step, the product and the first inverse step run in registers on
// 16-row groups (thread t owns rows 16t .. 16t + 15 of both operands), and
// steps 1 and 2 only touch the 256-row blocks of the calling warp, so they are
// separated by warp barriers only.  With a sum mode other than kMidAlone, gC
// is the row's accumulator in global memory: thread t keeps its 16 products
// (frequency order) at gC[16t .. 16t + 15]; kMidFirst and kMidInner return
// after writing it (sA then holds nothing of use).  Ends with a block barrier.
template <class F>
__device__ __forceinline__ void middle_row_13_f(typename F::T *sA, typename F::T *sB, const typename F::T *tw,
                                                typename F::T linv, typename F::T *gC = nullptr,
                                                int mode = kMidAlone) {
    using T = typename F::T;
    static_assert(st_n(13) == 3 && st_q(13, 0) == 5 && st_q(13, 1) == 4 && st_q(13, 2) == 4, "schedule");
    static_assert(kThreads == 512, "one 16-row group per thread in the fused step");
    fwd_step_f<F, 13, 0, 0, 2>(sA, sB, tw);
    __syncthreads();
    fwd_step_f<F, 13, 1, 0, 2>(sA, sB, tw);
    __syncwarp();
    {
        const int row0 = threadIdx.x << 4;
        T a[16], b[16], c[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) a[i] = sA[sp(row0 + i)];
#pragma unroll
        for (int i = 0; i < 16; ++i) b[i] = sB[sp(row0 + i)];
        dft_reg_f<F, 4>(a);
        dft_reg_f<F, 4>(b);
        // frequency k sits in register bitrev(k); the inverse step takes frequency order
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = F::prod(a[bitrev_c(k, 4)], b[bitrev_c(k, 4)], linv);
        if (mode != kMidAlone) {
            constexpr int PER = 16 / (int)sizeof(T);
            uint4 *g4 = reinterpret_cast<uint4 *>(gC + row0);
            if (mode != kMidFirst) {
#pragma unroll
                for (int q = 0; q < 16 / PER; ++q) {
                    T pc[PER];
                    unpack16(__ldcg(g4 + q), pc);
#pragma unroll
                    for (int j = 0; j < PER; ++j) c[PER * q + j] = F::add(c[PER * q + j], pc[j]);
                }
            }
            if (mode != kMidLast) {
#pragma unroll
                for (int q = 0; q < 16 / PER; ++q) {
                    T pc[PER];
#pragma unroll
                    for (int j = 0; j < PER; ++j) pc[j] = c[PER * q + j];
                    g4[q] = pack16(pc);
                }
            }
        }
        if (mode == kMidAlone || mode == kMidLast) {
            dft_reg_f<F, 4>(c);
#pragma unroll
            for (int i = 0; i < 16; ++i) sA[sp(row0 + i)] = c[bitrev_c((16 - i) & 15, 4)];
        }
    }
    if (mode == kMidFirst || mode == kMidInner) {
        __syncthreads();  // sA / sB free for the next row
        return;
    }
    __syncwarp();
    inv_step_f<F, 13, 1, 0, 1>(sA, sA, tw);
    __syncthreads();
    inv_step_f<F, 13, 0, 0, 1>(sA, sA, tw);
    __syncthreads();
}
__device__ __forceinline__ void middle_row_13(uint64_t *sA, uint64_t *sB, const uint64_t *tw, uint64_t linv) {
    middle_row_13_f<FieldGL>(sA, sB, tw, linv);
}

// Frequency held at position p after ntt_fwd<LOGR>: the digits k_j of p (step 0
// in the top bits) reassembled least-significant first.
template <int LOGR>
__device__ __forceinline__ uint32_t pos_to_freq(uint32_t p) {
    uint32_t f = 0;
#pragma unroll
    for (int j = 0; j < st_n(LOGR); ++j) {
        const int q = st_q(LOGR, j), off = st_off(LOGR, j);
        f |= ((p >> (LOGR - off - q)) & ((1u << q) - 1)) << off;
    }
    return f;
}

// Fill tw[e] = omega_R^e (e < R) from the global table of omega_8192^e.
template <int LOGR, class T>
__device__ __forceinline__ void load_roots(T *tw, const T *__restrict__ g8192) {
    for (int e = threadIdx.x; e < (1 << LOGR); e += kThreads) tw[tw_swz(e)] = __ldg(g8192 + (e << (kSmallLg - LOGR)));
}

__device__ __forceinline__ int bitrev(int k, int lg) {
    return lg == 0 ? 0 : (int)(__brev((unsigned)k) >> (32 - lg));
}

}  // namespace cm
