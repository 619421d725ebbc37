// On-chip transform steps over the lazily reduced field F25 (q = 5 * 2^25 + 1).
//
// The same mixed-radix decomposition as ntt_device.cuh (steps of radix <= 32,
// the four-step split of Def. ntt applied recursively over shared memory),
// written for the cost structure of this field:
//
// - Step roots come from per-step tables laid out for the thread that uses
//   them.  Step J multiplies output k1 of column i2 by omega_(N_J)^(i2 k1)
//   (N_J = 2^(LOGR - OFF_J), M_J = N_J / RD_J columns); its table holds that
//   root at [(k1 - 1) M_J + i2] as a pair (w, floor(w 2^32 / q)) for the
//   Shoup product (three multiplies, no compare).  A thread reads its
//   RD_J - 1 roots at fixed offsets from its own base i2 (no index
//   arithmetic), and the lanes of a warp, which take consecutive columns,
//   read consecutive pairs.
// - The inverse transform takes every root inverted, i.e. it runs the exact
//   inverse steps with omega in place of omega^-1.  That computes
//   F_omega Pi^-1 (Pi: the forward transform's digit-reversed order) instead
//   of F_omega^-1 Pi^-1, and F_omega = L J F_omega^-1 with J the index
//   negation n -> -n mod L.  So the "inverse" uses the forward tables, its
//   register DFTs store in plain bit-reversed order, and after the 1 / L
//   folded into the pointwise product position g holds the convolution
//   coefficient at (L - g) mod L; the parity readers index accordingly.
// - Values: forward steps take inputs in [0, 2q) and leave [0, 2q) (the root
//   product or red); inverse steps take any 32-bit value, bring each input to
//   [0, 2q) by the root product or red, and leave the raw DFT output (below
//   20 q, dft_reg_f25).
#pragma once
#include <stdint.h>

#include "ntt_device.cuh"

namespace cm {

// Offset (in root pairs) of step J's table within the tables of a transform
// of length 2^logr, and the pairs of all of them (steps 0 .. st_n - 2; the
// last step has no roots).  The set for length 2^logr starts at pair 2^logr
// of RootTables25::steps, and has fewer than 2^logr pairs.
__host__ __device__ __forceinline__ constexpr int st25_tab_off(int logr, int j) {
    int o = 0, off = 0;
    for (int i = 0; i < j; ++i) {
        const int q = st_q(logr, i);
        o += ((1 << q) - 1) * (1 << (logr - off - q));
        off += q;
    }
    return o;
}
__host__ __device__ __forceinline__ constexpr int st25_tab_words(int logr) {
    return st25_tab_off(logr, st_n(logr) - 1);
}

// Copy the step tables of length 2^LOGR (pairs) into shared memory at dst
// (8-byte aligned; ends without a barrier).  NT: the threads that copy.
template <int LOGR, int NT = kThreads>
__device__ __forceinline__ void load_steps25(uint32_t *dst, const uint32_t *__restrict__ steps) {
    const uint2 *src = reinterpret_cast<const uint2 *>(steps) + (1 << LOGR);
    uint2 *d = reinterpret_cast<uint2 *>(dst);
    for (int i = threadIdx.x; i < st25_tab_words(LOGR); i += NT) d[i] = __ldg(src + i);
}
// Shared-memory words of the step tables of length 2^LOGR.
__host__ __device__ __forceinline__ constexpr int st25_smem_words(int logr) { return 2 * st25_tab_words(logr); }

// The step tables of length 2^LOGR into shared memory at dst (16-byte
// aligned) by asynchronous 16-byte copies (cp.async, sm_80 and later), so that
// other work proceeds while they land; the issuing thread waits with
// cp_async_wait_all(), then a barrier publishes them.  NT: the threads that copy.
template <int LOGR, int NT = kThreads>
__device__ __forceinline__ void prefetch_steps25(uint32_t *dst, const uint32_t *__restrict__ steps) {
    constexpr int kVec = st25_smem_words(LOGR) / 4;  // pair counts are even: whole vectors
    static_assert(st25_smem_words(LOGR) % 4 == 0, "whole 16-byte vectors");
    const uint4 *src = reinterpret_cast<const uint4 *>(steps + 2 * (1 << LOGR));  // pair 2^LOGR
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    for (int e = threadIdx.x; e < kVec; e += NT)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16u * e), "l"(src + e) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// x times the root pair r = (w, floor(w 2^32 / q)) -> [0, 2q), any 32-bit x.
__device__ __forceinline__ uint32_t shoup_pair(uint32_t x, uint2 r) { return f25_shoup(x, r.x, r.y); }

// Padded shared-memory position of input i1 of an item whose first input is
// element e0, inputs S elements apart: linear in i1 when S >= 32 (sp adds one
// word per 32 elements).
template <int S>
__device__ __forceinline__ int sp_at(int e0, int p0, int i1) {
    if constexpr (S >= 32)
        return p0 + i1 * (S + S / 32);
    else
        return sp(e0 + i1 * S);
}

// Forward step J over NBUF buffers (see fwd_step_f for the item layout).
// BITS0: step 0 has radix 16 and 0/1 inputs; its DFTs come from the bit table
// (RootTablesT::bits16, in shared memory at tab16).
// tid: this thread's index among the kThreads that share the step.
template <int LOGR, int J, int NCOL_LG, int NBUF, bool BITS0 = false>
__device__ __forceinline__ void fwd_step25(uint32_t *s0, uint32_t *s1, const uint32_t *tab,
                                           const uint32_t *tab16 = nullptr, int tid = threadIdx.x) {
    constexpr int OFF = st_off(LOGR, J), LQ = st_q(LOGR, J), RD = 1 << LQ;
    constexpr int LN = LOGR - OFF, LM = LN - LQ, M = 1 << LM;
    constexpr int ITEMS = (1 << (LOGR - LQ)) << NCOL_LG;
    constexpr int S = M << NCOL_LG;
    const uint2 *tJ = reinterpret_cast<const uint2 *>(tab) + st25_tab_off(LOGR, J);
    for (int item = tid; item < ITEMS * NBUF; item += kThreads) {
        const int bi = (NBUF == 2 && item >= ITEMS) ? 1 : 0;
        const int it = item - bi * ITEMS;
        uint32_t *s = bi ? s1 : s0;
        const int c = it & ((1 << NCOL_LG) - 1);
        const int rest = it >> NCOL_LG;
        const int i2 = rest & (M - 1);
        const int e0 = ((((rest >> LM) << LN) + i2) << NCOL_LG) + c;
        const int p0 = sp(e0);
        uint32_t v[RD];
        if constexpr (BITS0 && J == 0) {
            static_assert(RD == 16, "the bit table holds radix-16 DFTs");
            uint32_t p = 0;
#pragma unroll
            for (int i1 = 0; i1 < RD; ++i1) p |= s[sp_at<S>(e0, p0, i1)] << i1;
            const uint32_t *tlo = tab16 + (p & 255u), *thi = tab16 + (p >> 8);
#pragma unroll
            for (int k = 0; k < RD; ++k) {
                const uint32_t a = tlo[k << 8], b = thi[k << 8];
                v[bitrev_c(k, LQ)] = (k & 1) ? f25_sub(a, b) : f25_add(a, b);
            }
        } else {
#pragma unroll
            for (int i1 = 0; i1 < RD; ++i1) v[i1] = s[sp_at<S>(e0, p0, i1)];
            dft_reg_f25<LQ>(v);
        }
        const uint2 *tw = tJ + i2;
#pragma unroll
        for (int k1 = 0; k1 < RD; ++k1) {
            uint32_t x = v[bitrev_c(k1, LQ)];
            if (LM > 0 && k1 > 0) {
                x = shoup_pair(x, tw[(k1 - 1) * M]);
            } else {
                x = f25_red(x);
            }
            s[sp_at<S>(e0, p0, k1)] = x;
        }
    }
}

// Step J of the inverse with every root inverted (forward roots, forward
// register DFT, outputs in plain bit-reversed order).
template <int LOGR, int J, int NCOL_LG, int NBUF>
__device__ __forceinline__ void inv_step25(uint32_t *s0, uint32_t *s1, const uint32_t *tab, int tid = threadIdx.x) {
    constexpr int OFF = st_off(LOGR, J), LQ = st_q(LOGR, J), RD = 1 << LQ;
    constexpr int LN = LOGR - OFF, LM = LN - LQ, M = 1 << LM;
    constexpr int ITEMS = (1 << (LOGR - LQ)) << NCOL_LG;
    constexpr int S = M << NCOL_LG;
    const uint2 *tJ = reinterpret_cast<const uint2 *>(tab) + st25_tab_off(LOGR, J);
    for (int item = tid; item < ITEMS * NBUF; item += kThreads) {
        const int bi = (NBUF == 2 && item >= ITEMS) ? 1 : 0;
        const int it = item - bi * ITEMS;
        uint32_t *s = bi ? s1 : s0;
        const int c = it & ((1 << NCOL_LG) - 1);
        const int rest = it >> NCOL_LG;
        const int i2 = rest & (M - 1);
        const int e0 = ((((rest >> LM) << LN) + i2) << NCOL_LG) + c;
        const int p0 = sp(e0);
        const uint2 *tw = tJ + i2;
        uint32_t v[RD];
#pragma unroll
        for (int k1 = 0; k1 < RD; ++k1) {
            const uint32_t x = s[sp_at<S>(e0, p0, k1)];
            v[k1] = (LM > 0 && k1 > 0) ? shoup_pair(x, tw[(k1 - 1) * M]) : f25_red(x);
        }
        dft_reg_f25<LQ>(v);
#pragma unroll
        for (int i1 = 0; i1 < RD; ++i1) s[sp_at<S>(e0, p0, i1)] = v[bitrev_c(i1, LQ)];
    }
}

template <int LOGR, int J, int NCOL_LG, int NBUF, bool BITS0>
__device__ __forceinline__ void fwd_from25(uint32_t *s0, uint32_t *s1, const uint32_t *tab, const uint32_t *tab16) {
    if constexpr (J < st_n(LOGR)) {
        fwd_step25<LOGR, J, NCOL_LG, NBUF, BITS0>(s0, s1, tab, tab16);
        __syncthreads();
        fwd_from25<LOGR, J + 1, NCOL_LG, NBUF, BITS0>(s0, s1, tab, tab16);
    }
}
template <int LOGR, int J, int NCOL_LG, int NBUF>
__device__ __forceinline__ void inv_from25(uint32_t *s0, uint32_t *s1, const uint32_t *tab) {
    if constexpr (J >= 0) {
        inv_step25<LOGR, J, NCOL_LG, NBUF>(s0, s1, tab);
        __syncthreads();
        inv_from25<LOGR, J - 1, NCOL_LG, NBUF>(s0, s1, tab);
    }
}

// Forward transform of every column (natural -> digit-reversed order, values
// in [0, 2q)); ends with a barrier.
template <int LOGR, int NCOL_LG, int NBUF, bool BITS0 = false>
__device__ __forceinline__ void ntt_fwd25(uint32_t *s0, uint32_t *s1, const uint32_t *tab,
                                          const uint32_t *tab16 = nullptr) {
    if constexpr (LOGR > 0) fwd_from25<LOGR, 0, NCOL_LG, NBUF, BITS0>(s0, s1, tab, tab16);
}
// Transform with every root inverted (digit-reversed -> natural order, up to
// the factor 2^LOGR and the index negation); ends with a barrier.
template <int LOGR, int NCOL_LG, int NBUF>
__device__ __forceinline__ void ntt_inv25(uint32_t *s0, uint32_t *s1, const uint32_t *tab) {
    if constexpr (LOGR > 0) inv_from25<LOGR, st_n(LOGR) - 1, NCOL_LG, NBUF>(s0, s1, tab);
}

// a b L^-1 for any 32-bit a, b (DFT outputs) -> [0, 2q).  linv packs the
// Shoup pair of L^-1 2^32 mod q (low word) and its quotient (high word):
// mont(red a, red b) = a b 2^-32, and the Shoup product restores the 2^32.
__device__ __forceinline__ uint32_t prod25(uint32_t a, uint32_t b, uint64_t linv) {
    return f25_shoup(f25_mont(f25_red(a), f25_red(b)), (uint32_t)linv, (uint32_t)(linv >> 32));
}

}  // namespace cm
