// NTT kernels of the extractor path (GB300, sm_103a).
//
// A length-L transform (L = 2^lg) is a product of in-place passes over HBM:
//   L = R_1 * ... * R_k * B,  B <= 2^13 contiguous (on chip), R_j <= 2^12.
// Forward pass j takes every block of N_j = R_j * S_j contiguous elements
// (S_j = L / (R_1 ... R_j)) as an R_j x S_j matrix, transforms each column
// (length R_j, stride S_j) and multiplies entry (k, c) by omega_{N_j}^(c k)
// (the four-step split of Def. ntt).  The B-blocks are then transformed on
// chip.  The inverse applies the exact inverse of every pass in reverse order,
// so the frequency order in between never matters: the pointwise product of
// Thm. convolution is taken in whatever order both operands share.
//
// Kernels:
// Each kernel is a template over the field policy F (FieldGL, FieldF30,
// FieldF25).  Over the lazily reduced F25, forward passes leave values in
// [0, 2q), inverse passes and the middle any representative below 12 q; a
// parity is read from the canonical value (F::canon).
//
//   k_fused_small<LG>  whole extraction for L <= 2^13 in one CTA: bit unpack,
//                      forward NTT of both operands, product * L^-1, inverse NTT,
//                      parity of the output window, bit pack.
//   k_pass<...>        one column pass; the first forward pass reads packed bits,
//                      the last inverse pass writes parity bytes of the window.
//   k_middle           B = 2^13 rows of both operands: forward row NTTs,
//                      product * L^-1, inverse row NTT (one read of each operand,
//                      one write).
//   k_pack             parity bytes -> packed output words (and the Dodis
//                      precondition: zero output if x is constant).
//   k_allsame          Dodis precondition flags (any 1 bit, any 0 bit in x).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_internal.h"
#include "ntt25.cuh"
#include "ntt_device.cuh"

namespace cm {

// ---------------------------------------------------------------------------
// Whole extraction on one CTA (L = 2^LG <= 2^13).
// ---------------------------------------------------------------------------
// Shared memory (words of F::T): both operands, then the roots (F25: the step
// root pairs, 16-byte aligned for the asynchronous copy).
template <class F, int LG>
__host__ __device__ constexpr int small_tw_off() {
    return F::kLazy ? (2 * sp_size(1 << LG) + 3) & ~3 : 2 * sp_size(1 << LG);
}
template <class F, int LG>
__host__ __device__ constexpr int small_smem_words() {
    return small_tw_off<F, LG>() + (F::kLazy ? st25_smem_words(LG) : (1 << LG));
}
template <class F, int LG>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_small(BitMap amap, BitMap bmap, uint64_t lo, uint64_t m, uint64_t linv_,
              uint64_t *__restrict__ z, const uint32_t *__restrict__ pre,
              uint32_t *__restrict__ status, RootTablesT<typename F::T> rt) {
    using T = typename F::T;
    constexpr int L = 1 << LG;
    const T linv = (T)linv_;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    T *sB = sA + sp_size(L);
    T *tw = sA + small_tw_off<F, LG>();
    if constexpr (F::kLazy)
        prefetch_steps25<LG>(tw, rt.steps);  // lands while the operands unpack
    else
        load_roots<LG>(tw, rt.small);
    if constexpr (LG >= 5) {
        // one run of 32 positions per thread, read as one or two words; thread
        // t of a warp writes run t at sp(32 t + i), bank (t + i) mod 32
        for (int u = threadIdx.x; u < 2 * (L / 32); u += kThreads) {
            const int op = u >= L / 32 ? 1 : 0;
            const int run = u - op * (L / 32);
            const uint32_t b = op ? bmap.get_run<32>(32 * (uint64_t)run) : amap.get_run<32>(32 * (uint64_t)run);
            T *dst = (op ? sB : sA) + sp(32 * run);
#pragma unroll
            for (int i = 0; i < 32; ++i) dst[i] = (T)((b >> i) & 1u);
        }
    } else {
        for (int i = threadIdx.x; i < L; i += kThreads) {
            sA[sp(i)] = (T)amap.get(i);
            sB[sp(i)] = (T)bmap.get(i);
        }
    }
    if constexpr (F::kLazy) cp_async_wait_all();
    __syncthreads();
    if constexpr (F::kLazy) {
        ntt_fwd25<LG, 0, 2>(sA, sB, tw);
        for (int i = threadIdx.x; i < L; i += kThreads) sA[sp(i)] = prod25(sA[sp(i)], sB[sp(i)], linv_);
        __syncthreads();
        ntt_inv25<LG, 0, 1>(sA, sA, tw);
    } else {
        ntt_fwd_f<F, LG, 0, 2>(sA, sB, tw);
        for (int i = threadIdx.x; i < L; i += kThreads) sA[sp(i)] = F::prod(sA[sp(i)], sB[sp(i)], linv);
        __syncthreads();
        ntt_inv_f<F, LG, 0, 1>(sA, sA, tw);
    }
    // F25's inverse leaves coefficient n at position (L - n) mod L
    auto at = [](uint64_t n) { return F::kLazy ? (int)((L - n) & (L - 1)) : (int)n; };

    const bool bad = pre && (pre[0] == 0u || pre[1] == 0u);
    if (bad && threadIdx.x == 0) atomicOr(status, kFlagPrecond);
    // window positions lo .. lo + m - 1, parity packed by warp ballots
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nwords = (m + 63) >> 6;
    for (uint64_t w = warp; w < nwords; w += kThreads / 32) {
        const uint64_t p0 = (w << 6) + lane, p1 = p0 + 32;
        const uint32_t b0 = (p0 < m) ? (uint32_t)(F::canon(sA[sp(at(lo + p0))]) & 1u) : 0u;
        const uint32_t b1 = (p1 < m) ? (uint32_t)(F::canon(sA[sp(at(lo + p1))]) & 1u) : 0u;
        const uint32_t w0 = __ballot_sync(0xffffffffu, b0);
        const uint32_t w1 = __ballot_sync(0xffffffffu, b1);
        if (lane == 0) z[w] = bad ? 0ull : ((uint64_t)w1 << 32 | w0);
    }
}

// v[j] *= omega^((c0 + j) k 2^esh), j < VW: the pass twiddles of VW consecutive
// columns of one row.  For VW >= 4 the roots are a geometric run: two table
// lookups (the first root and the step) and a running product replace one
// lookup per element.
template <class F, int VW>
__device__ __forceinline__ void row_twiddle(typename F::T (&v)[VW], uint64_t k, uint64_t c0, int esh,
                                            const typename F::T *lo, const typename F::T *hi) {
    using T = typename F::T;
    if (k == 0) return;
    if constexpr (VW >= 4) {
        T w = big_root_f<F>(lo, hi, (uint32_t)((c0 * k) << esh));
        const T d = big_root_f<F>(lo, hi, (uint32_t)(k << esh));
#pragma unroll
        for (int j = 0; j < VW; ++j) {
            v[j] = F::twmul(v[j], w);
            if (j + 1 < VW) w = F::twmul(w, d);
        }
    } else {
#pragma unroll
        for (int j = 0; j < VW; ++j) {
            const uint32_t E = (uint32_t)(((c0 + j) * k) << esh);
            if (E) v[j] = F::twmul(v[j], big_root_f<F>(lo, hi, E));
        }
    }
}

// A forward pass over input bits in the 32-bit field whose first on-chip step
// has radix 16 takes that step's DFTs from the bit table (fwd_step_f, BITS0).
// The table (4096 elements) follows the roots in shared memory, 16-byte aligned.
template <class F, int LOGR, bool INV, bool BITS_IN>
__host__ __device__ constexpr bool pass_bits_table() {
    return !INV && BITS_IN && sizeof(typename F::T) == 4 && st_q(LOGR, 0) == 4;
}
// Shared memory of a column pass: the tile, then the step roots (F25: root
// pairs, 8-byte aligned), then the bit table (16-byte aligned).
template <class F, int LOGR>
__host__ __device__ constexpr int pass_tw_off() {
    return F::kLazy ? (sp_size(1 << (LOGR + F::ncol_lg(LOGR))) + 1) & ~1 : sp_size(1 << (LOGR + F::ncol_lg(LOGR)));
}
template <class F, int LOGR>
__host__ __device__ constexpr int pass_tw_words() {
    return F::kLazy ? st25_smem_words(LOGR) : (1 << LOGR);
}
template <class F, int LOGR>
__host__ __device__ constexpr int pass_table_off() {
    return (pass_tw_off<F, LOGR>() + pass_tw_words<F, LOGR>() + 3) & ~3;
}
constexpr int kBitsTable = 16 * 256;

// ---------------------------------------------------------------------------
// One column pass over tiles of R = 2^LOGR rows x C = 2^F::ncol_lg(LOGR) columns.
// ---------------------------------------------------------------------------
// Tiles 0 .. ntiles - 1 of the grid work on (data, map); a forward pass may
// take both operands in one launch, tiles ntiles .. 2 ntiles - 1 on (data2, map2).
template <class F, int LOGR, bool INV, bool BITS_IN, bool PARITY_OUT>
__global__ void __launch_bounds__(kThreads, sizeof(typename F::T) == 4 ? 2 : 1)
k_pass(typename F::T *__restrict__ data1, BitMap map1, typename F::T *__restrict__ data2, BitMap map2,
       uint64_t ntiles, int lgN, int lgS, uint8_t *__restrict__ par, uint64_t lo, uint64_t m,
       RootTablesT<typename F::T> rt) {
    using T = typename F::T;
    constexpr int R = 1 << LOGR;
    constexpr int NCOL_LG = F::ncol_lg(LOGR);
    constexpr int C = 1 << NCOL_LG;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    T *tw = smem + pass_tw_off<F, LOGR>();
    if constexpr (F::kLazy)
        load_steps25<LOGR>(tw, rt.steps);
    else
        load_roots<LOGR>(tw, rt.small);
    constexpr bool BTAB = pass_bits_table<F, LOGR, INV, BITS_IN>();
    T *tab = smem + pass_table_off<F, LOGR>();
    if constexpr (BTAB) {
        for (int i = threadIdx.x; i < kBitsTable / 4; i += kThreads)
            reinterpret_cast<uint4 *>(tab)[i] = __ldg(reinterpret_cast<const uint4 *>(rt.bits16) + i);
    }
    const uint64_t S = 1ull << lgS;
    const uint64_t tiles_per_blk = S >> NCOL_LG;
    const bool second = blockIdx.x >= ntiles;
    const uint64_t tile = second ? blockIdx.x - ntiles : blockIdx.x;
    T *__restrict__ data = second ? data2 : data1;
    const BitMap map = second ? map2 : map1;
    const uint64_t blk = tile / tiles_per_blk;
    const uint64_t col0 = (tile - blk * tiles_per_blk) << NCOL_LG;
    const uint64_t base = (blk << lgN) + col0;
    const int esh = F::kAdicity - lgN;  // omega_N = g^(2^(adicity - lgN))

    // rows are stored in the digit-reversed order of the on-chip transform:
    // row p of the tile holds frequency pos_to_freq(p) (forward) and is read
    // back as such (inverse), so the pass twiddle uses that frequency.  Each
    // access moves 16 consecutive bytes of a tile row (VW elements).
    constexpr int VW = 16 / (int)sizeof(T);
    static_assert(C % VW == 0, "tile rows hold whole 16-byte vectors");
#pragma unroll 4
    for (int q = threadIdx.x; q < R * C / VW; q += kThreads) {
        const int e0 = q * VW;
        const int i = e0 >> NCOL_LG, c = e0 & (C - 1);
        const uint64_t g = base + ((uint64_t)i << lgS) + c;
        T v[VW];
        if (BITS_IN) {
            const uint32_t bits = map.get_run<VW>(g);
#pragma unroll
            for (int j = 0; j < VW; ++j) v[j] = (T)((bits >> j) & 1u);
        } else {
            unpack16(*reinterpret_cast<const uint4 *>(data + g), v);
        }
        // F25's inverse takes every root inverted: the forward row roots, on
        // values brought below 2q first (the root is below 2q, not below q)
        if (INV) {
            if constexpr (F::kLazy) {
#pragma unroll
                for (int j = 0; j < VW; ++j) v[j] = F::red(v[j]);
                row_twiddle<F, VW>(v, pos_to_freq<LOGR>(i), col0 + c, esh, rt.big_lo_fwd, rt.big_hi_fwd);
            } else
                row_twiddle<F, VW>(v, pos_to_freq<LOGR>(i), col0 + c, esh, rt.big_lo_inv, rt.big_hi_inv);
        }
#pragma unroll
        for (int j = 0; j < VW; ++j) smem[sp(e0 + j)] = v[j];
    }
    __syncthreads();
    if constexpr (F::kLazy) {
        if constexpr (INV)
            ntt_inv25<LOGR, NCOL_LG, 1>(smem, smem, tw);
        else
            ntt_fwd25<LOGR, NCOL_LG, 1, BTAB>(smem, smem, tw, tab);
    } else if (INV) {
        ntt_inv_f<F, LOGR, NCOL_LG, 1>(smem, smem, tw);
    } else {
        ntt_fwd_f<F, LOGR, NCOL_LG, 1, BTAB>(smem, smem, tw, tab);
    }
#pragma unroll 4
    for (int q = threadIdx.x; q < R * C / VW; q += kThreads) {
        const int e0 = q * VW;
        const int i = e0 >> NCOL_LG, c = e0 & (C - 1);
        const uint64_t g = base + ((uint64_t)i << lgS) + c;
        T v[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) v[j] = smem[sp(e0 + j)];
        if (!INV) row_twiddle<F, VW>(v, pos_to_freq<LOGR>(i), col0 + c, esh, rt.big_lo_fwd, rt.big_hi_fwd);
        if (PARITY_OUT) {
            // F25: position g holds coefficient (L - g) mod L, L = 2^lgN (this
            // pass is the transform's first)
            const uint64_t lmask = (1ull << lgN) - 1;
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                const uint64_t n = F::kLazy ? ((lmask + 1 - (g + j)) & lmask) : g + j;
                const uint64_t p = n - lo;
                if (n >= lo && p < m) par[p] = (uint8_t)(F::canon(v[j]) & 1u);
            }
        } else {
            *reinterpret_cast<uint4 *>(data + g) = pack16(v);
        }
    }
}

}  // namespace cm
