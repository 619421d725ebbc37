// Column passes and the fused middle for transforms over F25 (q = 5 * 2^25 + 1)
// of length L = R * 2^13 with R = 2^9 .. 2^12 (L = 2^22 .. 2^25).
//
// Same decomposition as k_pass / k_middle (four-step split of Def. ntt: a
// column pass over tiles of R rows x C = 2^(14 - LOGR) columns, the rows of
// 2^13 on chip), arranged so that every element crosses shared memory as few
// times as the steps need:
//   k25_fwd  the tile's input bits are loaded once per row into shared memory
//            (C <= 32 bits a row); step 0 reads its 0/1 inputs from there
//            into a register DFT (faster here than the radix-16 bit table,
//            whose random lookups conflict on banks); the last step
//            multiplies by the pass twiddle omega_N^(col freq) and stores
//            straight from registers to HBM.
//   k25_inv  the first step loads straight from HBM and multiplies by the pass
//            twiddle (every root inverted, as in ntt25.cuh); the last step
//            writes the parity bytes of the output window straight from
//            registers (position g holds coefficient (L - g) mod L).
//   k25_middle  step 0 of both operands loads straight from HBM; the last
//            inverse step stores straight to HBM.
// The pass twiddle of output k1 of last-step item (c, blk) is
// omega_N^(col (f_b + k1 2^OFFL)) = beta * P[c][k1]: beta = omega_N^(col f_b) per
// item (f_b = the frequency of the item's first row; Montgomery form, a lazy
// Montgomery product), P[c][k1] = omega_N^(col k1 2^OFFL) per tile (C x
// RD_last root pairs in shared memory, a Shoup product that also brings the
// raw DFT output to [0, 2q) first).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "cm_kernels.cuh"

namespace cm {

template <int LOGR>
struct Pass25 {
    static_assert(LOGR >= 9 && LOGR <= 12, "tiles of at most 32 columns");
    static constexpr int R = 1 << LOGR;
    static constexpr int NCOL_LG = kTileLg - LOGR;
    static constexpr int C = 1 << NCOL_LG;
    static constexpr int NST = st_n(LOGR);
    static constexpr int LAST = NST - 1;
    static constexpr int QL = st_q(LOGR, LAST), RDL = 1 << QL, OFFL = st_off(LOGR, LAST);
    static constexpr int Q0 = st_q(LOGR, 0), RD0 = 1 << Q0, M0 = R / RD0;
    static constexpr int Q1 = st_q(LOGR, 1), RD1 = 1 << Q1, N1 = R / RD0, M1 = N1 / RD1;  // step 1 (of 3)
    using BitsT = std::conditional_t<(C <= 8), uint8_t, std::conditional_t<(C <= 16), uint16_t, uint32_t>>;
    // The tile holds element e = row * C + col at word tile_at(e): e with the
    // column bits above log2 C XORed by the last step's block index (mod 32 /
    // C).  The last step's lanes take C columns of 32 / C consecutive blocks
    // (stride RD_last C words): without the XOR they would share banks.  The
    // other steps' lanes take 32 consecutive words, which the XOR (constant
    // within an aligned group of 32, since RD_last C >= 64) only permutes.
    static constexpr int SW_SHIFT = QL + NCOL_LG, SW_MASK = C >= 32 ? 0 : 32 / C - 1;
    static_assert(SW_SHIFT >= 5, "XOR constant within 32-word groups");
    // shared memory layout (32-bit words): tile, step root pairs, P pairs,
    // row bits
    static constexpr int O_STEPS = 1 << kTileLg;
    static constexpr int O_P = O_STEPS + st25_smem_words(LOGR);
    static constexpr int O_BITS = O_P + 2 * C * RDL;
    static constexpr int W_FWD = O_BITS + (int)(R * sizeof(BitsT) + 3) / 4;
    static constexpr int W_INV = O_BITS;
    static_assert(NST >= 2 && C * RDL <= kThreads, "two or more steps; one P entry per thread");
    static_assert(W_FWD * 4 <= 113 * 1024, "two CTAs per SM");
};

// Bulk prefetch of `bytes` (a multiple of 16) at a 16-byte aligned global
// address into L2 (cp.async.bulk.prefetch, sm_90 and later; no completion).
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int LOGR>
__device__ __forceinline__ int tile_at(int e) {
    using PS = Pass25<LOGR>;
    return e ^ (((e >> PS::SW_SHIFT) & PS::SW_MASK) << PS::NCOL_LG);
}

// P[k1 * C + c] = omega_N^(col k1 2^OFFL) as a Shoup pair (plain root,
// quotient), col = col0 + c; omega_N = g25^(2^esh).
template <int LOGR>
__device__ __forceinline__ void load_pass_p25(uint2 *P, uint32_t col0, int esh, const RootTables25 &rt) {
    using PS = Pass25<LOGR>;
    const int t = threadIdx.x;
    if (t < PS::C * PS::RDL) {
        const uint64_t col = col0 + (uint32_t)(t & (PS::C - 1)), k1 = (uint32_t)(t >> PS::NCOL_LG);
        const uint32_t E = (uint32_t)(((col * k1) << (PS::OFFL + esh)) & ((1ull << 25) - 1));
        const uint32_t w = f25_canon(f25_mont(big_root_f<FieldF25>(rt.big_lo_fwd, rt.big_hi_fwd, E), 1u));
        P[t] = make_uint2(w, f25_shoup_q(w));
    }
}

// The middle step (step 1 of three) of the tile's columns: forward (roots on
// the outputs) or with every root inverted (roots on the inputs).
template <int LOGR, bool INV>
__device__ __forceinline__ void tile_step1_25(uint32_t *tile, const uint32_t *steps) {
    using PS = Pass25<LOGR>;
    constexpr int C = PS::C, NCOL_LG = PS::NCOL_LG, RD = PS::RD1, M = PS::M1, N = PS::N1;
    constexpr int LM = LOGR - PS::Q0 - PS::Q1;  // log2 M
    const uint2 *tJ = reinterpret_cast<const uint2 *>(steps) + st25_tab_off(LOGR, 1);
    for (int item = threadIdx.x; item < (PS::R / RD) * C; item += kThreads) {
        const int c = item & (C - 1), rest = item >> NCOL_LG;
        const int i2 = rest & (M - 1), blk = rest >> LM;
        const int e0 = ((blk * N + i2) << NCOL_LG) + c;
        const uint2 *tw = tJ + i2;
        uint32_t v[RD];
        if constexpr (!INV) {
#pragma unroll
            for (int i1 = 0; i1 < RD; ++i1) v[i1] = tile[tile_at<LOGR>(e0 + ((i1 * M) << NCOL_LG))];
            dft_reg_f25<PS::Q1>(v);
#pragma unroll
            for (int k1 = 0; k1 < RD; ++k1) {
                const uint32_t x = v[bitrev_c(k1, PS::Q1)];
                tile[tile_at<LOGR>(e0 + ((k1 * M) << NCOL_LG))] = k1 ? shoup_pair(x, tw[(k1 - 1) * M]) : f25_red(x);
            }
        } else {
#pragma unroll
            for (int k1 = 0; k1 < RD; ++k1) {
                const uint32_t x = tile[tile_at<LOGR>(e0 + ((k1 * M) << NCOL_LG))];
                v[k1] = k1 ? shoup_pair(x, tw[(k1 - 1) * M]) : f25_red(x);
            }
            dft_reg_f25<PS::Q1>(v);
#pragma unroll
            for (int i1 = 0; i1 < RD; ++i1) tile[tile_at<LOGR>(e0 + ((i1 * M) << NCOL_LG))] = v[bitrev_c(i1, PS::Q1)];
        }
    }
}

// ---------------------------------------------------------------------------
// Forward column pass from bits (both operands: tiles ntiles .. 2 ntiles - 1
// take the second).
// ---------------------------------------------------------------------------
template <int LOGR>
__global__ void __launch_bounds__(kThreads, 2)
k25_fwd(uint32_t *__restrict__ data1, BitMap map1, uint32_t *__restrict__ data2, BitMap map2, uint32_t ntiles,
        int lgN, int lgS, RootTables25 rt) {
    using PS = Pass25<LOGR>;
    using BitsT = typename PS::BitsT;
    constexpr int C = PS::C, NCOL_LG = PS::NCOL_LG, M0 = PS::M0, RD0 = PS::RD0, RDL = PS::RDL;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *steps = tile + PS::O_STEPS;
    uint2 *P = reinterpret_cast<uint2 *>(tile + PS::O_P);
    BitsT *sbits = reinterpret_cast<BitsT *>(tile + PS::O_BITS);

    const bool second = blockIdx.x >= ntiles;
    const uint32_t t_ = second ? blockIdx.x - ntiles : blockIdx.x;
    uint32_t *__restrict__ data = second ? data2 : data1;
    const BitMap map = second ? map2 : map1;
    const uint32_t S = 1u << lgS;
    const uint32_t tiles_per_blk = S >> NCOL_LG;
    const uint32_t blkN = t_ / tiles_per_blk;
    const uint32_t col0 = (t_ - blkN * tiles_per_blk) << NCOL_LG;
    const uint32_t base = (blkN << lgN) + col0;  // < L <= 2^25
    const int esh = FieldF25::kAdicity - lgN;

    load_steps25<LOGR>(steps, rt.steps);
    load_pass_p25<LOGR>(P, col0, esh, rt);
    for (int i = threadIdx.x; i < PS::R; i += kThreads) sbits[i] = (BitsT)map.get_run<C>(base + (uint64_t)i * S);
    __syncthreads();

    // step 0: 0/1 inputs from the row bits
    {
        const uint2 *tw0 = reinterpret_cast<const uint2 *>(steps) + st25_tab_off(LOGR, 0);
        for (int item = threadIdx.x; item < M0 * C; item += kThreads) {
            const int c = item & (C - 1), i2 = item >> NCOL_LG;
            uint32_t v[RD0];
#pragma unroll
            for (int i1 = 0; i1 < RD0; ++i1) v[i1] = ((uint32_t)sbits[i2 + M0 * i1] >> c) & 1u;
            dft_reg_f25<PS::Q0>(v);
            const uint2 *tw = tw0 + i2;
            const int e0 = item;  // (i2 << NCOL_LG) + c
#pragma unroll
            for (int k1 = 0; k1 < RD0; ++k1) {
                const uint32_t x = v[bitrev_c(k1, PS::Q0)];
                tile[tile_at<LOGR>(e0 + ((k1 * M0) << NCOL_LG))] = k1 ? shoup_pair(x, tw[(k1 - 1) * M0]) : f25_red(x);
            }
        }
    }
    __syncthreads();
    if constexpr (PS::NST == 3) {
        tile_step1_25<LOGR, false>(tile, steps);
        __syncthreads();
    }
    // last step (no step roots): pass twiddle, store to HBM
    for (int item = threadIdx.x; item < (PS::R / RDL) * C; item += kThreads) {
        const int c = item & (C - 1), blk = item >> NCOL_LG;
        const uint32_t col = col0 + c;
        const uint32_t fb = pos_to_freq<LOGR>((uint32_t)(blk * RDL));
        const uint32_t beta = big_root_f<FieldF25>(rt.big_lo_fwd, rt.big_hi_fwd, (col * fb) << esh);
        const int e0 = ((blk * RDL) << NCOL_LG) + c;
        uint32_t v[RDL];
#pragma unroll
        for (int i1 = 0; i1 < RDL; ++i1) v[i1] = tile[tile_at<LOGR>(e0 + (i1 << NCOL_LG))];
        dft_reg_f25<PS::QL>(v);
        uint32_t *g = data + base + (uint32_t)(blk * RDL) * S + c;
#pragma unroll
        for (int k1 = 0; k1 < RDL; ++k1) g[(uint32_t)k1 * S] = f25_mont(shoup_pair(v[bitrev_c(k1, PS::QL)], P[k1 * C + c]), beta);
    }
}

// ---------------------------------------------------------------------------
// Inverse column pass (every root inverted) with the parity of the window:
// par[n - lo] = bit 0 of coefficient n for n in [lo, lo + m).
// ---------------------------------------------------------------------------
template <int LOGR>
__global__ void __launch_bounds__(kThreads, 2)
k25_inv(const uint32_t *__restrict__ data, int lgN, int lgS, uint8_t *__restrict__ par, uint64_t lo, uint64_t m,
        RootTables25 rt) {
    using PS = Pass25<LOGR>;
    constexpr int C = PS::C, NCOL_LG = PS::NCOL_LG, M0 = PS::M0, RD0 = PS::RD0, RDL = PS::RDL;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *steps = tile + PS::O_STEPS;
    uint2 *P = reinterpret_cast<uint2 *>(tile + PS::O_P);

    const uint32_t S = 1u << lgS;
    const uint32_t tiles_per_blk = S >> NCOL_LG;
    const uint32_t blkN = blockIdx.x / tiles_per_blk;
    const uint32_t col0 = (blockIdx.x - blkN * tiles_per_blk) << NCOL_LG;
    const uint32_t base = (blkN << lgN) + col0;
    const int esh = FieldF25::kAdicity - lgN;
    // a programmatic dependent (the pack with the tail) may start once every
    // CTA of this grid has: its CTAs fill the SMs this grid's last wave leaves
    asm volatile("griddepcontrol.launch_dependents;");

    load_steps25<LOGR>(steps, rt.steps);
    load_pass_p25<LOGR>(P, col0, esh, rt);
    __syncthreads();

    // first step (the forward's last): load from HBM, pass twiddle, DFT
    for (int item = threadIdx.x; item < (PS::R / RDL) * C; item += kThreads) {
        const int c = item & (C - 1), blk = item >> NCOL_LG;
        const uint32_t col = col0 + c;
        const uint32_t fb = pos_to_freq<LOGR>((uint32_t)(blk * RDL));
        const uint32_t beta = big_root_f<FieldF25>(rt.big_lo_fwd, rt.big_hi_fwd, (col * fb) << esh);
        const uint32_t *g = data + base + (uint32_t)(blk * RDL) * S + c;
        uint32_t v[RDL];
#pragma unroll
        for (int k1 = 0; k1 < RDL; ++k1) v[k1] = f25_mont(shoup_pair(g[(uint32_t)k1 * S], P[k1 * C + c]), beta);
        dft_reg_f25<PS::QL>(v);
        const int e0 = ((blk * RDL) << NCOL_LG) + c;
#pragma unroll
        for (int i1 = 0; i1 < RDL; ++i1) tile[tile_at<LOGR>(e0 + (i1 << NCOL_LG))] = v[bitrev_c(i1, PS::QL)];
    }
    __syncthreads();
    if constexpr (PS::NST == 3) {
        tile_step1_25<LOGR, true>(tile, steps);
        __syncthreads();
    }
    // last step (the forward's step 0): parity of the window positions
    {
        const uint32_t lmask = (1u << lgN) - 1;
        const uint2 *tw0 = reinterpret_cast<const uint2 *>(steps) + st25_tab_off(LOGR, 0);
        for (int item = threadIdx.x; item < M0 * C; item += kThreads) {
            const int c = item & (C - 1), i2 = item >> NCOL_LG;
            const uint2 *tw = tw0 + i2;
            const int e0 = item;
            uint32_t v[RD0];
#pragma unroll
            for (int k1 = 0; k1 < RD0; ++k1) {
                const uint32_t x = tile[tile_at<LOGR>(e0 + ((k1 * M0) << NCOL_LG))];
                v[k1] = k1 ? shoup_pair(x, tw[(k1 - 1) * M0]) : f25_red(x);
            }
            dft_reg_f25<PS::Q0>(v);
            const uint32_t g0 = base + (uint32_t)i2 * S + c;
#pragma unroll
            for (int i1 = 0; i1 < RD0; ++i1) {
                const uint32_t n = (lmask + 1 - (g0 + (uint32_t)(M0 * i1) * S)) & lmask;
                const uint64_t p = (uint64_t)n - lo;
                if (n >= lo && p < m) par[p] = (uint8_t)(f25_canon(v[bitrev_c(i1, PS::Q0)]) & 1u);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Fused middle (rows of 2^13), two CTAs of 512 threads per SM.  Per row as
// middle_row_13_f: forward steps 0 and 1 of both operands, per thread 16 rows
// in registers (step 2 of both, the product scaled by L^-1, step 2 of the
// inverse), inverse steps 1 and 0 (every root inverted); step 0 of both
// operands loads from HBM and the last inverse step stores to HBM.  Step 1
// takes Shoup root pairs; step 0's roots (31 x 256 of them) stay single
// words in Montgomery form, so that two CTAs still fit an SM.
// ---------------------------------------------------------------------------
constexpr int kMid0Words = 31 * 256;                         // step 0: omega_8192^(i2 k1) 2^32 mod q
constexpr int kMid1Pairs = st25_tab_words(13) - kMid0Words;  // step 1: root pairs
static_assert(st25_tab_off(13, 1) == kMid0Words, "step 0 of 2^13 has 31 x 256 roots");

__global__ void __launch_bounds__(kThreads, 2)
k25_middle(uint32_t *__restrict__ A, const uint32_t *__restrict__ Bv, uint32_t *__restrict__ Cacc, int mode,
           uint32_t nrows, uint64_t linv, RootTables25 rt) {
    constexpr int Bn = 1 << kMidLgMax;
    static_assert(st_q(13, 0) == 5 && st_q(13, 1) == 4 && st_q(13, 2) == 4 && kThreads == 512,
                  "step 0: one radix-32 column of one operand per thread");
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint2 *pairs1 = reinterpret_cast<uint2 *>(smem_raw);                  // kMid1Pairs
    uint32_t *mont0 = reinterpret_cast<uint32_t *>(pairs1 + kMid1Pairs);  // kMid0Words
    uint32_t *sA = mont0 + kMid0Words;
    uint32_t *sB = sA + sp_size(Bn);
    // rows r, r + grid, ... of both operands (and of the accumulator when it
    // is read), into L2 one row ahead; the first while the tables load
    auto prefetch_row = [&](uint32_t r) {
        const uint32_t at = r << kMidLgMax;
        l2_prefetch(A + at, sizeof(uint32_t) << kMidLgMax);
        l2_prefetch(Bv + at, sizeof(uint32_t) << kMidLgMax);
        if (mode == kMidInner || mode == kMidLast) l2_prefetch(Cacc + at, sizeof(uint32_t) << kMidLgMax);
    };
    if (threadIdx.x == 0 && blockIdx.x < nrows) prefetch_row(blockIdx.x);
    {
        const uint2 *src = reinterpret_cast<const uint2 *>(rt.steps) + (1 << 13) + kMid0Words;
        for (int i = threadIdx.x; i < kMid1Pairs; i += kThreads) pairs1[i] = __ldg(src + i);
        for (int i = threadIdx.x; i < kMid0Words; i += kThreads) {
            const int k1 = 1 + (i >> 8), i2 = i & 255;
            mont0[i] = __ldg(rt.small + i2 * k1);  // omega_8192^(i2 k1), i2 k1 < 8192
        }
    }
    __syncthreads();
    // fwd_step25 / inv_step25 find step J's pairs at pair st25_tab_off(13, J) of
    // their table argument: step 1's pairs sit at that offset from tab1
    const uint32_t *tab1 = reinterpret_cast<const uint32_t *>(pairs1 - kMid0Words);
    const int t = threadIdx.x;
    const int i2 = t & 255;
    const uint32_t *tw0 = mont0 + i2;  // step 0: [(k1 - 1) 256 + i2]
    const int p0 = sp(i2);
    constexpr int STRIDE0 = 256 + 8;  // sp(i2 + 256 k) - sp(i2)
    for (uint32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const uint32_t row = r << kMidLgMax;
        if (t == 0 && r + gridDim.x < nrows) prefetch_row(r + gridDim.x);  // asynchronous: nothing waits
        {
            // step 0: threads 0 .. 255 take A, 256 .. 511 take B
            uint32_t v[32];
            if (t < 256) {
#pragma unroll
                for (int i1 = 0; i1 < 32; ++i1) v[i1] = A[row + i2 + 256 * i1];
            } else {
#pragma unroll
                for (int i1 = 0; i1 < 32; ++i1) v[i1] = __ldg(Bv + row + i2 + 256 * i1);
            }
            dft_reg_f25<5>(v);
            uint32_t *s = t < 256 ? sA : sB;
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                uint32_t x = v[bitrev_c(k1, 5)];
                x = k1 ? f25_mont(x, tw0[(k1 - 1) * 256]) : f25_red(x);
                s[p0 + k1 * STRIDE0] = x;
            }
        }
        __syncthreads();
        fwd_step25<13, 1, 0, 2>(sA, sB, tab1);
        __syncwarp();  // step 1 and the fused step touch the 256-row blocks of the calling warp only
        {
            const int row0 = t << 4;
            const int q0 = sp(row0);  // the 16 rows of a group do not cross a pad word
            uint32_t a[16];
            {
                uint32_t b[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] = sA[q0 + i];
                dft_reg_f25<4>(a);
#pragma unroll
                for (int i = 0; i < 16; ++i) b[i] = sB[q0 + i];
                dft_reg_f25<4>(b);
                // frequency k sits in register bitrev(k) of both
#pragma unroll
                for (int j = 0; j < 16; ++j) a[j] = prod25(a[j], b[j], linv);
            }
            uint32_t c[16];  // the products in frequency order (a renaming of a)
#pragma unroll
            for (int k = 0; k < 16; ++k) c[k] = a[bitrev_c(k, 4)];
            if (mode != kMidAlone) {
                uint4 *g4 = reinterpret_cast<uint4 *>(Cacc + row + row0);
                if (mode != kMidFirst) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 pc = __ldcg(g4 + q);
                        c[4 * q + 0] = f25_add(c[4 * q + 0], pc.x);
                        c[4 * q + 1] = f25_add(c[4 * q + 1], pc.y);
                        c[4 * q + 2] = f25_add(c[4 * q + 2], pc.z);
                        c[4 * q + 3] = f25_add(c[4 * q + 3], pc.w);
                    }
                }
                if (mode != kMidLast) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        g4[q] = make_uint4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
                }
            }
            if (mode == kMidAlone || mode == kMidLast) {
                dft_reg_f25<4>(c);
#pragma unroll
                for (int i = 0; i < 16; ++i) sA[q0 + i] = c[bitrev_c(i, 4)];
            }
        }
        if (mode == kMidFirst || mode == kMidInner) {
            __syncthreads();  // sA / sB free for the next row
            continue;
        }
        __syncwarp();
        inv_step25<13, 1, 0, 1>(sA, sA, tab1);
        __syncthreads();
        if (t < 256) {
            // inverse step 0 (roots inverted) straight to HBM
            uint32_t v[32];
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                const uint32_t x = sA[p0 + k1 * STRIDE0];
                v[k1] = k1 ? f25_mont(x, tw0[(k1 - 1) * 256]) : f25_red(x);
            }
            dft_reg_f25<5>(v);
#pragma unroll
            for (int i1 = 0; i1 < 32; ++i1) A[row + i2 + 256 * i1] = v[bitrev_c(i1, 5)];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
template <int LOGR>
static cudaError_t launch_fwd25_t(const PassArgs &a, cudaStream_t st) {
    using PS = Pass25<LOGR>;
    const size_t sm = PS::W_FWD * sizeof(uint32_t);
    auto kern = k25_fwd<LOGR>;
    cudaError_t e = smem_attr_once<k25_fwd<LOGR>>((int)sm);
    if (e != cudaSuccess) return e;
    const uint32_t tiles = (uint32_t)(a.L >> kTileLg);
    const uint32_t grid = a.data2 ? 2 * tiles : tiles;
    kern<<<grid, kThreads, sm, st>>>(static_cast<uint32_t *>(a.data), a.map, static_cast<uint32_t *>(a.data2), a.map2,
                                     tiles, a.lgN, a.lgS, a.rt25);
    return cudaGetLastError();
}

template <int LOGR>
static cudaError_t launch_inv25_t(const PassArgs &a, cudaStream_t st) {
    using PS = Pass25<LOGR>;
    const size_t sm = PS::W_INV * sizeof(uint32_t);
    auto kern = k25_inv<LOGR>;
    cudaError_t e = smem_attr_once<k25_inv<LOGR>>((int)sm);
    if (e != cudaSuccess) return e;
    const uint32_t tiles = (uint32_t)(a.L >> kTileLg);
    kern<<<tiles, kThreads, sm, st>>>(static_cast<const uint32_t *>(a.data), a.lgN, a.lgS, a.par, a.lo, a.m, a.rt25);
    return cudaGetLastError();
}

bool pass25_fused(const PassArgs &a, int logr) {
    // the single column pass of a transform of 2^22 .. 2^25: forward from bits,
    // inverse with parity out
    return logr >= 9 && logr <= 12 && a.lgN == logr + kMidLgMax && (a.inv ? a.parity_out : a.bits_in);
}

cudaError_t launch_pass25(const PassArgs &a, int logr, cudaStream_t st) {
    if (!pass25_fused(a, logr)) return a.inv ? launch_pass_inv25(a, logr, st) : launch_pass_fwd25(a, logr, st);
    switch (logr) {
        case 9: return a.inv ? launch_inv25_t<9>(a, st) : launch_fwd25_t<9>(a, st);
        case 10: return a.inv ? launch_inv25_t<10>(a, st) : launch_fwd25_t<10>(a, st);
        case 11: return a.inv ? launch_inv25_t<11>(a, st) : launch_fwd25_t<11>(a, st);
        default: return a.inv ? launch_inv25_t<12>(a, st) : launch_fwd25_t<12>(a, st);
    }
}

cudaError_t launch_middle25(void *A, const void *B, void *C, int mode, uint64_t L, uint64_t linv,
                            const RootTables25 &rt, int nsm, cudaStream_t st) {
    const size_t sm = 2 * kMid1Pairs * sizeof(uint32_t) + (kMid0Words + 2 * sp_size(1 << kMidLgMax)) * sizeof(uint32_t);
    cudaError_t e = smem_attr_once<k25_middle>((int)sm);
    if (e != cudaSuccess) return e;
    const uint64_t rows = L >> kMidLgMax;
    const uint64_t grid = rows < 2ull * nsm ? rows : 2ull * nsm;
    k25_middle<<<(unsigned)grid, kThreads, sm, st>>>(static_cast<uint32_t *>(A), static_cast<const uint32_t *>(B),
                                                     static_cast<uint32_t *>(C), C ? mode : (int)kMidAlone,
                                                     (uint32_t)rows, linv, rt);
    return cudaGetLastError();
}

}  // namespace cm
