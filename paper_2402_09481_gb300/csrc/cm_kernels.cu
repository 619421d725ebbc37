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
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_internal.h"
#include "ntt_device.cuh"

namespace cm {

// ---------------------------------------------------------------------------
// Whole extraction on one CTA (L = 2^LG <= 2^13).
// ---------------------------------------------------------------------------
template <int LG>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_small(BitMap amap, BitMap bmap, uint64_t lo, uint64_t m, uint64_t linv,
              uint64_t *__restrict__ z, const uint32_t *__restrict__ pre,
              uint32_t *__restrict__ status, RootTables rt) {
    constexpr int L = 1 << LG;
    extern __shared__ uint64_t smem[];
    uint64_t *sA = smem;
    uint64_t *sB = smem + sp_size(L);
    for (int i = threadIdx.x; i < L; i += kThreads) {
        sA[sp(i)] = amap.get(i);
        sB[sp(i)] = bmap.get(i);
    }
    __syncthreads();
    ntt_dif<LG, 0, 2>(sA, sB, rt.small_fwd);
    for (int i = threadIdx.x; i < L; i += kThreads)
        sA[sp(i)] = gl_mul(gl_mul(sA[sp(i)], sB[sp(i)]), linv);
    __syncthreads();
    ntt_dit<LG, 0, 1>(sA, sA, rt.small_inv);

    const bool bad = pre && (pre[0] == 0u || pre[1] == 0u);
    if (bad && threadIdx.x == 0) atomicOr(status, kFlagPrecond);
    // window positions lo .. lo + m - 1, parity packed by warp ballots
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t nwords = (m + 63) >> 6;
    for (uint64_t w = warp; w < nwords; w += kThreads / 32) {
        const uint64_t p0 = (w << 6) + lane, p1 = p0 + 32;
        const uint32_t b0 = (p0 < m) ? (uint32_t)(sA[sp((int)(lo + p0))] & 1u) : 0u;
        const uint32_t b1 = (p1 < m) ? (uint32_t)(sA[sp((int)(lo + p1))] & 1u) : 0u;
        const uint32_t w0 = __ballot_sync(0xffffffffu, b0);
        const uint32_t w1 = __ballot_sync(0xffffffffu, b1);
        if (lane == 0) z[w] = bad ? 0ull : ((uint64_t)w1 << 32 | w0);
    }
}

// ---------------------------------------------------------------------------
// One column pass over tiles of R = 2^LOGR rows x C = 2^(kTileLg - LOGR) columns.
// ---------------------------------------------------------------------------
template <int LOGR, bool INV, bool BITS_IN, bool PARITY_OUT>
__global__ void __launch_bounds__(kThreads, 1)
k_pass(uint64_t *__restrict__ data, BitMap map, int lgN, int lgS, uint8_t *__restrict__ par,
       uint64_t lo, uint64_t m, RootTables rt) {
    constexpr int R = 1 << LOGR;
    constexpr int NCOL_LG = kTileLg - LOGR;
    constexpr int C = 1 << NCOL_LG;
    extern __shared__ uint64_t smem[];
    const uint64_t S = 1ull << lgS;
    const uint64_t tiles_per_blk = S >> NCOL_LG;
    const uint64_t tile = blockIdx.x;
    const uint64_t blk = tile / tiles_per_blk;
    const uint64_t col0 = (tile - blk * tiles_per_blk) << NCOL_LG;
    const uint64_t base = (blk << lgN) + col0;
    const int esh = 32 - lgN;  // omega_N = g^(2^(32 - lgN))

    for (int e = threadIdx.x; e < R * C; e += kThreads) {
        const int i = e >> NCOL_LG, c = e & (C - 1);
        const uint64_t g = base + ((uint64_t)i << lgS) + c;
        uint64_t v = BITS_IN ? map.get(g) : data[g];
        if (INV) {
            const uint32_t E = (uint32_t)(((col0 + c) * (uint64_t)i) << esh);
            if (E) v = gl_mul(v, big_root(rt.big_lo_inv, rt.big_hi_inv, E));
        }
        smem[sp(e)] = v;
    }
    __syncthreads();
    ntt_dif<LOGR, NCOL_LG, 1>(smem, smem, INV ? rt.small_inv : rt.small_fwd);
    for (int e = threadIdx.x; e < R * C; e += kThreads) {
        const int k = e >> NCOL_LG, c = e & (C - 1);
        uint64_t v = smem[sp((bitrev(k, LOGR) << NCOL_LG) + c)];
        const uint64_t g = base + ((uint64_t)k << lgS) + c;
        if (!INV) {
            const uint32_t E = (uint32_t)(((col0 + c) * (uint64_t)k) << esh);
            if (E) v = gl_mul(v, big_root(rt.big_lo_fwd, rt.big_hi_fwd, E));
        }
        if (PARITY_OUT) {
            const uint64_t p = g - lo;
            if (g >= lo && p < m) par[p] = (uint8_t)(v & 1u);
        } else {
            data[g] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Fused middle: rows of B = 2^13 contiguous elements of both operands.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1)
k_middle(uint64_t *__restrict__ A, const uint64_t *__restrict__ Bv, uint64_t linv, RootTables rt) {
    constexpr int LG = kMidLgMax;
    constexpr int Bn = 1 << LG;
    extern __shared__ uint64_t smem[];
    uint64_t *sA = smem;
    uint64_t *sB = smem + sp_size(Bn);
    const uint64_t row = (uint64_t)blockIdx.x << LG;
    const ulonglong2 *a2 = reinterpret_cast<const ulonglong2 *>(A + row);
    const ulonglong2 *b2 = reinterpret_cast<const ulonglong2 *>(Bv + row);
    for (int i = threadIdx.x; i < Bn / 2; i += kThreads) {
        const ulonglong2 va = a2[i], vb = __ldg(b2 + i);
        sA[sp(2 * i)] = va.x;
        sA[sp(2 * i + 1)] = va.y;
        sB[sp(2 * i)] = vb.x;
        sB[sp(2 * i + 1)] = vb.y;
    }
    __syncthreads();
    ntt_dif<LG, 0, 2>(sA, sB, rt.small_fwd);
    for (int i = threadIdx.x; i < Bn; i += kThreads)
        sA[sp(i)] = gl_mul(gl_mul(sA[sp(i)], sB[sp(i)]), linv);
    __syncthreads();
    ntt_dit<LG, 0, 1>(sA, sA, rt.small_inv);
    ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(A + row);
    for (int i = threadIdx.x; i < Bn / 2; i += kThreads)
        o2[i] = make_ulonglong2(sA[sp(2 * i)], sA[sp(2 * i + 1)]);
}

// ---------------------------------------------------------------------------
// Parity bytes -> packed words.  One warp builds one 64-bit word per iteration.
// ---------------------------------------------------------------------------
__global__ void k_pack(const uint8_t *__restrict__ par, uint64_t m, uint64_t *__restrict__ z,
                       const uint32_t *__restrict__ pre, uint32_t *__restrict__ status) {
    const bool bad = pre && (pre[0] == 0u || pre[1] == 0u);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kFlagPrecond);
    const int lane = threadIdx.x & 31;
    const uint64_t nwords = (m + 63) >> 6;
    const uint64_t wstride = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t w = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nwords;
         w += wstride) {
        const uint64_t p0 = (w << 6) + lane, p1 = p0 + 32;
        const uint32_t b0 = (p0 < m) ? par[p0] : 0u;
        const uint32_t b1 = (p1 < m) ? par[p1] : 0u;
        const uint32_t w0 = __ballot_sync(0xffffffffu, b0);
        const uint32_t w1 = __ballot_sync(0xffffffffu, b1);
        if (lane == 0) z[w] = bad ? 0ull : ((uint64_t)w1 << 32 | w0);
    }
}

// flags[0] |= 1 if some bit of x[0..n) is 1; flags[1] |= 1 if some bit is 0.
__global__ void k_allsame(const uint64_t *__restrict__ x, uint64_t n, uint32_t *__restrict__ flags) {
    const uint64_t nw = (n + 63) >> 6;
    uint32_t any1 = 0, any0 = 0;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t mask = ~0ull;
        if (w == nw - 1 && (n & 63)) mask = (1ull << (n & 63)) - 1;
        const uint64_t v = __ldg(x + w);
        any1 |= (v & mask) != 0;
        any0 |= (~v & mask) != 0;
    }
    any1 = __any_sync(0xffffffffu, any1);
    any0 = __any_sync(0xffffffffu, any0);
    if ((threadIdx.x & 31) == 0) {
        if (any1) atomicOr(flags + 0, 1u);
        if (any0) atomicOr(flags + 1, 1u);
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
template <int LG>
static cudaError_t launch_small_lg(const Launch &q) {
    const size_t sm = 2 * sp_size(1 << LG) * sizeof(uint64_t);
    auto kern = k_fused_small<LG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<1, kThreads, sm, q.stream>>>(q.amap, q.bmap, q.lo, q.m, q.linv, q.z, q.pre, q.status, q.rt);
    return cudaGetLastError();
}

cudaError_t launch_small(const Launch &q, int lg) {
    switch (lg) {
#define CM_CASE(k) case k: return launch_small_lg<k>(q);
        CM_CASE(1) CM_CASE(2) CM_CASE(3) CM_CASE(4) CM_CASE(5) CM_CASE(6) CM_CASE(7)
        CM_CASE(8) CM_CASE(9) CM_CASE(10) CM_CASE(11) CM_CASE(12) CM_CASE(13)
#undef CM_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <int LOGR, bool INV, bool BITS_IN, bool PARITY_OUT>
static cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st) {
    const size_t sm = sp_size(1 << kTileLg) * sizeof(uint64_t);
    auto kern = k_pass<LOGR, INV, BITS_IN, PARITY_OUT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = a.L >> kTileLg;
    kern<<<(unsigned)tiles, kThreads, sm, st>>>(a.data, a.map, a.lgN, a.lgS, a.par, a.lo, a.m, a.rt);
    return cudaGetLastError();
}

template <int LOGR>
static cudaError_t launch_pass_r(const PassArgs &a, cudaStream_t st) {
    if (!a.inv) {
        return a.bits_in ? launch_pass_t<LOGR, false, true, false>(a, st)
                         : launch_pass_t<LOGR, false, false, false>(a, st);
    }
    return a.parity_out ? launch_pass_t<LOGR, true, false, true>(a, st)
                        : launch_pass_t<LOGR, true, false, false>(a, st);
}

cudaError_t launch_pass(const PassArgs &a, int logr, cudaStream_t st) {
    switch (logr) {
#define CM_CASE(k) case k: return launch_pass_r<k>(a, st);
        CM_CASE(1) CM_CASE(2) CM_CASE(3) CM_CASE(4) CM_CASE(5) CM_CASE(6)
        CM_CASE(7) CM_CASE(8) CM_CASE(9) CM_CASE(10) CM_CASE(11) CM_CASE(12)
#undef CM_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_middle(uint64_t *A, const uint64_t *B, uint64_t L, uint64_t linv,
                          const RootTables &rt, cudaStream_t st) {
    const size_t sm = 2 * sp_size(1 << kMidLgMax) * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(k_middle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_middle<<<(unsigned)(L >> kMidLgMax), kThreads, sm, st>>>(A, B, linv, rt);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t *par, uint64_t m, uint64_t *z, const uint32_t *pre,
                        uint32_t *status, int nsm, cudaStream_t st) {
    const uint64_t nwords = (m + 63) >> 6;
    uint64_t blocks = (nwords + 7) / 8;  // 8 warps per block
    const uint64_t cap = (uint64_t)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    k_pack<<<(unsigned)blocks, 256, 0, st>>>(par, m, z, pre, status);
    return cudaGetLastError();
}

cudaError_t launch_allsame(const uint64_t *x, uint64_t n, uint32_t *flags, int nsm, cudaStream_t st) {
    const uint64_t nw = (n + 63) >> 6;
    uint64_t blocks = (nw + 255) / 256;
    const uint64_t cap = (uint64_t)nsm * 4;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    k_allsame<<<(unsigned)blocks, 256, 0, st>>>(x, n, flags);
    return cudaGetLastError();
}

}  // namespace cm
