// Launchers of the fused middle, the pack and the precondition kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_kernels.cuh"

namespace cm {

// ---------------------------------------------------------------------------
// Fused middle: rows of B = 2^13 contiguous elements of both operands.
// ---------------------------------------------------------------------------
template <class F>
__global__ void __launch_bounds__(kThreads, sizeof(typename F::T) == 4 ? 2 : 1)
k_middle(typename F::T *__restrict__ A, const typename F::T *__restrict__ Bv, typename F::T *__restrict__ C,
         int mode, uint64_t nrows, uint64_t linv_, RootTablesT<typename F::T> rt) {
    using T = typename F::T;
    constexpr int LG = kMidLgMax;
    constexpr int Bn = 1 << LG;
    constexpr int PER = 16 / sizeof(T);  // elements per 16-byte access
    const T linv = (T)linv_;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    T *sB = sA + sp_size(Bn);
    T *tw = sB + sp_size(Bn);
    load_roots<LG>(tw, rt.small);
    // persistent: each CTA walks rows blockIdx.x, blockIdx.x + gridDim.x, ...
    for (uint64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const uint64_t row = r << LG;
        const uint4 *a4 = reinterpret_cast<const uint4 *>(A + row);
        const uint4 *b4 = reinterpret_cast<const uint4 *>(Bv + row);
        for (int i = threadIdx.x; i < Bn / PER; i += kThreads) {
            T pa[PER], pb[PER];
            unpack16(a4[i], pa);
            unpack16(__ldg(b4 + i), pb);
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                sA[sp(PER * i + j)] = pa[j];
                sB[sp(PER * i + j)] = pb[j];
            }
        }
        __syncthreads();
        middle_row_13_f<F>(sA, sB, tw, linv, C ? C + row : nullptr, mode);
        if (mode == kMidFirst || mode == kMidInner) continue;  // the product went to C
        // result row -> A (in place)
        uint4 *o4 = reinterpret_cast<uint4 *>(A + row);
        for (int i = threadIdx.x; i < Bn / PER; i += kThreads) {
            T pv[PER];
#pragma unroll
            for (int j = 0; j < PER; ++j) pv[j] = sA[sp(PER * i + j)];
            o4[i] = pack16(pv);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Parity bytes -> packed words.  Over the floor(m / 512) whole groups of 512
// positions a warp builds eight 64-bit words per iteration; past them, one.
// ---------------------------------------------------------------------------
__global__ void k_pack(const uint8_t *__restrict__ par, uint64_t m, uint64_t *__restrict__ z,
                       const uint32_t *__restrict__ pre, uint32_t *__restrict__ status) {
    const bool bad = pre && (pre[0] == 0u || pre[1] == 0u);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kFlagPrecond);
    const int lane = threadIdx.x & 31;
    const uint64_t nwords = (m + 63) >> 6;
    const uint64_t wstride = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t warp0 = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // Groups of 8 words whose 512 parity bytes all lie below m: one 16-byte
    // load per lane (16 positions), packed by a multiply per 4 bytes (bytes are
    // 0 or 1: byte 3 of x * 0x01020408 is b0 + 2 b1 + 4 b2 + 8 b3, no carries),
    // and four lanes' 16 bits joined by shuffles into one word.
    const uint64_t ngroups = (reinterpret_cast<uintptr_t>(par) & 15) ? 0 : (m >> 9);
    for (uint64_t g = warp0; g < ngroups; g += wstride) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(par + (g << 9)) + lane);
        const uint32_t u = ((v.x * 0x01020408u) >> 24) | (((v.y * 0x01020408u) >> 24) << 4) |
                           (((v.z * 0x01020408u) >> 24) << 8) | (((v.w * 0x01020408u) >> 24) << 12);
        const uint32_t t = u | (__shfl_down_sync(0xffffffffu, u, 1) << 16);
        const uint32_t t2 = __shfl_down_sync(0xffffffffu, t, 2);
        if ((lane & 3) == 0) z[(g << 3) + (lane >> 2)] = bad ? 0ull : ((uint64_t)t2 << 32 | t);
    }
    for (uint64_t w = (ngroups << 3) + warp0; w < nwords; w += wstride) {
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

cudaError_t launch_pass(const PassArgs &a, int logr, cudaStream_t st) {
    if (a.field == kFieldF25) return launch_pass25(a, logr, st);
    if (a.field == kFieldF30) return a.inv ? launch_pass_inv30(a, logr, st) : launch_pass_fwd30(a, logr, st);
    return a.inv ? launch_pass_inv(a, logr, st) : launch_pass_fwd(a, logr, st);
}

template <class F>
static cudaError_t launch_middle_f(void *A, const void *B, void *C, int mode, uint64_t L, uint64_t linv,
                                   const RootTablesT<typename F::T> &rt, int nsm, cudaStream_t st) {
    using T = typename F::T;
    const size_t sm = (2 * sp_size(1 << kMidLgMax) + (1 << kMidLgMax)) * sizeof(T);
    cudaError_t e = smem_attr_once<k_middle<F>>((int)sm);
    if (e != cudaSuccess) return e;
    const uint64_t rows = L >> kMidLgMax;
    const uint64_t per_sm = sizeof(T) == 4 ? 2 : 1;  // resident CTAs per SM (shared memory, registers)
    const uint64_t grid = rows < per_sm * nsm ? rows : per_sm * nsm;
    k_middle<F><<<(unsigned)grid, kThreads, sm, st>>>(static_cast<T *>(A), static_cast<const T *>(B),
                                                      static_cast<T *>(C), C ? mode : (int)kMidAlone, rows, linv,
                                                      rt);
    return cudaGetLastError();
}

cudaError_t launch_middle(int field, void *A, const void *B, void *C, int mode, uint64_t L, uint64_t linv,
                          const RootTables &rt, const RootTables30 &rt30, const RootTables25 &rt25, int nsm,
                          cudaStream_t st) {
    if (field == kFieldF25) return launch_middle25(A, B, C, mode, L, linv, rt25, nsm, st);
    return field == kFieldF30 ? launch_middle_f<FieldF30>(A, B, C, mode, L, linv, rt30, nsm, st)
                              : launch_middle_f<FieldGL>(A, B, C, mode, L, linv, rt, nsm, st);
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

// z[i] ^= t[i]: joins the output windows of a blocked extraction.
__global__ void k_xor_into(uint64_t *__restrict__ z, const uint64_t *__restrict__ t, uint64_t words) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x)
        z[i] ^= t[i];
}

cudaError_t launch_xor_into(uint64_t *z, const uint64_t *t, uint64_t words, int nsm, cudaStream_t st) {
    uint64_t blocks = (words + 255) / 256;
    const uint64_t cap = (uint64_t)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    k_xor_into<<<(unsigned)blocks, 256, 0, st>>>(z, t, words);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dense tail of a middle product: z_i ^= sum_{t<T} a_t b_{t+i} (mod 2), i < m,
// with a_t = A_{K-1-t} and b_v = B_v read through the product's operand maps,
// T <= kTailMax.  The CTA gathers the T tail bits of a once (warp ballots into
// shared memory); then one thread builds one 64-bit output word: the 64 + T - 1
// seed bits it needs sit in registers, and every tail term with a_t = 1 XORs
// in the 64-bit run of them that starts at offset t.
// ---------------------------------------------------------------------------
constexpr int kTailThreads = 256;
static_assert(kTailMax == kTailThreads && kTailMax % 64 == 0, "one tail bit per thread");

// One output word of the tail: the XOR over the set tail bits t of the 64
// seed bits starting at offset t of W (W[q] = seed bits 64 q .. 64 q + 63 of
// this word's run).  sal holds the tail bits, 32 a word; they are the same in
// every thread, so the loop over the set ones does not diverge and runs about
// T / 2 times; each 64-bit run is two 32-bit funnel shifts.
template <int NW>
__device__ __forceinline__ uint64_t tail_word(const uint32_t *sal, const uint64_t (&W)[NW + 1]) {
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int h = 0; h < 2 * NW; ++h) {
        // offsets 32 h .. 32 h + 31: 32-bit words h, h + 1, h + 2 of the run
        const uint32_t v0 = h & 1 ? (uint32_t)(W[h >> 1] >> 32) : (uint32_t)W[h >> 1];
        const uint32_t v1 = h & 1 ? (uint32_t)W[(h >> 1) + 1] : (uint32_t)(W[h >> 1] >> 32);
        const uint32_t v2 = h & 1 ? (uint32_t)(W[(h >> 1) + 1] >> 32) : (uint32_t)W[(h >> 1) + 1];
        uint32_t l2 = 0, h2 = 0;  // a second pair of accumulators: two chains
        uint32_t a = sal[h];
        while (a) {
            const int s = __ffs(a) - 1;
            a &= a - 1;
            lo ^= __funnelshift_r(v0, v1, s);
            hi ^= __funnelshift_r(v1, v2, s);
            if (!a) break;
            const int u = __ffs(a) - 1;
            a &= a - 1;
            l2 ^= __funnelshift_r(v0, v1, u);
            h2 ^= __funnelshift_r(v1, v2, u);
        }
        lo ^= l2;
        hi ^= h2;
    }
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

// Seed positions k .. k + 64 (NW + 1) - 1 of map b as NW + 1 words: when the
// run maps to one run of source bits (no cut at len, no wrap, not reversed)
// from NW + 1 or NW + 2 word loads; else position by position in a loop that
// is not unrolled (runs at the ends of the window only), so that the code a
// warp executes stays a few hundred instructions: these kernels run one short
// wave, and their time goes to fetching the instructions they run.
template <int NW>
__device__ __forceinline__ void seed_words(const BitMap &b, uint64_t k, uint64_t (&W)[NW + 1]) {
    constexpr uint64_t kSpan = 64 * (NW + 1);
    if (k + kSpan <= b.len && b.mode != kReverse) {
        uint64_t lo = k;
        if (b.mode == kModForward) {
            lo = k + b.off;
            if (lo >= b.srclen) lo -= b.srclen;
            if (lo >= b.srclen) lo -= b.srclen;
        }
        if (lo + kSpan <= b.srclen) {
            const uint64_t *src = b.src + (lo >> 6);
            const int sh = (int)(lo & 63);
            uint64_t u[NW + 2];
#pragma unroll
            for (int q = 0; q <= NW; ++q) u[q] = __ldg(src + q);
            // the word after the run's last is read only when the run reaches into it
            u[NW + 1] = sh ? __ldg(src + NW + 1) : 0ull;
#pragma unroll
            for (int q = 0; q <= NW; ++q) W[q] = sh ? (u[q] >> sh) | (u[q + 1] << (64 - sh)) : u[q];
            return;
        }
    }
#pragma unroll
    for (int q = 0; q <= NW; ++q) {
        uint64_t v = 0;
#pragma unroll 1
        for (int j = 0; j < 64; ++j) v |= b.get(k + 64 * q + j) << j;
        W[q] = v;
    }
}

// NW = ceil(T / 64) words of tail bits.
template <int NW>
__global__ void __launch_bounds__(kTailThreads)
k_tail(BitMap amap, BitMap bmap, uint64_t K, uint32_t T, uint64_t m, uint64_t *__restrict__ z,
       const uint32_t *__restrict__ pre) {
    if (pre && (pre[0] == 0u || pre[1] == 0u)) return;  // the pack kernel left z zero
    __shared__ uint32_t sal[kTailMax / 32];
    {
        const int t = threadIdx.x;  // one tail position per thread
        const uint32_t bit = (uint32_t)t < T ? (uint32_t)amap.get(K - 1 - (uint64_t)t) : 0u;
        const uint32_t w = __ballot_sync(0xffffffffu, bit);
        if ((t & 31) == 0) sal[t >> 5] = w;
    }
    __syncthreads();
    const uint64_t nwords = (m + 63) >> 6;
    for (uint64_t w = (uint64_t)blockIdx.x * kTailThreads + threadIdx.x; w < nwords;
         w += (uint64_t)gridDim.x * kTailThreads) {
        uint64_t W[NW + 1];  // seed bits 64 w .. 64 w + 64 (NW + 1) - 1
        seed_words<NW>(bmap, w << 6, W);
        uint64_t acc = tail_word<NW>(sal, W);
        if (w == nwords - 1 && (m & 63)) acc &= (1ull << (m & 63)) - 1;
        z[w] ^= acc;
    }
}

cudaError_t launch_tail(const BitMap &amap, const BitMap &bmap, uint64_t K, uint32_t T, uint64_t m, uint64_t *z,
                        const uint32_t *pre, int nsm, cudaStream_t st) {
    if (T == 0 || T > (uint32_t)kTailMax || T > K) return cudaErrorInvalidValue;
    const uint64_t nwords = (m + 63) >> 6;
    uint64_t blocks = (nwords + kTailThreads - 1) / kTailThreads;
    const uint64_t cap = (uint64_t)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    switch ((T + 63) / 64) {
        case 1: k_tail<1><<<(unsigned)blocks, kTailThreads, 0, st>>>(amap, bmap, K, T, m, z, pre); break;
        case 2: k_tail<2><<<(unsigned)blocks, kTailThreads, 0, st>>>(amap, bmap, K, T, m, z, pre); break;
        case 3: k_tail<3><<<(unsigned)blocks, kTailThreads, 0, st>>>(amap, bmap, K, T, m, z, pre); break;
        default: k_tail<4><<<(unsigned)blocks, kTailThreads, 0, st>>>(amap, bmap, K, T, m, z, pre); break;
    }
    return cudaGetLastError();
}

// k_pack and k_tail in one pass: one thread per output word (the grid covers
// every word) XORs the tail terms (tail_word) into its 64 packed parity bytes
// (four 16-byte loads when the word lies below m).  The tail depends on the
// input bits only, the parity bytes on the kernel before (the inverse pass):
// launched as its programmatic dependent, the kernel computes the tail while
// that pass's last CTAs still run and waits for it (griddepcontrol.wait, which
// returns at once in an ordinary launch) only before it reads the parity.
template <int NW>
__global__ void __launch_bounds__(kTailThreads)
k_pack_tail(const uint8_t *__restrict__ par, uint64_t m, uint64_t *__restrict__ z, const uint32_t *__restrict__ pre,
            uint32_t *__restrict__ status, BitMap amap, BitMap bmap, uint64_t K, uint32_t T) {
    __shared__ uint32_t sal[kTailMax / 32];
    const uint64_t nwords = (m + 63) >> 6;
    const uint64_t w = (uint64_t)blockIdx.x * kTailThreads + threadIdx.x;  // one word a thread (grid covers m)
    uint64_t W[NW + 1];  // seed bits 64 w .. 64 w + 64 (NW + 1) - 1
    if (w < nwords) {
        seed_words<NW>(bmap, w << 6, W);
    } else {
#pragma unroll
        for (int q = 0; q <= NW; ++q) W[q] = 0;
    }
    {
        const int t = threadIdx.x;  // one tail position per thread
        const uint32_t bit = (uint32_t)t < T ? (uint32_t)amap.get(K - 1 - (uint64_t)t) : 0u;
        const uint32_t b = __ballot_sync(0xffffffffu, bit);
        if ((t & 31) == 0) sal[t >> 5] = b;
    }
    // the precondition flags come from a kernel that finished before the
    // inverse pass began
    const bool bad = pre && (pre[0] == 0u || pre[1] == 0u);
    if (bad && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kFlagPrecond);
    __syncthreads();
    if (w >= nwords) return;
    uint64_t acc = tail_word<NW>(sal, W);
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the parity bytes are complete and visible
    uint64_t packed = 0;
    if ((reinterpret_cast<uintptr_t>(par) & 15) == 0 && (w << 6) + 64 <= m) {
        const uint4 *src = reinterpret_cast<const uint4 *>(par + (w << 6));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint4 v = __ldcg(src + k);  // L2, never a line an L1 kept from before the wait
            const uint64_t u = ((v.x * 0x01020408u) >> 24) | (((v.y * 0x01020408u) >> 24) << 4) |
                               (((v.z * 0x01020408u) >> 24) << 8) | (((v.w * 0x01020408u) >> 24) << 12);
            packed |= u << (16 * k);
        }
    } else {
#pragma unroll 1
        for (int b = 0; b < 64; ++b) {
            const uint64_t p = (w << 6) + b;
            if (p < m) packed |= (uint64_t)(__ldcg(par + p) & 1u) << b;
        }
    }
    acc ^= packed;
    if (w == nwords - 1 && (m & 63)) acc &= (1ull << (m & 63)) - 1;
    z[w] = bad ? 0ull : acc;
}

cudaError_t launch_pack_tail(const uint8_t *par, uint64_t m, uint64_t *z, const uint32_t *pre, uint32_t *status,
                             const TailArgs &a, int nsm, cudaStream_t st) {
    if (a.T == 0 || a.T > (uint32_t)kTailMax || a.T > a.K) return cudaErrorInvalidValue;
    const uint64_t nwords = (m + 63) >> 6;
    const uint64_t blocks = (nwords + kTailThreads - 1) / kTailThreads;  // one word a thread
    if (blocks == 0 || blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    (void)nsm;
    // a programmatic dependent of the kernel before it, except under stream
    // capture (the graphs of a batch keep plain edges)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return cudaGetLastError();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kTailThreads);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
    auto go = [&](auto kern) { return cudaLaunchKernelEx(&cfg, kern, par, m, z, pre, status, a.amap, a.bmap, a.K, a.T); };
    switch ((a.T + 63) / 64) {
        case 1: return go(k_pack_tail<1>);
        case 2: return go(k_pack_tail<2>);
        case 3: return go(k_pack_tail<3>);
        default: return go(k_pack_tail<4>);
    }
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

namespace cm {

// Field self-test: the device arithmetic (PTX carry chains) against the C
// forms, on edge values and SplitMix64 samples; counts disagreements.
__global__ void k_field_selftest(uint64_t count, uint64_t seed, unsigned long long *bad) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    auto mix = [](uint64_t z) {
        z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
        z ^= z >> 27; z *= 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    const uint64_t edge[12] = {0, 1, 2, 0xFFFFFFFFull, 0x100000000ull, 0xFFFFFFFF00000000ull,
                               GL_P - 1, GL_P - 2, 0x7FFFFFFFFFFFFFFFull, 0x8000000000000000ull,
                               0xFFFFFFFEFFFFFFFFull, 0x00000000FFFFFFFEull};
    uint64_t a = mix(seed + 2 * i * 0x9E3779B97F4A7C15ull), b = mix(seed + (2 * i + 1) * 0x9E3779B97F4A7C15ull);
    if (i < 144) {
        a = edge[i % 12];
        b = edge[i / 12];
    }
    a = gl_canon(a);
    b = gl_canon(b);
    unsigned long long n = 0;
    n += gl_add_ptx(a, b) != gl_add_c(a, b);
    n += gl_sub_ptx(a, b) != gl_sub_c(a, b);
    n += gl_mul_ptx(a, b) != gl_mul_c(a, b);
#pragma unroll
    for (int s = 0; s <= 96; ++s) n += gl_shl_ptx(a, s) != gl_shl_c(a, s);
    // the 32-bit field against plain 64-bit modular arithmetic
    const uint32_t e30[8] = {0u, 1u, 2u, F30_Q - 1, F30_Q - 2, 0x80000000u, 0x7FFFFFFFu, F30_R};
    uint32_t a3 = (uint32_t)(a % F30_Q), b3 = (uint32_t)(b % F30_Q);
    if (i < 64) {
        a3 = e30[i % 8];
        b3 = e30[i / 8];
    }
    constexpr uint32_t rinv = f30_pow(F30_R, F30_Q - 2);
    n += f30_add(a3, b3) != (uint32_t)(((uint64_t)a3 + b3) % F30_Q);
    n += f30_sub(a3, b3) != (uint32_t)(((uint64_t)a3 + F30_Q - b3) % F30_Q);
    n += f30_mont(a3, b3) != f30_mulmod(f30_mulmod(a3, b3), rinv);
    const uint32_t w32 = f30_pow(F30_G30, 1ull << 25);
    uint32_t wj = 1;
    for (int j = 0; j < 32; ++j) {
        n += f30_mont(a3, kF30Tw32[j]) != f30_mulmod(a3, wj);
        wj = f30_mulmod(wj, w32);
    }
    // the lazily reduced field: values and ranges.  x is any 32-bit word (the
    // representatives the kernels hold), c, d canonical, e, f in [0, 2q).
    {
        constexpr uint64_t Q = F25_Q;
        constexpr uint32_t rinv25 = f25_pow(F25_R, F25_Q - 2);
        const uint32_t ex[8] = {0u, 1u, F25_Q - 1, F25_Q, 2 * F25_Q - 1, 12 * F25_Q, 0x7FFFFFFFu, 0xFFFFFFFFu};
        const uint32_t x = i < 64 ? ex[i % 8] : (uint32_t)(a >> 32);
        const uint32_t c = i < 64 ? (uint32_t)(ex[i / 8] % Q) : (uint32_t)(b % Q);
        const uint32_t d = (uint32_t)((a ^ b) % Q);
        const uint32_t e = (uint32_t)(a % (2 * Q)), f = i < 64 ? (uint32_t)(ex[i / 8] % (2 * Q)) : (uint32_t)(b % (2 * Q));
        const uint32_t r = f25_red(x), k = f25_canon(x);
        n += r >= 2 * Q || r % Q != x % Q;
        n += k != x % Q;
        const uint32_t ad = f25_add(e, f), sb = f25_sub(e, f);
        n += ad >= 2 * Q || ad % Q != (e + (uint64_t)f) % Q;
        n += sb >= 2 * Q || sb % Q != (e % Q + Q - f % Q) % Q;
        const uint32_t mo = f25_mont(x, c);  // any x, canonical root
        n += mo == 0 || mo >= 2 * Q || mo % Q != f25_mulmod(f25_mulmod((uint32_t)(x % Q), c), rinv25);
        if (x < 0x80000000u) {  // x < 2^31, root in [0, 2q)
            const uint32_t m2 = f25_mont(x, f);
            n += m2 >= 2 * Q || m2 % Q != f25_mulmod(f25_mulmod((uint32_t)(x % Q), (uint32_t)(f % Q)), rinv25);
        }
        const uint32_t sh = f25_shoup(x, d, f25_shoup_q(d));
        n += sh >= 2 * Q || sh % Q != f25_mulmod((uint32_t)(x % Q), d);
        const uint32_t w25 = f25_pow(F25_G25, 1ull << 20);
        uint32_t wk = 1;
        for (int j = 0; j < 32; ++j) {
            const uint32_t t = f25_shoup(x, kF25W32[j], kF25W32Q[j]);
            n += t >= 2 * Q || t % Q != f25_mulmod((uint32_t)(x % Q), wk);
            wk = f25_mulmod(wk, w25);
        }
    }
    if (n) atomicAdd(bad, n);
}

}  // namespace cm

namespace cm {

// Independent chains x <- x w of the field's product, kChains per thread;
// the chains' sum goes to *sink so that nothing is dead code.  The lazily
// reduced field times its Shoup product by a constant root (the product its
// transforms use for constant and table roots).
constexpr int kChains = 8;
template <class F>
__global__ void __launch_bounds__(256) k_modmul_rate(uint32_t iters, typename F::T w, typename F::T *sink) {
    using T = typename F::T;
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + 977u * (c + 1) + blockIdx.x);
    const uint32_t wq = F::kLazy ? f25_shoup_q((uint32_t)w) : 0u;
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if constexpr (F::kLazy)
                x[c] = f25_shoup(x[c], (uint32_t)w, wq);
            else
                x[c] = F::twmul(x[c], w);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == (T)0x5bd1e995u) *sink = s;  // practically never; keeps the chains live
}

template <class F>
static cm_status modmul_rate(int nsm, typename F::T w, double *rate) {
    using T = typename F::T;
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return CM_ENOMEM;
    cudaEvent_t a = nullptr, b = nullptr;
    cm_status st = CM_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) st = CM_EDEVICE;
    const unsigned grid = 4u * (unsigned)nsm;
    const uint32_t iters = 4096;
    float ms = 0.f;
    if (st == CM_OK) {
        k_modmul_rate<F><<<grid, 256>>>(iters, w, sink);  // warm-up
        cudaEventRecord(a);
        k_modmul_rate<F><<<grid, 256>>>(iters, w, sink);
        cudaEventRecord(b);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.f)
            st = CM_EDEVICE;
    }
    if (st == CM_OK) *rate = (double)grid * 256.0 * kChains * iters / (ms * 1e-3);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(sink);
    return st;
}

}  // namespace cm

extern "C" cm_status cm_modmul_rate(int device, uint32_t field, double *per_second) {
    if (!per_second || (field != CM_FIELD_GOLDILOCKS && field != CM_FIELD_Q30 && field != CM_FIELD_Q25))
        return CM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return CM_EDEVICE;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return CM_EDEVICE;
    if (field == CM_FIELD_Q30) return cm::modmul_rate<cm::FieldF30>(nsm, f30_to_mont(12345u), per_second);
    if (field == CM_FIELD_Q25) return cm::modmul_rate<cm::FieldF25>(nsm, 12345u, per_second);
    return cm::modmul_rate<cm::FieldGL>(nsm, 0x123456789ABCDEFull, per_second);
}

extern "C" cm_status cm_field_selftest(int device, uint64_t count, uint64_t seed, uint64_t *mismatches) {
    if (!mismatches) return CM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return CM_EDEVICE;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return CM_ENOMEM;
    cm_status st = CM_OK;
    unsigned long long h = 0;
    if (cudaMemset(d, 0, sizeof(*d)) != cudaSuccess) st = CM_EDEVICE;
    if (st == CM_OK) {
        const uint64_t blocks = (count + 255) / 256;
        cm::k_field_selftest<<<(unsigned)(blocks ? blocks : 1), 256>>>(count, seed, d);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = CM_EDEVICE;
    }
    cudaFree(d);
    *mismatches = h;
    return st;
}
