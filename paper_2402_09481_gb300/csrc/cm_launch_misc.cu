// Launchers of the fused middle, the pack and the precondition kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_kernels.cuh"

namespace cm {

// ---------------------------------------------------------------------------
// Fused middle: rows of B = 2^13 contiguous elements of both operands.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1)
k_middle(uint64_t *__restrict__ A, const uint64_t *__restrict__ Bv, uint64_t nrows, uint64_t linv,
         RootTables rt) {
    constexpr int LG = kMidLgMax;
    constexpr int Bn = 1 << LG;
    extern __shared__ uint64_t smem[];
    uint64_t *sA = smem;
    uint64_t *sB = smem + sp_size(Bn);
    uint64_t *tw = sB + sp_size(Bn);
    load_roots<LG>(tw, rt.small);
    // persistent: each CTA walks rows blockIdx.x, blockIdx.x + gridDim.x, ...
    for (uint64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const uint64_t row = r << LG;
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
        middle_row_13(sA, sB, tw, linv);
        ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(A + row);
        for (int i = threadIdx.x; i < Bn / 2; i += kThreads)
            o2[i] = make_ulonglong2(sA[sp(2 * i)], sA[sp(2 * i + 1)]);
        __syncthreads();
    }
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

cudaError_t launch_pass(const PassArgs &a, int logr, cudaStream_t st) {
    return a.inv ? launch_pass_inv(a, logr, st) : launch_pass_fwd(a, logr, st);
}

cudaError_t launch_middle(uint64_t *A, const uint64_t *B, uint64_t L, uint64_t linv,
                          const RootTables &rt, int nsm, cudaStream_t st) {
    const size_t sm = (2 * sp_size(1 << kMidLgMax) + (1 << kMidLgMax)) * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(k_middle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const uint64_t rows = L >> kMidLgMax;
    const uint64_t grid = rows < (uint64_t)nsm ? rows : (uint64_t)nsm;
    k_middle<<<(unsigned)grid, kThreads, sm, st>>>(A, B, rows, linv, rt);
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
    if (n) atomicAdd(bad, n);
}

}  // namespace cm

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
