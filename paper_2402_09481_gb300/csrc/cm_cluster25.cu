// Whole extraction for transform lengths L = CL * 2^13 (2^14 .. 2^17) in ONE
// launch: a thread-block cluster of CL CTAs holds both operands in
// distributed shared memory, 2^13 elements of each per CTA, over the lazily
// reduced field of 5 * 2^25 + 1.
//
// The transform is the four-step split of Def. ntt with the CL-point DFTs
// across the cluster: with n = p M + j (M = 2^13, p < CL) and k = k1 + CL k2,
//   X[k] = sum_j omega_M^(j k2) [omega_L^(j k1) sum_p x[p M + j] omega_CL^(p k1)].
//   0. CTA p unpacks input bits p M .. p M + M - 1 of both operands.
//   1. CTA r takes columns j of its slice (M / CL of them), reads x[p M + j]
//      from every CTA p (DSMEM loads), runs the CL-point DFT in registers,
//      multiplies output k1 by omega_L^(j k1) and stores it back to CTA k1
//      at position j (DSMEM stores): CTA k1 then holds the sequence of k1.
//   2. Every CTA transforms its 2^13 elements on chip (ntt25.cuh), forms the
//      pointwise product with L^-1 (Thm. convolution) and runs the transform
//      with every root inverted, which leaves u_k1[j] = sum_k2 P[k1 + CL k2]
//      omega_M^(j k2) at position j.
//   3. The inverse across the cluster takes the same forward roots:
//      out[p M + j] = sum_k1 omega_CL^(p k1) (omega_L^(j k1) u_k1[j]), and
//      out[g] is the convolution coefficient (L - g) mod L (ntt25.cuh).
//   4. Parities of the output window [lo, lo + m) go into a bitmap spread
//      over the cluster's shared memory (warp ballots, DSMEM atomics), and
//      each CTA writes its words of z.
// Cluster barriers separate the phases; no CTA touches another's shared
// memory after the last one.  The step roots of the on-chip transforms are
// copied asynchronously while the cross-cluster step runs.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_internal.h"
#include "ntt25.cuh"
#include "ntt_device.cuh"

namespace cg = cooperative_groups;

namespace cm {
namespace {

constexpr int kClM = 1 << kMidLgMax;  // elements of each operand per CTA
constexpr int kClBits = kClM / 32;    // output bitmap words per CTA (L / 32 in all)

__host__ __device__ constexpr int lg_of(int v) { return v <= 1 ? 0 : 1 + lg_of(v / 2); }

// Shared memory (words): both operands, the step root pairs of length 2^13
// (16-byte aligned: 2 sp_size(2^13) + 2 is a multiple of 4), the bitmap
// slice, then the cross-step roots omega_L^(k1 j) (Montgomery form) at
// [(k1 - 1) J + jj] for k1 = 1 .. CL - 1 and this CTA's columns j = r J + jj
// (J = 2^13 / CL).
constexpr int kClTabOff = 2 * sp_size(kClM) + 2;
constexpr int kClBitsOff = kClTabOff + st25_smem_words(kMidLgMax);
constexpr int kClRootOff = kClBitsOff + kClBits;
constexpr size_t cluster_smem_words(int cl) { return (size_t)kClRootOff + (size_t)(cl - 1) * (kClM / cl); }

// Distributed shared memory through its 32-bit shared::cluster addresses.
// Ordering against the phases comes from the cluster barriers (which the
// compiler does not move these across), so the accesses carry no memory
// clobber and the compiler may interleave them with shared-memory loads.
__device__ __forceinline__ uint32_t cl_mapa(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ uint32_t cl_ld(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void cl_st(uint32_t a, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v));
}
// The two halves of a cluster barrier: every thread of the cluster arrives
// once (its earlier shared-memory writes released), then waits for all.
__device__ __forceinline__ void cl_arrive_release() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cl_wait_acquire() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
__device__ __forceinline__ void cl_or(uint32_t a, uint32_t v) {
    asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// OR run R (bit b = output bit s + b) into the cluster's output bitmap, bits
// outside [0, m) dropped.  Output bit i is bit i & 31 of word (i >> 5) % kClBits
// of CTA (i >> 5) / kClBits; bits0 is the bitmap's shared::cluster address in
// this CTA.
__device__ __forceinline__ void or_run(uint32_t bits0, uint32_t R, int64_t s, uint64_t m) {
    if (s <= -32 || s >= (int64_t)m) return;
    if (s < 0) R &= ~0u << (uint32_t)(-s);
    const int64_t keep = (int64_t)m - s;
    if (keep < 32) R &= (1u << keep) - 1u;
    if (!R) return;
    const int64_t w = s >> 5;  // floor
    const uint32_t sh = (uint32_t)(s & 31);
    const uint32_t lo = R << sh, hi = sh ? R >> (32 - sh) : 0u;
    if (lo && w >= 0) cl_or(cl_mapa(bits0, (uint32_t)(w / kClBits)) + 4u * (uint32_t)(w % kClBits), lo);
    if (hi) cl_or(cl_mapa(bits0, (uint32_t)((w + 1) / kClBits)) + 4u * (uint32_t)((w + 1) % kClBits), hi);
}

template <int CL>
__global__ void __launch_bounds__(kThreads, 1)
k25_cluster(BitMap amap, BitMap bmap, uint64_t lo, uint64_t m, uint64_t linv, uint64_t *__restrict__ z,
            const uint32_t *__restrict__ pre, uint32_t *__restrict__ status, RootTables25 rt) {
    constexpr int LQ = lg_of(CL), LG = kMidLgMax + LQ;
    constexpr int64_t L = 1ll << LG;
    constexpr int J = kClM / CL;           // columns of the cross-cluster steps per CTA
    constexpr int ESH = kF25MaxLg - LG;    // omega_L = g^(2^ESH), g of order 2^25
    static_assert(J % kThreads == 0, "whole warps of consecutive columns");
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int lane = threadIdx.x & 31;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint32_t *sA = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *sB = sA + sp_size(kClM);
    uint32_t *tw = sA + kClTabOff;
    uint32_t *bits = sA + kClBitsOff;
    uint32_t *roots = sA + kClRootOff;
    // shared::cluster address of word 0 in CTA p: rank p's operands, bitmap
    const uint32_t base0 = (uint32_t)__cvta_generic_to_shared(sA);
    uint32_t base[CL];
#pragma unroll
    for (int p = 0; p < CL; ++p) base[p] = cl_mapa(base0, (uint32_t)p);
    const uint32_t bits0 = base0 + 4u * kClBitsOff;

    prefetch_steps25<kMidLgMax>(tw, rt.steps);  // needed from phase 2 on
    for (int i = threadIdx.x; i < kClBits; i += kThreads) bits[i] = 0u;
    // 0. operands: one run of 32 positions per thread (kClM / 32 runs each),
    //    read as one or two words; thread t of a warp writes run t at
    //    sp(32 t + i), bank (t + i) mod 32: no conflicts
    for (int u = threadIdx.x; u < 2 * (kClM / 32); u += kThreads) {
        const int op = u >= kClM / 32 ? 1 : 0;
        const int run = u - op * (kClM / 32);
        const uint32_t bitsr = (op ? bmap : amap).get_run<32>((uint64_t)r * kClM + 32 * run);
        uint32_t *dst = (op ? sB : sA) + sp(32 * run);
#pragma unroll
        for (int i = 0; i < 32; ++i) dst[i] = (bitsr >> i) & 1u;
    }
    // the operands are what the other CTAs read in phase 1: publish them, and
    // compute the cross-step roots while the other CTAs catch up (each root is
    // written and read by one thread of this CTA only: the same jj mapping in
    // phases 1 and 3)
    cl_arrive_release();
    // cross-step roots: the powers of omega_L^j for this thread's columns
    for (int jj = threadIdx.x; jj < J; jj += kThreads) {
        const uint32_t w = big_root_f<FieldF25>(rt.big_lo_fwd, rt.big_hi_fwd, (uint32_t)(r * J + jj) << ESH);
        uint32_t wk = w;
#pragma unroll
        for (int k1 = 1; k1 < CL; ++k1) {
            roots[(k1 - 1) * J + jj] = wk;
            if (k1 + 1 < CL) wk = FieldF25::twmul(wk, w);
        }
    }
    cl_wait_acquire();  // every CTA of the cluster runs and its operands are in place

    // 1. CL-point DFTs across the cluster, both operands of column j together
    //    (all 2 CL remote loads in flight); column j is read and written by
    //    this thread only
    for (int jj = threadIdx.x; jj < J; jj += kThreads) {
        const uint32_t oA = 4u * (uint32_t)sp(r * J + jj), oB = oA + 4u * (uint32_t)sp_size(kClM);
        uint32_t va[CL], vb[CL];
#pragma unroll
        for (int p = 0; p < CL; ++p) {
            va[p] = cl_ld(base[p] + oA);
            vb[p] = cl_ld(base[p] + oB);
        }
        dft_reg_f25<LQ>(va);
        dft_reg_f25<LQ>(vb);
        cl_st(base[0] + oA, f25_red(va[0]));
        cl_st(base[0] + oB, f25_red(vb[0]));
#pragma unroll
        for (int k1 = 1; k1 < CL; ++k1) {
            const uint32_t w = roots[(k1 - 1) * J + jj];
            cl_st(base[k1] + oA, FieldF25::twmul(f25_red(va[bitrev_c(k1, LQ)]), w));
            cl_st(base[k1] + oB, FieldF25::twmul(f25_red(vb[bitrev_c(k1, LQ)]), w));
        }
    }
    cp_async_wait_all();  // this thread's step roots have landed; the barrier publishes them
    cluster.sync();

    // 2. on-chip transforms, product, transform with inverted roots
    ntt_fwd25<kMidLgMax, 0, 2>(sA, sB, tw);
    for (int i = threadIdx.x; i < kClM; i += kThreads) sA[sp(i)] = prod25(sA[sp(i)], sB[sp(i)], linv);
    __syncthreads();
    ntt_inv25<kMidLgMax, 0, 1>(sA, sA, tw);
    cluster.sync();

    // 3. inverse across the cluster, 4. window parities into the bitmap
    for (int jj = threadIdx.x; jj < J; jj += kThreads) {
        const int j = r * J + jj;
        const uint32_t oA = 4u * (uint32_t)sp(j);
        uint32_t v[CL];
#pragma unroll
        for (int k1 = 0; k1 < CL; ++k1) v[k1] = cl_ld(base[k1] + oA);
        v[0] = f25_red(v[0]);
#pragma unroll
        for (int k1 = 1; k1 < CL; ++k1) v[k1] = FieldF25::twmul(f25_red(v[k1]), roots[(k1 - 1) * J + jj]);
        dft_reg_f25<LQ>(v);
        // lane p keeps the ballot of output p (positions p M + j0 + t, t < 32)
        uint32_t mine = 0;
#pragma unroll
        for (int p = 0; p < CL; ++p) {
            const uint32_t b = __ballot_sync(0xffffffffu, f25_canon(v[bitrev_c(p, LQ)]) & 1u);
            if (lane == p) mine = b;
        }
        if (lane < CL) {
            // lanes t of the ballot hold coefficient (L - g0 - t) mod L
            const int64_t g0 = (int64_t)lane * kClM + (j - lane);
            if (g0 == 0) {  // position 0 holds coefficient 0
                if ((mine & 1u) && lo == 0) or_run(bits0, 1u, 0, m);
                mine &= ~1u;
            }
            // reversed: bit b <- lane 31 - b, coefficient L - g0 - 31 + b
            or_run(bits0, __brev(mine), L - g0 - 31 - (int64_t)lo, m);
        }
    }
    cluster.sync();

    const bool bad = pre && (pre[0] == 0u || pre[1] == 0u);
    if (bad && r == 0 && threadIdx.x == 0) atomicOr(status, kFlagPrecond);
    const uint64_t nwords = (m + 63) >> 6;
    for (int w = threadIdx.x; w < kClBits / 2; w += kThreads) {
        const uint64_t zw = (uint64_t)r * (kClBits / 2) + w;
        if (zw < nwords) z[zw] = bad ? 0ull : ((uint64_t)bits[2 * w + 1] << 32 | bits[2 * w]);
    }
}

template <int CL>
cudaLaunchConfig_t cluster_config(cudaStream_t st, cudaLaunchAttribute *at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = cluster_smem_words(CL) * sizeof(uint32_t);
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// Kernel attributes (once per CUDA context) and whether one cluster fits.
template <int CL>
cudaError_t cluster_prepare(bool *fits) {
    *fits = false;
    cudaError_t e = smem_attr_once<k25_cluster<CL>>((int)(cluster_smem_words(CL) * sizeof(uint32_t)));
    if (e != cudaSuccess) return e;
    if (CL > 8 && (e = cudaFuncSetAttribute(k25_cluster<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
                      cudaSuccess)
        return e;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_config<CL>(nullptr, at);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k25_cluster<CL>, &cfg);
    if (e != cudaSuccess) return e;
    *fits = n >= 1;
    return cudaSuccess;
}

template <int CL>
cudaError_t launch_t(const Launch &q) {
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_config<CL>(q.stream, at);
    return cudaLaunchKernelEx(&cfg, k25_cluster<CL>, q.amap, q.bmap, q.lo, q.m, (uint64_t)q.linv, q.z, q.pre,
                              q.status, q.rt25);
}

}  // namespace

cudaError_t cluster25_prepare(int lg, bool *fits) {
    switch (lg) {
        case 14: return cluster_prepare<2>(fits);
        case 15: return cluster_prepare<4>(fits);
        case 16: return cluster_prepare<8>(fits);
        case 17: return cluster_prepare<16>(fits);
        default: *fits = false; return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cluster25(const Launch &q, int lg) {
    switch (lg) {
        case 14: return launch_t<2>(q);
        case 15: return launch_t<4>(q);
        case 16: return launch_t<8>(q);
        case 17: return launch_t<16>(q);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
