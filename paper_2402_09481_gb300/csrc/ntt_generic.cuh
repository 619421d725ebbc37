// Runtime-size on-chip transforms for the batched work-list kernel, over a
// field policy F of ntt_device.cuh (lazily reduced fields: every step brings
// its DFT inputs below 2q by the root product or F::red, as in ntt_device.cuh).
//
// Same mixed-radix decimation-in-frequency steps as ntt_device.cuh (the
// four-step split of Def. ntt applied recursively over shared memory, with
// power-of-two twiddles inside each register sub-transform), but the column
// length R = 2^logr and the column count are runtime values, so one kernel can
// serve every instance of a batch.  Radices are at most 16 (q <= 4); the
// register sub-transform is the only compile-time part.  All roots come from
// one shared-memory table of omega_8192^e, e < 8192, read with stride
// 2^(13 - logr).
#pragma once
#include <stdint.h>

#include "ntt_device.cuh"

namespace cm {

__host__ __device__ constexpr int rt_nsteps(int logr) { return (logr + 3) / 4; }
__host__ __device__ inline int rt_q(int logr, int j) {
    const int n = rt_nsteps(logr);
    return logr / n + (j < logr % n ? 1 : 0);
}

template <class F, int LQ, bool INV>
__device__ __forceinline__ void step_rt(typename F::T *s0, typename F::T *s1, int nbuf, int logr, int off,
                                        int ncol_lg, const typename F::T *tw8192) {
    using T = typename F::T;
    constexpr int RD = 1 << LQ;
    const int LN = logr - off, LM = LN - LQ;
    const int items = (1 << (logr - LQ)) << ncol_lg;
    const int tws = off + kSmallLg - logr;
    const int cmask = (1 << ncol_lg) - 1, mmask = (1 << LM) - 1;
    for (int item = threadIdx.x; item < items * nbuf; item += kThreads) {
        const int bi = item >= items;
        const int it = item - (bi ? items : 0);
        T *s = bi ? s1 : s0;
        const int c = it & cmask;
        const int rest = it >> ncol_lg;
        const int i2 = rest & mmask;
        const int row0 = ((rest >> LM) << LN) + i2;
        T v[RD];
        if (!INV) {
#pragma unroll
            for (int i1 = 0; i1 < RD; ++i1) v[i1] = s[sp(((row0 + (i1 << LM)) << ncol_lg) + c)];
            dft_reg_f<F, LQ>(v);
#pragma unroll
            for (int k1 = 0; k1 < RD; ++k1) {
                T x = v[bitrev_c(k1, LQ)];
                if (k1 > 0 && i2 > 0) {
                    x = F::twmul(x, tw8192[tw_swz((i2 * k1) << tws)]);
                } else {
                    x = F::red(x);  // lazy fields: back below 2q for the next step
                }
                s[sp(((row0 + (k1 << LM)) << ncol_lg) + c)] = x;
            }
        } else {
#pragma unroll
            for (int k1 = 0; k1 < RD; ++k1) {
                T x = s[sp(((row0 + (k1 << LM)) << ncol_lg) + c)];
                if (k1 > 0 && i2 > 0) {
                    x = F::twmul(x, tw8192[tw_swz((8192 - ((i2 * k1) << tws)) & 8191)]);
                } else {
                    x = F::red(x);
                }
                v[k1] = x;
            }
            dft_reg_f<F, LQ>(v);
#pragma unroll
            for (int i1 = 0; i1 < RD; ++i1)
                s[sp(((row0 + (i1 << LM)) << ncol_lg) + c)] = v[bitrev_c((RD - i1) & (RD - 1), LQ)];
        }
    }
}

template <class F, bool INV>
__device__ __forceinline__ void step_dispatch(int q, typename F::T *s0, typename F::T *s1, int nbuf, int logr,
                                              int off, int ncol_lg, const typename F::T *tw) {
    switch (q) {
        case 1: step_rt<F, 1, INV>(s0, s1, nbuf, logr, off, ncol_lg, tw); break;
        case 2: step_rt<F, 2, INV>(s0, s1, nbuf, logr, off, ncol_lg, tw); break;
        case 3: step_rt<F, 3, INV>(s0, s1, nbuf, logr, off, ncol_lg, tw); break;
        default: step_rt<F, 4, INV>(s0, s1, nbuf, logr, off, ncol_lg, tw); break;
    }
}

// Forward transform of every column (natural -> digit-reversed); ends with a barrier.
template <class F>
__device__ __forceinline__ void ntt_fwd_rt(typename F::T *s0, typename F::T *s1, int nbuf, int logr, int ncol_lg,
                                           const typename F::T *tw) {
    int off = 0;
    for (int j = 0; j < rt_nsteps(logr); ++j) {
        const int q = rt_q(logr, j);
        step_dispatch<F, false>(q, s0, s1, nbuf, logr, off, ncol_lg, tw);
        __syncthreads();
        off += q;
    }
}

// Inverse of ntt_fwd_rt up to the factor R; ends with a barrier.
template <class F>
__device__ __forceinline__ void ntt_inv_rt(typename F::T *s0, typename F::T *s1, int nbuf, int logr, int ncol_lg,
                                           const typename F::T *tw) {
    int off = logr;
    for (int j = rt_nsteps(logr) - 1; j >= 0; --j) {
        const int q = rt_q(logr, j);
        off -= q;
        step_dispatch<F, true>(q, s0, s1, nbuf, logr, off, ncol_lg, tw);
        __syncthreads();
    }
}

// Frequency held at position p after ntt_fwd_rt(logr).
__device__ __forceinline__ uint32_t pos_to_freq_rt(uint32_t p, int logr) {
    uint32_t f = 0;
    int off = 0;
    for (int j = 0; j < rt_nsteps(logr); ++j) {
        const int q = rt_q(logr, j);
        f |= ((p >> (logr - off - q)) & ((1u << q) - 1)) << off;
        off += q;
    }
    return f;
}

}  // namespace cm
