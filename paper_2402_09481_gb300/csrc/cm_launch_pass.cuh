// Launcher templates of the column passes k_pass<F, LOGR, ...>; each field's
// forward and inverse launchers live in their own translation unit so that the
// instantiations compile in parallel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_kernels.cuh"

namespace cm {

template <class F>
static const RootTablesT<typename F::T> &pass_tables(const PassArgs &a);
template <>
inline const RootTables &pass_tables<FieldGL>(const PassArgs &a) { return a.rt; }
template <>
inline const RootTables30 &pass_tables<FieldF30>(const PassArgs &a) { return a.rt30; }
template <>
inline const RootTables25 &pass_tables<FieldF25>(const PassArgs &a) { return a.rt25; }

template <class F, int LOGR, bool INV, bool BITS_IN, bool PARITY_OUT>
static cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st) {
    using T = typename F::T;
    constexpr int TILE_LG = LOGR + F::ncol_lg(LOGR);
    constexpr bool BTAB = pass_bits_table<F, LOGR, INV, BITS_IN>();
    const size_t sm =
        (BTAB ? pass_table_off<F, LOGR>() + kBitsTable : pass_tw_off<F, LOGR>() + pass_tw_words<F, LOGR>()) *
        sizeof(T);
    auto kern = k_pass<F, LOGR, INV, BITS_IN, PARITY_OUT>;
    cudaError_t e = smem_attr_once<k_pass<F, LOGR, INV, BITS_IN, PARITY_OUT>>((int)sm);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = a.L >> TILE_LG;
    const uint64_t grid = a.data2 ? 2 * tiles : tiles;
    kern<<<(unsigned)grid, kThreads, sm, st>>>(static_cast<T *>(a.data), a.map, static_cast<T *>(a.data2), a.map2,
                                                tiles, a.lgN, a.lgS, a.par, a.lo, a.m, pass_tables<F>(a));
    return cudaGetLastError();
}

template <class F, int LOGR>
static cudaError_t launch_fwd_r(const PassArgs &a, cudaStream_t st) {
    return a.bits_in ? launch_pass_t<F, LOGR, false, true, false>(a, st)
                     : launch_pass_t<F, LOGR, false, false, false>(a, st);
}

template <class F, int LOGR>
static cudaError_t launch_inv_r(const PassArgs &a, cudaStream_t st) {
    return a.parity_out ? launch_pass_t<F, LOGR, true, false, true>(a, st)
                        : launch_pass_t<F, LOGR, true, false, false>(a, st);
}

template <class F, bool INV, int LOGR>
static cudaError_t launch_r(const PassArgs &a, cudaStream_t st) {
    if constexpr (INV)
        return launch_inv_r<F, LOGR>(a, st);
    else
        return launch_fwd_r<F, LOGR>(a, st);
}

template <class F, bool INV>
static cudaError_t launch_pass_dispatch(const PassArgs &a, int logr, cudaStream_t st) {
    switch (logr) {
#define CM_CASE(k) case k: return launch_r<F, INV, k>(a, st);
        CM_CASE(1) CM_CASE(2) CM_CASE(3) CM_CASE(4) CM_CASE(5) CM_CASE(6)
        CM_CASE(7) CM_CASE(8) CM_CASE(9) CM_CASE(10) CM_CASE(11) CM_CASE(12)
#undef CM_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
