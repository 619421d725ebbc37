// Launchers of the forward column passes k_pass<LOGR, fwd, ...>.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_kernels.cuh"

namespace cm {

template <int LOGR, bool INV, bool BITS_IN, bool PARITY_OUT>
static cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t st) {
    const size_t sm = (sp_size(1 << kTileLg) + (1 << LOGR)) * sizeof(uint64_t);
    auto kern = k_pass<LOGR, INV, BITS_IN, PARITY_OUT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = a.L >> kTileLg;
    kern<<<(unsigned)tiles, kThreads, sm, st>>>(a.data, a.map, a.lgN, a.lgS, a.par, a.lo, a.m, a.rt);
    return cudaGetLastError();
}

template <int LOGR>
static cudaError_t launch_fwd_r(const PassArgs &a, cudaStream_t st) {
    return a.bits_in ? launch_pass_t<LOGR, false, true, false>(a, st)
                     : launch_pass_t<LOGR, false, false, false>(a, st);
}

cudaError_t launch_pass_fwd(const PassArgs &a, int logr, cudaStream_t st) {
    switch (logr) {
#define CM_CASE(k) case k: return launch_fwd_r<k>(a, st);
        CM_CASE(1) CM_CASE(2) CM_CASE(3) CM_CASE(4) CM_CASE(5) CM_CASE(6)
        CM_CASE(7) CM_CASE(8) CM_CASE(9) CM_CASE(10) CM_CASE(11) CM_CASE(12)
#undef CM_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
