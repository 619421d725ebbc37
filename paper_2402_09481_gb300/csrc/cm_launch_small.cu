// Launchers of the single-CTA extraction k_fused_small<LG>, LG = 1 .. 13.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_kernels.cuh"

namespace cm {

template <class F, int LG>
static cudaError_t launch_small_f(const Launch &q, const RootTablesT<typename F::T> &rt) {
    const size_t sm = (size_t)small_smem_words<F, LG>() * sizeof(typename F::T);
    auto kern = k_fused_small<F, LG>;
    cudaError_t e = smem_attr_once<k_fused_small<F, LG>>((int)sm);
    if (e != cudaSuccess) return e;
    kern<<<1, kThreads, sm, q.stream>>>(q.amap, q.bmap, q.lo, q.m, q.linv, q.z, q.pre, q.status, rt);
    return cudaGetLastError();
}

template <int LG>
static cudaError_t launch_small_lg(const Launch &q) {
    if (q.field == kFieldF25) return launch_small_f<FieldF25, LG>(q, q.rt25);
    return q.field == kFieldF30 ? launch_small_f<FieldF30, LG>(q, q.rt30) : launch_small_f<FieldGL, LG>(q, q.rt);
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

}  // namespace cm
