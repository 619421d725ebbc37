// Composed two-source extractor (Section "Composing extractors"): a strong
// seeded extractor appended to a strong two-source extractor.  The two-source
// output s = Ext_1(x, y) is the seed of the seeded extractor, whose input is
// the two-source weak seed y; the composed output is s followed by
// t = Ext_2(y, s).  Both stages are the library's own single calls, run in
// stream order; a small kernel appends t after bit m1 of the output.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm.h"
#include "cm_ctx.h"
#include "cm_internal.h"

using namespace cm;

namespace {

// Bits of the seed operand of an extraction of `kind` (cm_kind) with input
// length n and output length m; 0 for an unknown kind.
uint64_t seed_bits(int kind, uint64_t n, uint64_t m) {
    switch (kind) {
        case CM_TOEPLITZ: return n + m - 1;
        case CM_CIRCULANT: return n + 1;
        case CM_DODIS: return n;
        default: return 0;
    }
}

// z bits m1 .. m1 + m2 - 1 <- t bits 0 .. m2 - 1; z bits below m1 are kept and
// bits from m1 + m2 to the end of the last word are written 0.
__global__ void k_append_bits(uint64_t *z, uint64_t m1, const uint64_t *__restrict__ t, uint64_t m2) {
    const uint64_t w0 = m1 >> 6, off = m1 & 63;
    const uint64_t wend = (m1 + m2 + 63) >> 6, tw = (m2 + 63) >> 6;
    for (uint64_t w = w0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < wend;
         w += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = w - w0;
        uint64_t v = j < tw ? t[j] << off : 0;
        if (off && j >= 1 && j - 1 < tw) v |= t[j - 1] >> (64 - off);
        if (j == 0 && off) v |= z[w] & ((1ull << off) - 1);
        const uint64_t used = m1 + m2 - 64 * w;  // bits of this word inside the output (>= 1)
        if (used < 64) v &= (1ull << used) - 1;
        z[w] = v;
    }
}

cm_status run_kind(cm_ctx *ctx, int kind, const uint64_t *x, uint64_t n, const uint64_t *y, uint64_t m, uint64_t *z,
                   cm_stream st) {
    if (kind == CM_TOEPLITZ) return cm_toeplitz(ctx, x, n, y, m, z, st);
    if (kind == CM_CIRCULANT) return cm_circulant(ctx, x, n, y, m, z, st);
    return cm_dodis(ctx, x, y, n, m, z, st);
}

}  // namespace

extern "C" cm_status cm_compose(cm_ctx *ctx, int kind1, const uint64_t *x, uint64_t n1, const uint64_t *y,
                                uint64_t m1, int kind2, uint64_t n2, uint64_t m2, uint64_t *z, cm_stream stream) {
    if (!ctx || !x || !y || !z) return CM_EINVAL;
    // both stages' argument rules (lengths up to 2^40, primes, m <= n) before any work
    if (!valid_args(kind1, n1, m1) || !valid_args(kind2, n2, m2)) return CM_EINVAL;
    if (n2 > seed_bits(kind1, n1, m1) || seed_bits(kind2, n2, m2) > m1) return CM_EINVAL;  // prefixes of y and s
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t tw = (m2 + 63) >> 6;
    void *tbuf = nullptr;
    if (8 * tw > ctx->budget) return CM_ENOMEM;
    if (cudaMallocFromPoolAsync(&tbuf, 8 * tw, ctx->pool, st) != cudaSuccess) {
        cudaGetLastError();
        return CM_ENOMEM;
    }
    uint64_t *t = static_cast<uint64_t *>(tbuf);
    cm_status s = run_kind(ctx, kind1, x, n1, y, m1, z, stream);  // s = Ext_1(x, y) into z
    if (s == CM_OK) s = run_kind(ctx, kind2, y, n2, z, m2, t, stream);  // t = Ext_2(y, s)
    if (s == CM_OK) {
        const uint64_t words = ((m1 + m2 + 63) >> 6) - (m1 >> 6);
        const int threads = 256;
        const uint64_t want = (words + threads - 1) / threads;
        const int blocks = (int)(want < (uint64_t)(4 * ctx->nsm) ? want : (uint64_t)(4 * ctx->nsm));
        ProfScope ps(ctx, "k_append_bits", st);
        k_append_bits<<<blocks, threads, 0, st>>>(z, m1, t, m2);
        if (cudaGetLastError() != cudaSuccess) s = CM_EDEVICE;
    }
    cudaFreeAsync(tbuf, st);
    return s;
}
