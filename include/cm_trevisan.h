/*
 * Trevisan's extractor, one-bit step on the GPU (Section "Trevisan
 * implementation" of arXiv 2402.09481; the paper names a GPU version of this
 * step as future work, Section "Conclusion and future work").
 *
 * Trevisan(x, y)_i = Ext1(x, y_{S_i}) for the sets S_1 .. S_m of a weak design
 * over the seed y.  Ext1 is the Reed-Solomon-Hadamard (RSH) one-bit
 * extractor: with l bits per field element (l = ceil(log2 n + 2 log2(2/eps1)),
 * eps1 the per-bit error),
 *   - the input x (n bits) is cut into s = ceil(n / l) chunks x_1 .. x_s of l
 *     bits, the last padded with 0s; a chunk is an element of GF(2^l) by its
 *     binary representation, the chunk's first bit the most significant
 *     coefficient (the paper's example: l = 3, {0, 0, 1} is the element 1);
 *   - alpha1 = the first l bits of the one-bit seed, alpha2 = the next l bits,
 *     read the same way;
 *   - p = sum_{i=1..s} x_i alpha1^(s-i) in GF(2^l) (Eq. poly), and the output
 *     bit is the GF(2) inner product of the coefficients of alpha2 and p.
 * The paper does not fix the representation of GF(2^l): this library takes
 * GF(2)[x] modulo the irreducible trinomial x^l + x^k + 1 with the smallest
 * k, or, where none exists, the irreducible pentanomial
 * x^l + x^a + x^b + x^c + 1 (l > a > b > c > 0) with the smallest (a, b, c)
 * in lexicographic order (cm_rsh_modulus).  The paper's weak design (the
 * block weak design of Mauerer et al.) is cited, not stated, so the sets are
 * an input (cm_trevisan) or the callers pass the one-bit seeds directly
 * (cm_trevisan_rsh).
 *
 * Bit strings are uint64 words, bit i at word i >> 6, bit i & 63; device
 * pointers, stream-ordered like cm_toeplitz; output tail bits are written 0.
 */
#ifndef CM_TREVISAN_H
#define CM_TREVISAN_H

#include <stdint.h>

#include "cm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* l = ceil(log2(n) + 2 log2(2 / eps1)); 0 if n = 0 or eps1 is not in (0, 1). */
uint32_t cm_rsh_field_bits(uint64_t n, double eps1);

/* The GF(2^l) modulus used for l (2 <= l <= 256): *count = 1 and taps[0] = k
 * for x^l + x^k + 1, or *count = 3 and taps = {a, b, c} for
 * x^l + x^a + x^b + x^c + 1.  Host only.  CM_EINVAL for l outside 2 .. 256. */
cm_status cm_rsh_modulus(uint32_t l, uint32_t taps[3], uint32_t *count);

/* m RSH one-bit extractions of x (n bits, 1 <= n <= 2^40): output bit i
 * (z: ceil(m/64) words, written) uses the 2l-bit one-bit seed at bits
 * 2 l i .. 2 l i + 2l - 1 of `seeds` (ceil(2 l m / 64) words).  2 <= l <= 256,
 * 1 <= m <= 2^32.  Scratch: ceil(n / l) chunks of ceil(l / 64) words, from
 * the context's pool.  CM_EINVAL for bad arguments, CM_ENOMEM over the HBM
 * budget. */
cm_status cm_trevisan_rsh(cm_ctx *ctx, const uint64_t *x, uint64_t n, uint32_t l, const uint64_t *seeds,
                          uint64_t m, uint64_t *z, cm_stream stream);

/* Trevisan(x, y): sets is an m x t row-major array of seed indices (device,
 * uint32, each < d, every row in increasing order), the weak design's
 * S_1 .. S_m; the one-bit seed of output i is y at sets[i][0 .. 2l), read in
 * the order given (t >= 2l; entries past 2l are not read; an index >= d
 * reads 0).  y: d bits.  Otherwise as cm_trevisan_rsh
 * (plus 2 l m bits of scratch for the gathered seeds). */
cm_status cm_trevisan(cm_ctx *ctx, const uint64_t *x, uint64_t n, const uint64_t *y, uint64_t d,
                      const uint32_t *sets, uint32_t t, uint64_t m, uint32_t l, uint64_t *z, cm_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* CM_TREVISAN_H */
