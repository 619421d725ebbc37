/*
 * cm_vn.h -- Von Neumann extractor on the GPU, part of libcm.so.
 *
 * Section "Von Neumann" and Alg. vn of arXiv 2402.09481: for
 * j = 0 .. floor(n/2) - 1 the pair (x_{2j}, x_{2j+1}) yields the output bit
 * x_{2j} when the two bits differ and nothing when they are equal; outputs keep
 * the order of j.  A trailing odd bit belongs to no pair.  The output length m
 * (the number of unequal pairs) is known only after the pass.  Alg. vn ends in
 * an error step for an input whose bits are all the same; here the extraction
 * fails when it yields no output bit (m = 0).
 *
 * Bit strings use the packed layout of cm.h (bit i is bit i & 63 of word
 * i >> 6, least significant first).
 */
#ifndef CM_VN_H
#define CM_VN_H

#include <stdint.h>

#include "cm.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Von Neumann extraction of the n-bit string x into z on the device: a pair
 * filter and an order-keeping bit compaction, as three kernels (per-tile counts
 * and their scan, zeroing of the output words that tiles share, compression
 * and write-out at the scanned offsets).
 *
 * x: device, ceil(n/64) words, 16-byte aligned.  z: device, 8-byte aligned,
 * room for ceil(floor(n/2)/64) words (the most the output can take).  m_out:
 * device pointer to one uint64_t that receives m.  On return of the stream
 * work z holds the m output bits in words 0 .. ceil(m/64) - 1, the bits past m
 * in the last of them are 0, and later words of z are not written.  The call
 * is asynchronous on `stream`; scratch (64.25 KiB + 12 bytes per 4096 input
 * words) comes from the context pool.
 *
 * Errors: CM_EINVAL for a NULL pointer, n < 2 (no pair), a misaligned pointer
 * or n >= 2^46.  If every pair is equal the call still returns CM_OK,
 * *m_out = 0 and cm_device_status() reports CM_EPRECOND (the error of Alg. vn).
 * No CTA waits on another: the scan runs in the CTA that finishes counting
 * last.
 */
cm_status cm_von_neumann(cm_ctx *ctx, const uint64_t *x, uint64_t n, uint64_t *z, uint64_t *m_out,
                         cm_stream stream);

/*
 * The same on HOST buffers, synchronous: copies x host->device, runs the
 * extraction, reads m, copies ceil(m/64) words of z device->host and
 * synchronizes `stream`.  x_host: ceil(n/64) words; z_host: room for
 * ceil(floor(n/2)/64) words; *m receives the output length.  Returns
 * CM_EPRECOND (with *m = 0) when every pair is equal (the context's device
 * status also records it); argument errors as cm_von_neumann.
 */
cm_status cm_von_neumann_host(cm_ctx *ctx, const uint64_t *x_host, uint64_t n, uint64_t *z_host,
                              uint64_t *m, cm_stream stream);

/* Scratch bytes cm_von_neumann takes from the pool for an n-bit input. */
uint64_t cm_von_neumann_scratch_bytes(uint64_t n);

#ifdef __cplusplus
}
#endif

#endif /* CM_VN_H */
