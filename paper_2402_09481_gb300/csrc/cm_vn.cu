// Von Neumann extractor (Section "Von Neumann", Alg. vn): pair filter and
// order-keeping bit compaction on the GPU.
//
// The input is cut into tiles of 4096 words (32 KiB).  Three kernels, with no
// waiting between CTAs:
//
//   k_vn_count  reads each tile once and counts its unequal pairs (a popcount
//               of the pair-difference mask per word).  Each CTA (4 per SM)
//               takes a chunk of consecutive tiles and records each tile's
//               offset inside the chunk; the CTA that finishes last (a
//               done-counter taken after a memory fence, so every other CTA's
//               sums are visible to it) turns the chunk sums into chunk
//               offsets and writes m.
//   k_vn_zero   zeroes the output words that two or more tiles share (a tile's
//               first and last word when only partly its own), a thread a tile.
//   k_vn_write  re-reads each tile, compresses every word with a 64 KiB
//               shared-memory table (one byte per 16-bit chunk: the outputs of
//               those 8 pairs, in order), packs the bits into a shared staging
//               buffer aligned to the tile's global output offset, and writes
//               the words it alone owns with plain coalesced stores and the
//               shared ones with atomic ORs into the zeroed words.
//
// So each output word is written once (or ORed together from pieces), nothing
// is zero-filled in bulk, and the cost over a single pass is the second read of
// the input.  k_vn_write walks tiles blockIdx.x, + gridDim.x, ... with the next
// tile's words loading into registers while the current one is written out.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_ctx.h"
#include "cm_internal.h"
#include "cm_vn.h"

namespace cm {
namespace {

constexpr int kVnTileWords = 4096;                      // 32 KiB of input
constexpr int kCountThreads = 512;                      // k_vn_count: 8 words a thread per tile
constexpr int kCountWpt = kVnTileWords / kCountThreads;
constexpr int kWriteThreads = 512;                      // k_vn_write: 8 words a thread
constexpr int kVnWpt = kVnTileWords / kWriteThreads;
constexpr int kVnStageWords = kVnTileWords / 2 + 2;     // <= 32 bits a word, + offset word, + guard
constexpr size_t kWriteSmem = 65536 + 8 * (size_t)kVnStageWords + 2 * 256 + 4 * 64;
constexpr size_t kVnHeaderBytes = 256;                  // done counter
constexpr uint32_t kMaxChunks = 4096;                   // count CTAs (4 per SM) at most

// This thread's CNT consecutive words starting at word w0: zeros past the
// input, the last word masked to whole pairs (pairs past floor(n/2) count as
// equal and give nothing).
template <int CNT>
__device__ __forceinline__ void vn_load(const uint64_t *__restrict__ x, uint64_t words, uint64_t lastmask,
                                        uint64_t w0, uint64_t (&wv)[CNT]) {
    if (w0 + CNT <= words) {
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(x + w0);
#pragma unroll
        for (int i = 0; i < CNT / 2; ++i) {
            const ulonglong2 v = __ldg(p + i);
            wv[2 * i] = v.x;
            wv[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < CNT; ++i) wv[i] = (w0 + i < words) ? __ldg(x + w0 + i) : 0ull;
    }
    if (w0 + CNT >= words) {
#pragma unroll
        for (int i = 0; i < CNT; ++i)
            if (w0 + i == words - 1) wv[i] &= lastmask;
    }
}

__device__ __forceinline__ uint32_t pair_count(uint64_t w) {
    const uint64_t d = (w ^ (w >> 1)) & 0x5555555555555555ull;  // bit 2j: pair j differs
    return __popc((uint32_t)d) + __popc((uint32_t)(d >> 32));
}

// Output offset of tile t: the exclusive sum over earlier chunks plus the
// offset inside its chunk of `per` consecutive tiles.
__device__ __forceinline__ uint64_t tile_offset(const uint64_t *__restrict__ base, const uint64_t *__restrict__ loff,
                                                uint32_t per, uint32_t t) {
    return __ldg(base + t / per) + __ldg(loff + t);
}

__global__ void __launch_bounds__(kCountThreads, 4)
k_vn_count(const uint64_t *__restrict__ x, uint64_t words, uint64_t lastmask, uint32_t ntiles, uint32_t per,
           uint32_t *__restrict__ cnt, uint64_t *__restrict__ loff, uint64_t *__restrict__ csum,
           uint64_t *__restrict__ base, uint64_t *__restrict__ m_out, uint32_t *__restrict__ done,
           uint32_t *__restrict__ status) {
    __shared__ uint32_t red[2][kCountThreads / 32];
    __shared__ uint64_t wex[kCountThreads / 32];
    __shared__ uint32_t last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // ---- count the chunk of tiles [blockIdx.x * per, + per) in order ----
    // Word order inside a tile does not matter for a count, so the loads are
    // fully coalesced: thread i takes 16-byte chunks i, i + 512, ... of the tile.
    const uint32_t t0 = blockIdx.x * per;
    const uint32_t t1 = min(ntiles, t0 + per);
    uint64_t running = 0;  // thread 0: output bits of the chunk so far
    int par = 0;
    for (uint32_t t = t0; t < t1; ++t, par ^= 1) {
        const uint64_t tb = (uint64_t)t * kVnTileWords;
        uint64_t wv[kCountWpt];
        if (tb + kVnTileWords <= words) {
            const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(x + tb);
#pragma unroll
            for (int i = 0; i < kCountWpt / 2; ++i) {
                const ulonglong2 v = __ldg(p + i * kCountThreads + tid);
                wv[2 * i] = v.x;
                wv[2 * i + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kCountWpt / 2; ++i) {
                const uint64_t w = tb + 2 * ((uint64_t)i * kCountThreads + tid);
                wv[2 * i] = w < words ? __ldg(x + w) : 0ull;
                wv[2 * i + 1] = w + 1 < words ? __ldg(x + w + 1) : 0ull;
            }
        }
        if (tb + kVnTileWords >= words) {  // the tile holding the last word
#pragma unroll
            for (int i = 0; i < kCountWpt / 2; ++i) {
                const uint64_t w = tb + 2 * ((uint64_t)i * kCountThreads + tid);
                if (w == words - 1) wv[2 * i] &= lastmask;
                if (w + 1 == words - 1) wv[2 * i + 1] &= lastmask;
            }
        }
        uint32_t c = 0;
#pragma unroll
        for (int i = 0; i < kCountWpt; ++i) c += pair_count(wv[i]);
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) red[par][warp] = c;  // alternate buffers: one barrier per tile
        __syncthreads();
        if (tid == 0) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kCountThreads / 32; ++w) s += red[par][w];
            cnt[t] = s;
            loff[t] = running;
            running += s;
        }
    }
    if (tid == 0) {
        csum[blockIdx.x] = running;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;

    // ---- the CTA that finished last: exclusive sums over the chunks, and m ----
    __threadfence();
    const uint32_t nch = gridDim.x;
    const uint32_t q = (nch + kCountThreads - 1) / kCountThreads;  // chunks a thread
    uint64_t mine = 0;
    for (uint32_t j = 0; j < q; ++j) {
        const uint32_t i = tid * q + j;
        if (i < nch) mine += __ldcg(csum + i);
    }
    uint64_t inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wex[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint64_t s = lane < kCountThreads / 32 ? wex[lane] : 0;
        uint64_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += u;
        }
        __syncwarp();
        if (lane < kCountThreads / 32) wex[lane] = si - s;  // exclusive offset of each warp
        if (lane == kCountThreads / 32 - 1) {
            *m_out = si;
            if (si == 0) atomicOr(status, kFlagPrecond);
        }
    }
    __syncthreads();
    uint64_t O = wex[warp] + (inc - mine);
    for (uint32_t j = 0; j < q; ++j) {
        const uint32_t i = tid * q + j;
        if (i >= nch) break;
        base[i] = O;
        O += __ldcg(csum + i);
    }
}

// Zero the output words two or more tiles share (a tile's first and last word
// when only partly its own); one thread per tile.
__global__ void k_vn_zero(uint32_t ntiles, uint32_t per, const uint32_t *__restrict__ cnt,
                          const uint64_t *__restrict__ loff, const uint64_t *__restrict__ base,
                          uint64_t *__restrict__ z) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint32_t c = __ldg(cnt + t);
    if (!c) return;
    const uint64_t O = tile_offset(base, loff, per, t);
    const uint64_t f = O >> 6, l = (O + c - 1) >> 6;
    const bool head_part = (O & 63) != 0, tail_part = ((O + c) & 63) != 0;
    if (head_part || (f == l && tail_part)) z[f] = 0;
    if (l != f && tail_part) z[l] = 0;
}

__global__ void __launch_bounds__(kWriteThreads, 2)
k_vn_write(const uint64_t *__restrict__ x, uint64_t words, uint64_t lastmask, uint32_t ntiles, uint32_t per,
           const uint32_t *__restrict__ cnt, const uint64_t *__restrict__ loff, const uint64_t *__restrict__ base,
           uint64_t *__restrict__ z) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *lut = smem;                                                     // 65536 entries
    uint64_t *stage = reinterpret_cast<uint64_t *>(smem + 65536);             // kVnStageWords
    uint16_t *t8 = reinterpret_cast<uint16_t *>(stage + kVnStageWords);      // 256 entries
    uint32_t *wsum = reinterpret_cast<uint32_t *>(t8 + 256);                 // 64 words
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // Table of the pair filter over 4 pairs (8 bits): outputs | count << 8.
    if (tid < 256) {
        uint32_t v = 0, c = 0;
        for (int j = 0; j < 4; ++j) {
            const uint32_t a = (tid >> (2 * j)) & 1, b = (tid >> (2 * j + 1)) & 1;
            if (a != b) v |= a << c++;
        }
        t8[tid] = (uint16_t)(v | (c << 8));
    }
    for (int i = tid; i < kVnStageWords; i += kWriteThreads) stage[i] = 0;
    __syncthreads();
    // Over 8 pairs (16 bits), from two 4-pair lookups; four entries per store.
    for (int q = tid; q < 16384; q += kWriteThreads) {
        uint32_t packed = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t i = 4u * q + e;
            const uint32_t lo = t8[i & 255], hi = t8[i >> 8];
            packed |= ((lo & 255) | ((hi & 255) << (lo >> 8))) << (8 * e);
        }
        reinterpret_cast<uint32_t *>(lut)[q] = packed;
    }
    __syncthreads();

    uint32_t t = blockIdx.x;
    uint64_t cur[kVnWpt];
    if (t < ntiles)
        vn_load<kVnWpt>(x, words, lastmask, (uint64_t)t * kVnTileWords + (uint64_t)tid * kVnWpt, cur);
    while (t < ntiles) {
        const uint64_t O = tile_offset(base, loff, per, t);
        const uint32_t C = __ldg(cnt + t);
        const uint32_t tn = t + gridDim.x;
        const uint32_t s0 = (uint32_t)(O & 63);
        if (C != 0) {
            // ---- compress each word (<= 32 bits, pair order) and count ----
            uint32_t ov[kVnWpt], oc[kVnWpt], total = 0;
#pragma unroll
            for (int i = 0; i < kVnWpt; ++i) {
                const uint64_t w = cur[i];
                const uint64_t d = (w ^ (w >> 1)) & 0x5555555555555555ull;  // bit 2j: pair j differs
                const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
                const uint32_t dl = (uint32_t)d, dh = (uint32_t)(d >> 32);
                const uint32_t c0 = __popc(dl & 0xFFFFu), c01 = __popc(dl), c2 = __popc(dh & 0xFFFFu);
                oc[i] = c01 + __popc(dh);
                ov[i] = (uint32_t)lut[lo & 0xFFFFu] | ((uint32_t)lut[lo >> 16] << c0) |
                        ((uint32_t)lut[hi & 0xFFFFu] << c01) | ((uint32_t)lut[hi >> 16] << (c01 + c2));
                total += oc[i];
            }
            // ---- this thread's offset in the tile's output ----
            uint32_t inc = total;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            if (lane == 31) wsum[warp] = inc;
            __syncthreads();
            if (warp == 0) {
                const uint32_t w0 = lane < kWriteThreads / 32 ? wsum[lane] : 0;
                uint32_t si = w0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, si, o);
                    if (lane >= o) si += u;
                }
                if (lane < kWriteThreads / 32) wsum[32 + lane] = si - w0;
            }
            __syncthreads();

            // ---- pack; staging word i is output word (O >> 6) + i ----
            const uint32_t start = s0 + wsum[32 + warp] + (inc - total);
            uint64_t acc = 0;
            uint32_t pos = start & 63, k = start >> 6;
#pragma unroll
            for (int i = 0; i < kVnWpt; ++i) {
                const uint32_t c = oc[i], v = ov[i];
                if (c == 0) continue;
                acc |= (uint64_t)v << pos;
                if (pos + c >= 64) {  // pos >= 32 here
                    atomicOr(reinterpret_cast<unsigned long long *>(stage + k), (unsigned long long)acc);
                    ++k;
                    acc = (uint64_t)v >> (64 - pos);
                    pos = pos + c - 64;
                } else {
                    pos += c;
                }
            }
            if (pos) atomicOr(reinterpret_cast<unsigned long long *>(stage + k), (unsigned long long)acc);
        }
        // the next tile's words load while this one is written out
        uint64_t nxt[kVnWpt];
        if (tn < ntiles)
            vn_load<kVnWpt>(x, words, lastmask, (uint64_t)tn * kVnTileWords + (uint64_t)tid * kVnWpt, nxt);
        if (C != 0) {
            __syncthreads();
            // ---- write: words owned alone stored, partial words ORed ----
            const uint64_t f = O >> 6;
            const uint32_t nw = (s0 + C + 63) >> 6;  // staging words in use
            const bool tail_part = ((s0 + C) & 63) != 0;
            for (uint32_t i = tid; i < nw; i += kWriteThreads) {
                const uint64_t v = stage[i];
                if ((i == 0 && s0 != 0) || (i == nw - 1 && tail_part))
                    atomicOr(reinterpret_cast<unsigned long long *>(z + f + i), (unsigned long long)v);
                else
                    z[f + i] = v;
            }
            __syncthreads();  // staging reads done
            for (uint32_t i = tid; i < nw; i += kWriteThreads) stage[i] = 0;
        }
#pragma unroll
        for (int i = 0; i < kVnWpt; ++i) cur[i] = nxt[i];
        t = tn;
    }
}

}  // namespace

static uint64_t vn_words(uint64_t n) { return (2 * (n / 2) + 63) / 64; }
static uint32_t vn_tiles(uint64_t n) { return (uint32_t)((vn_words(n) + kVnTileWords - 1) / kVnTileWords); }

static bool vn_args_ok(const void *x, uint64_t n, const void *z, const void *m) {
    if (!x || !z || !m || n < 2 || n >= (1ull << 46)) return false;
    if (reinterpret_cast<uintptr_t>(x) & 15) return false;
    if ((reinterpret_cast<uintptr_t>(z) & 7) || (reinterpret_cast<uintptr_t>(m) & 7)) return false;
    return true;
}

static cm_status vn_enqueue(cm_ctx *ctx, const uint64_t *x, uint64_t n, uint64_t *z, uint64_t *m_out,
                            void *scratch, cudaStream_t st) {
    if (cudaFuncSetAttribute(k_vn_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWriteSmem) !=
        cudaSuccess)
        return CM_EDEVICE;
    const uint64_t words = vn_words(n);
    const uint32_t tiles = vn_tiles(n);
    const uint64_t vb = 2 * (n / 2) - 64 * (words - 1);  // valid bits of the last word, 1..64
    const uint64_t lastmask = vb >= 64 ? ~0ull : ((1ull << vb) - 1);
    const uint32_t cgrid = tiles < (uint32_t)(4 * ctx->nsm) ? tiles : (uint32_t)(4 * ctx->nsm);
    const uint32_t per = (tiles + cgrid - 1) / cgrid;
    const uint32_t nch = (tiles + per - 1) / per;  // chunks with at least one tile
    uint8_t *b = static_cast<uint8_t *>(scratch);
    uint32_t *done = reinterpret_cast<uint32_t *>(b);
    uint64_t *loff = reinterpret_cast<uint64_t *>(b + kVnHeaderBytes);
    uint64_t *csum = loff + tiles;
    uint64_t *base = csum + kMaxChunks;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(base + kMaxChunks);
    if (cudaMemsetAsync(done, 0, sizeof(uint32_t), st) != cudaSuccess) return CM_EDEVICE;
    {
        ProfScope ps(ctx, "k_vn_count", st);
        k_vn_count<<<nch, kCountThreads, 0, st>>>(x, words, lastmask, tiles, per, cnt, loff, csum, base, m_out,
                                                  done, ctx->d_status);
    }
    {
        ProfScope ps(ctx, "k_vn_zero", st);
        k_vn_zero<<<(tiles + 255) / 256, 256, 0, st>>>(tiles, per, cnt, loff, base, z);
    }
    const uint32_t grid = tiles < (uint32_t)(2 * ctx->nsm) ? tiles : (uint32_t)(2 * ctx->nsm);
    {
        ProfScope ps(ctx, "k_vn_write", st);
        k_vn_write<<<grid, kWriteThreads, kWriteSmem, st>>>(x, words, lastmask, tiles, per, cnt, loff, base, z);
    }
    return cudaGetLastError() == cudaSuccess ? CM_OK : CM_EDEVICE;
}

}  // namespace cm

extern "C" uint64_t cm_von_neumann_scratch_bytes(uint64_t n) {
    if (n < 2) return 0;
    return cm::kVnHeaderBytes + 12ull * cm::vn_tiles(n) + 16ull * cm::kMaxChunks;
}

extern "C" cm_status cm_von_neumann(cm_ctx *ctx, const uint64_t *x, uint64_t n, uint64_t *z, uint64_t *m_out,
                                    cm_stream stream) {
    if (!ctx || !cm::vn_args_ok(x, n, z, m_out)) return CM_EINVAL;
    const uint64_t sb = cm_von_neumann_scratch_bytes(n);
    if (sb > ctx->budget) return CM_ENOMEM;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, sb, ctx->pool, st) != cudaSuccess) {
        cudaGetLastError();
        return CM_ENOMEM;
    }
    cm_status s = cm::vn_enqueue(ctx, x, n, z, m_out, scratch, st);
    if (cudaFreeAsync(scratch, st) != cudaSuccess && s == CM_OK) s = CM_EDEVICE;
    return s;
}

extern "C" cm_status cm_von_neumann_host(cm_ctx *ctx, const uint64_t *xh, uint64_t n, uint64_t *zh, uint64_t *m,
                                         cm_stream stream) {
    if (!ctx || !xh || !zh || !m || n < 2 || n >= (1ull << 46)) return CM_EINVAL;
    const uint64_t xw = (n + 63) / 64, zw = (n / 2 + 63) / 64;
    const uint64_t sb = cm_von_neumann_scratch_bytes(n);
    const uint64_t xoff = (sb + 255) & ~255ull;
    const uint64_t zoff = xoff + ((8 * xw + 255) & ~255ull);
    const uint64_t moff = zoff + ((8 * zw + 255) & ~255ull);
    const uint64_t total = moff + 256;
    if (total > ctx->budget) return CM_ENOMEM;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return CM_EDEVICE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *buf = nullptr;
    if (cudaMallocFromPoolAsync(&buf, total, ctx->pool, st) != cudaSuccess) {
        cudaGetLastError();
        return CM_ENOMEM;
    }
    uint8_t *b = static_cast<uint8_t *>(buf);
    uint64_t *xd = reinterpret_cast<uint64_t *>(b + xoff);
    uint64_t *zd = reinterpret_cast<uint64_t *>(b + zoff);
    uint64_t *md = reinterpret_cast<uint64_t *>(b + moff);
    cm_status s = CM_OK;
    uint64_t mh = 0;
    if (cudaMemcpyAsync(xd, xh, 8 * xw, cudaMemcpyHostToDevice, st) != cudaSuccess) s = CM_EDEVICE;
    if (s == CM_OK) s = cm::vn_enqueue(ctx, xd, n, zd, md, b, st);
    if (s == CM_OK && (cudaMemcpyAsync(&mh, md, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess))
        s = CM_EDEVICE;
    if (s == CM_OK && mh > 0 &&
        cudaMemcpyAsync(zh, zd, 8 * ((mh + 63) / 64), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = CM_EDEVICE;
    cudaFreeAsync(buf, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && s == CM_OK) s = CM_EDEVICE;
    *m = s == CM_OK ? mh : 0;
    if (s == CM_OK && mh == 0) s = CM_EPRECOND;
    return s;
}
