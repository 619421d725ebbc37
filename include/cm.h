/*
 * cm.h -- C ABI of the GB300 NTT randomness-extractor library (libcm.so).
 *
 * The library computes the Toeplitz, Circulant and Dodis et al. extractors of
 * Cryptomite (arXiv 2402.09481) on one NVIDIA GB300 GPU.  Each output is a
 * GF(2) matrix-vector product, computed exactly as an integer convolution by a
 * number-theoretic transform (Def. ntt and Thm. convolution of the paper),
 * then reduced mod 2.  The transform runs over one of three prime fields, each
 * large enough that every convolution coefficient (a count of at most the
 * product's length) is exact: q = 5 * 2^25 + 1 with lazy reduction for
 * transforms up to 2^25, the paper's own q = 3 * 2^30 + 1 (Section
 * "Performance") up to 2^30, and Goldilocks p = 2^64 - 2^32 + 1 up to 2^32.
 * The choice changes speed, never a result bit.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Bit strings are arrays of uint64_t words: bit i is bit (i & 63) of word
 * i >> 6 (least significant first).  Bit 0 is the paper's x_0 / y_0.  A string
 * of k bits occupies ceil(k / 64) words.  Input bits past the length are
 * ignored; output bits past m are written as 0.
 *
 * Unless stated otherwise, data pointers are DEVICE pointers on the context's
 * GPU, the caller owns every buffer, and calls are asynchronous and
 * stream-ordered on `stream` (a cudaStream_t; NULL is the legacy default
 * stream).  The library keeps no pointer to caller memory after the stream
 * work of the call completes.  Scratch memory comes from a memory pool owned by
 * the context (stream-ordered allocation on the same stream), so concurrent
 * calls on different streams do not share scratch.
 *
 * Errors: every call returns a cm_status.  Argument errors are detected on the
 * host before anything is enqueued; nothing aborts and no exception crosses
 * the ABI.  The Dodis et al. precondition (x neither all-0 nor all-1) is
 * checked on the device: on violation the output is zero-filled and the
 * context's device status records CM_EPRECOND, read back by
 * cm_device_status().
 */
#ifndef CM_H
#define CM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cm_ctx cm_ctx;
typedef void *cm_stream; /* cudaStream_t */

typedef enum {
    CM_OK = 0,
    CM_EINVAL = 1,     /* invalid argument: length, pointer, size beyond limits */
    CM_EPRECOND = 2,   /* Dodis et al.: x is all-0 or all-1 (device-detected) */
    CM_ENOMEM = 3,     /* scratch allocation failed or HBM budget exceeded */
    CM_EAGAIN = 4,     /* not ready / queue full; retry */
    CM_ETIMEDOUT = 5,  /* a bounded wait ran out */
    CM_EDEVICE = 6,    /* CUDA runtime error */
    CM_ENOTFOUND = 7   /* unknown ticket */
} cm_status;

/* Extractor kinds (used by the batched and serving interfaces). */
typedef enum { CM_TOEPLITZ = 0, CM_CIRCULANT = 1, CM_DODIS = 2 } cm_kind;

/* Device-status bits accumulated by kernels, read by cm_device_status(). */
#define CM_FLAG_PRECOND 0x1u  /* a Dodis et al. call saw a constant x */
#define CM_FLAG_TIMEOUT 0x2u  /* a bounded device wait ran out */

typedef struct {
    uint64_t hbm_budget_bytes; /* cap on scratch held at once; 0 = 80% of free HBM */
    /* log2 of the longest transform one product may use, 8..32; 0 = 32.  A
     * single extraction whose K + m - 1 is longer runs as several products
     * (see cm_toeplitz); lowering it trades transforms for scratch. */
    uint32_t max_transform_lg;
    /* Transform field of the single calls: CM_FIELD_AUTO takes the field of
     * 5 * 2^25 + 1 (lazy reduction) for every product of length <= 2^25, the
     * field of 3 * 2^30 + 1 (the paper's small field, Section "Performance")
     * up to 2^30 and Goldilocks above (the planner may prefer blocks over the
     * smaller fields to one longer transform); CM_FIELD_Q30 skips the field of
     * 5 * 2^25 + 1; CM_FIELD_GOLDILOCKS takes Goldilocks throughout.  Results
     * are identical.  Batches and the server run their work-list instances
     * over 3 * 2^30 + 1 (Goldilocks in a CM_FIELD_GOLDILOCKS context). */
    uint32_t field;
    /* Most input blocks whose transform-domain products are summed before one
     * inverse transform; 0 = as many as keep every count below the field's
     * characteristic.  Later groups XOR their parities in.  Results are
     * identical for every value. */
    uint32_t max_sum_blocks;
    /* CM_PLAN_COST: the planner splits a product whenever that is estimated
     * faster; CM_PLAN_SINGLE: one transform whenever K + m - 1 fits the limit
     * (splits only longer products).  Results are identical. */
    uint32_t plan_mode;
    uint32_t reserved[4];
} cm_options;

#define CM_PLAN_COST 0u
#define CM_PLAN_SINGLE 1u

#define CM_FIELD_AUTO 0u
#define CM_FIELD_GOLDILOCKS 1u
#define CM_FIELD_Q30 2u /* q = 3 * 2^30 + 1 (and Goldilocks above 2^30) */
#define CM_FIELD_Q25 3u /* reported by cm_plan_query only: q = 5 * 2^25 + 1 */

/* Create a context on CUDA device `device`: root tables resident in HBM, a
 * scratch memory pool.  opt may be NULL.  Returns CM_EDEVICE if the device is
 * unusable, CM_EINVAL if out is NULL, opt->max_transform_lg is outside
 * 8..32 (and not 0) or opt->field is not a CM_FIELD_* value. */
cm_status cm_create(cm_ctx **out, int device, const cm_options *opt);

/* Synchronize the device and free everything the context owns. */
void cm_destroy(cm_ctx *ctx);

/* Static string for a status code. */
const char *cm_status_str(int status);

/*
 * Toeplitz extractor, Eq. toep-ext / Eq. toep of the paper:
 *   z = toep(y) x over GF(2), toep(y)[i][j] = y[(i - j) mod (n + m - 1)],
 *   i < m, j < n.
 * x: n bits (ceil(n/64) words).  y: n + m - 1 bits.  z: m bits (ceil(m/64)
 * words, written).  Requires 1 <= n, m <= 2^40 (the input lengths the paper's
 * software accepts, Section "Introduction").  CM_EINVAL otherwise.
 *
 * Lengths (all three extractors): the middle product has K + m - 1 terms
 * (K = n, n + 1, n for Toeplitz, Circulant, Dodis et al.).  It runs as one
 * transform of the smallest power of two >= K + m - 1, or split: over input
 * blocks (GF(2)-linearity: the output is the parity of the sum over blocks;
 * the blocks of one output window share one transform length, their
 * transform-domain products are added and one inverse transform serves the
 * window) and over output windows; up to 256 leading terms (t < T) may be
 * left out of the transforms and XORed in by a dense GF(2) kernel, so that
 * the rest fits a transform half as long.  A planner picks the form with the lowest
 * estimated GPU time among those whose transforms fit 2^32 (or the context's
 * max_transform_lg) and whose scratch fits the HBM budget: a split is taken
 * when it is faster, e.g. 32-bit-field blocks of 2^30 instead of one
 * Goldilocks transform of 2^31, and whenever one transform cannot hold the
 * product.  Products run in turn with the scratch of one (cm_plan_query).
 */
cm_status cm_toeplitz(cm_ctx *ctx, const uint64_t *x, uint64_t n, const uint64_t *y, uint64_t m,
                      uint64_t *z, cm_stream stream);

/*
 * Circulant extractor, Def. ext-circ with Eq. circ-matrix:
 *   x' = [x, 0],  z = (circ(x') y)_{0..m-1},  circ(c)[i][j] = c[(j - i) mod P].
 * n is the INPUT length n_1 = P - 1 (the paper's Def. ext-circ calls the prime
 * n); P = n + 1 must be prime with 2 as a primitive root.
 * x: n bits.  y: n + 1 bits.  z: m bits, 1 <= m <= n <= 2^40 (blocked
 * beyond one transform as for cm_toeplitz).  CM_EINVAL otherwise.  x = 0 is
 * allowed (output 0).
 */
cm_status cm_circulant(cm_ctx *ctx, const uint64_t *x, uint64_t n, const uint64_t *y, uint64_t m,
                       uint64_t *z, cm_stream stream);

/*
 * Dodis et al. two-source extractor, matrix form of the paper's Section
 * "Dodis (and Circulant) implementation":
 *   z_i = sum_j x[(j - i) mod n] y_j (mod 2),  i < m
 * (equivalently the first m entries of R(x) * y, R(x) = x_0, x_{n-1}, ..., x_1).
 * x, y: n bits each; n prime with 2 as a primitive root; 1 <= m <= n <= 2^40
 * (blocked beyond one transform as for cm_toeplitz).  CM_EINVAL otherwise.  If x is all-0 or all-1 the call
 * still returns CM_OK (the check runs on the device), z is zero-filled and
 * cm_device_status() reports CM_EPRECOND.
 */
cm_status cm_dodis(cm_ctx *ctx, const uint64_t *x, const uint64_t *y, uint64_t n, uint64_t m,
                   uint64_t *z, cm_stream stream);

/*
 * Composed two-source extractor, Section "Composing extractors": a strong
 * seeded extractor appended to a strong two-source extractor, the two-source
 * output serving as the seed and the two-source weak seed as the input.
 *   stage 1: s = Ext_kind1(x, y), m1 bits (x: n1 bits; y: the seed length of
 *            kind1 for (n1, m1): n1 + m1 - 1, n1 + 1 or n1 bits);
 *   stage 2: t = Ext_kind2(input = bits 0 .. n2-1 of y, seed = the first bits
 *            of s), m2 bits; the seed takes n2 + m2 - 1 (Toeplitz), n2 + 1
 *            (Circulant) or n2 (Dodis et al.) bits of s.
 * z: m1 + m2 bits (ceil((m1 + m2)/64) words, written): s in bits 0 .. m1-1,
 * t in bits m1 .. m1+m2-1.  The paper names neither the seeded extractor nor
 * its lengths; the caller picks them (kind2 a cm_kind, n2 <= y's length,
 * stage 2's seed length <= m1), each stage with the argument rules of its
 * single call.  CM_EINVAL otherwise, before any work.  Device pointers,
 * stream-ordered; scratch: ceil(m2/64) words from the context pool besides
 * the stages' own.  A constant Dodis et al. input in either stage is reported
 * by cm_device_status (CM_EPRECOND) as for cm_dodis.
 */
cm_status cm_compose(cm_ctx *ctx, int kind1, const uint64_t *x, uint64_t n1, const uint64_t *y, uint64_t m1,
                     int kind2, uint64_t n2, uint64_t m2, uint64_t *z, cm_stream stream);

/* Synchronize `stream`, then read and clear the context's device status bits.
 * *flags (may be NULL) receives the CM_FLAG_* bits.  Returns CM_EPRECOND if
 * CM_FLAG_PRECOND was set, CM_ETIMEDOUT if CM_FLAG_TIMEOUT was set, CM_EDEVICE
 * on a CUDA error, else CM_OK. */
cm_status cm_device_status(cm_ctx *ctx, cm_stream stream, uint32_t *flags);

/*
 * End-to-end call on HOST buffers: copies x and y host->device, runs the
 * extraction of `kind` (cm_kind) with the same argument rules as cm_toeplitz /
 * cm_circulant / cm_dodis, copies z device->host, and synchronizes `stream`
 * before returning.  x_host, y_host, z_host are host pointers (pinned memory
 * gives full copy bandwidth; pageable works).  Word counts: x ceil(n/64);
 * y ceil((n+m-1)/64) for Toeplitz, ceil((n+1)/64) for Circulant, ceil(n/64)
 * for Dodis et al.; z ceil(m/64).  Device copies come from the context pool.
 * Returns CM_EPRECOND (z zero-filled) for a constant Dodis et al. x.
 */
cm_status cm_extract_host(cm_ctx *ctx, int kind, const uint64_t *x_host, uint64_t n,
                          const uint64_t *y_host, uint64_t m, uint64_t *z_host, cm_stream stream);

/*
 * Allocation-free Toeplitz extraction (the paper has no counterpart; this is a
 * deployment interface).  Same arguments, bit layout and result as
 * cm_toeplitz, but no context and no device allocation of any kind: it calls
 * neither cudaMalloc nor cudaFree nor any allocating library routine.  It is
 * for callers that cannot allocate device memory -- for example a host process
 * whose device memory is fully reserved by another allocator, or a
 * latency-critical loop that must never enter the driver's allocator -- and
 * that therefore cannot create a cm_ctx (cm_create allocates its tables and
 * memory pool).
 *
 * Limit: n + m - 1 <= 2^20 (CM_NOALLOC_MAX_LEN); larger sizes return
 * CM_EINVAL before any work is enqueued.  The scratch (two transform buffers of
 * 2^20 words and 2^20 parity bytes) and the root tables are fixed-size
 * __device__ arrays inside libcm.so: every GPU that loads the library holds
 * them, about 19 MB, until the process exits.
 *
 * The first call on a device (the device current on the calling thread) sets
 * that device up: it looks up the arrays' device addresses and fills the root
 * tables with a kernel on the legacy default stream, then synchronizes.  Make
 * that first call before any stream capture.  Later calls only enqueue work
 * on `stream`.  A device reset gives the device a new CUDA context, in which
 * the arrays start over: the first call after it sets the device up again
 * (the set-up remembers the context it ran in).
 *
 * All calls on a device share the one scratch array, which keeps the last
 * call's contents (nothing in it needs to start at zero: every word is written
 * before it is read).  Calls whose work overlaps on the GPU -- on different
 * streams, or from different threads without ordering -- race on the scratch
 * and give wrong results; order them on one stream or with events.
 */
#define CM_NOALLOC_MAX_LEN (1ull << 20)
cm_status cm_toeplitz_noalloc(const uint64_t *x, uint64_t n, const uint64_t *y, uint64_t m,
                              uint64_t *z, cm_stream stream);

/* ----- batched extraction ------------------------------------------------ */

/* One extraction of a batch.  Same argument rules as the single-call entry
 * points of that kind; x, y, z are device pointers owned by the caller and must
 * stay valid (and unchanged in place) for as long as the batch is launched. */
typedef struct {
    int32_t kind;       /* cm_kind */
    uint32_t reserved;  /* 0 */
    uint64_t n, m;      /* input length n_1 and output length, as for the single calls */
    const uint64_t *x;
    const uint64_t *y;
    uint64_t *z;
} cm_desc;

#define CM_BATCH_AUTOTUNE 0x1u /* time the candidate pass tiles on this batch, keep the fastest */
#define CM_BATCH_NO_GRAPH 0x2u /* do not capture a CUDA graph */
/* Failure-path test: the first instance with L > 2^13 waits for one more
 * forward tile than the work list holds, so its middle rows' bounded waits run
 * out: the launch ends early with CM_FLAG_TIMEOUT set in the device status
 * (cm_device_status then returns CM_ETIMEDOUT) and the outputs are undefined. */
#define CM_BATCH_TEST_STALL 0x4u

typedef struct cm_batch cm_batch;

typedef struct {
    uint32_t instances, work_items, solo_instances, tile_lg, grid, graph;
    uint64_t scratch_bytes, kernel_launches, output_bits, transform_elements;
} cm_batch_stats;

/*
 * Plan a batch of `count` extractions of any mix of kinds (the paper has no
 * batched form; each instance computes exactly what its single call computes).
 * All instances with transform length L <= 2^25 run in ONE persistent kernel
 * launch that walks a work list: an instance with L <= 2^13 is one item, a
 * larger one is split into forward column-pass tiles, fused middle rows,
 * inverse tiles with parity, and pack chunks, each item starting once the
 * items it depends on are done (bounded waits; CM_FLAG_TIMEOUT if one runs
 * out).  Instances with L > 2^25 run through the single-call kernels after it.
 * Scratch for every instance is allocated here (cudaMalloc, held until
 * cm_batch_destroy); CM_ENOMEM if it exceeds the context budget.  With
 * CM_BATCH_AUTOTUNE the candidate column-pass tiles (2^14 and 2^13 elements)
 * are timed on the batch itself and the faster is kept.  Unless
 * CM_BATCH_NO_GRAPH, the launch sequence is captured once into a CUDA graph.
 * CM_EINVAL if any descriptor is invalid (nothing is allocated).
 */
cm_status cm_batch_create(cm_ctx *ctx, const cm_desc *descs, uint32_t count, uint32_t flags,
                          cm_batch **out);

/* Enqueue one execution of the batch on `stream` (a graph launch when one was
 * captured and tracing is off).  Asynchronous; the outputs are complete when
 * the stream reaches this point.  Executions of one batch must not overlap
 * (they share its scratch and work list). */
cm_status cm_batch_launch(cm_batch *b, cm_stream stream);

/* Synchronize the device and free the batch's scratch, work list and graph. */
void cm_batch_destroy(cm_batch *b);

/* Plan statistics: work items, pass tile chosen, scratch bytes, kernel launches
 * per execution, total output bits and transform elements. */
cm_status cm_batch_info(const cm_batch *b, cm_batch_stats *stats);

/* One-shot batch: plan (no autotuning, no graph), run on `stream`, synchronize,
 * free.  Returns after the outputs are written. */
cm_status cm_batch_extract(cm_ctx *ctx, const cm_desc *descs, uint32_t count, cm_stream stream);

/* cm_batch_extract for batches whose every descriptor is Toeplitz (CM_EINVAL
 * otherwise). */
cm_status cm_batch_toeplitz(cm_ctx *ctx, const cm_desc *descs, uint32_t count, cm_stream stream);

/* ----- many inputs under one shared Toeplitz seed ------------------------- */

#define CM_ENGINE_AUTO 0 /* fastest engine, timed on the first call of an (n, m) */
#define CM_ENGINE_IMMA 1 /* INT8 tensor cores (mma.sync s8 x s8 -> s32), mod-2 epilogue */
#define CM_ENGINE_GF2 2  /* CUDA cores: XOR of AND over packed words, parity epilogue */
#define CM_ENGINE_BMMA 3 /* binary tensor cores (mma.sync b1 x b1 -> s32, AND-POPC), mod-2 epilogue */

/*
 * Z_c = toep(y) X_c over GF(2) for c < count: the Toeplitz extractor of Eq.
 * toep-ext / Eq. toep applied to `count` inputs under ONE seed y (n + m - 1
 * bits), computed as a dense blocked product of the m x n Toeplitz matrix
 * (expanded once from y, packed bits, zero-padded to whole tiles) with the
 * inputs.  X holds the inputs back to back, input c at word c*ceil(n/64)
 * (n bits each); Z receives output c at word c*ceil(m/64) (m bits each, tail
 * bits 0).  Device pointers, stream-ordered.  Every engine gives the same
 * bits as cm_toeplitz on each input.  The paper has no batched form; this is
 * its seeded extractor with the seed reused, which Section "Useful theorems
 * and results" permits for strong extractors.
 * Requires 1 <= n, m <= 2^24, n * m <= 2^34, 1 <= count <= 2^31, engine one
 * of CM_ENGINE_*; CM_EINVAL otherwise.  Scratch: the expanded matrix,
 * ceil(m/64)*64 * ceil(n/1024)*1024 / 8 bytes from the context pool.
 */
cm_status cm_batch_toeplitz_shared_seed(cm_ctx *ctx, const uint64_t *y, uint64_t n, uint64_t m,
                                        const uint64_t *X, uint64_t count, uint64_t *Z, int engine,
                                        cm_stream stream);

/* Engine CM_ENGINE_AUTO settled on for (n, m) after its first call, or
 * CM_ENGINE_AUTO if none yet (process-wide). */
int cm_shared_seed_engine(uint64_t n, uint64_t m);

/* ----- serving: continuous batching ------------------------------------- */

/* One extraction request: same argument rules as the single calls; device
 * pointers that must stay valid until the request is polled complete. */
#define CM_REQ_SEED_CACHE 0x1u /* y is immutable under seed_id: keep its transform resident */

typedef struct {
    int32_t kind;     /* cm_kind */
    uint32_t flags;   /* CM_REQ_* */
    uint64_t n, m;
    const uint64_t *x;
    const uint64_t *y;
    uint64_t *z;
    uint64_t seed_id; /* with CM_REQ_SEED_CACHE: names the seed y (the caller promises that
                         every request with this id has the same y contents) */
    uint64_t user;    /* free for the caller */
} cm_request;

typedef struct {
    int32_t status;  /* CM_OK, CM_EPRECOND (Dodis et al. constant x, z zeroed), CM_ETIMEDOUT, ... */
    uint32_t reserved;
    uint64_t t_submit_ns, t_admit_ns, t_done_ns;  /* steady clock: submitted, sent to the GPU, seen done */
    uint64_t wave;   /* the launch wave that carried it */
} cm_result;

typedef struct {
    uint64_t hbm_budget_bytes; /* scratch of requests on the device at once; 0 = half the context budget */
    uint32_t slots;            /* CUDA streams of concurrent waves, two wave slots each; 0 = 3 */
    uint32_t max_queue;        /* pending requests before cm_submit says CM_EAGAIN; 0 = 2^20 */
    uint32_t max_wave;         /* requests per wave; 0 = 512 */
    uint32_t express_slots;    /* extra high-priority slots for work-list-sized requests; 0 = 1,
                                  CM_SERVER_NO_EXPRESS = none */
    uint64_t seed_cache_bytes; /* resident seed transforms (within the budget); 0 = a quarter of it */
    uint32_t reserved[2];
} cm_server_options;
#define CM_SERVER_NO_EXPRESS 0xFFFFFFFFu

typedef struct {
    uint64_t submitted, completed, rejected, waves;
    uint64_t inflight_bytes, max_inflight_bytes, budget_bytes;
    uint64_t seed_cache_hits, seed_cache_misses, seed_cache_bytes, seed_cache_entries;
    uint32_t queued, busy_slots, slots, reserved; /* slots: wave slots, two per stream plus the express ones */
} cm_server_stats;

/*
 * Start the request server of a context (one per context): a worker thread
 * that admits pending requests in queue order into waves whenever a slot is
 * free, as long as their scratch fits in what the HBM budget leaves (a request
 * that does not fit yet is passed over by at most 16 waves, after which
 * nothing behind it starts until it fits).  A wave runs its requests with
 * transforms up to 2^21 as one work-list kernel (the cm_batch_create
 * machinery) and longer ones through the single-call planner, on the slot's
 * stream; a wave of one request runs the single-call kernels.  Waves on
 * different streams overlap on the device; each stream has two slots, so the
 * next wave is enqueued behind the running one.  Express slots (high stream
 * priority) take only requests up to 2^21, so that short requests are not
 * held behind long ones.  Requests flagged CM_REQ_SEED_CACHE (transform
 * length 2^14 .. 2^21) keep the forward transform of their seed operand
 * resident, keyed by (seed_id, kind, n, m); a later request with the same key
 * skips that transform (reuse of the seed is what the paper's strong
 * extractors allow).  Least recently used entries are dropped past
 * seed_cache_bytes.  The paper has no serving layer; each request computes
 * exactly its single call.
 */
cm_status cm_server_start(cm_ctx *ctx, const cm_server_options *opt);

/* Drain the queue, wait for the device, stop the worker (cm_destroy also does). */
cm_status cm_server_stop(cm_ctx *ctx);

/* Queue one request; *ticket identifies it.  CM_EINVAL for invalid arguments
 * or no server, CM_ENOMEM if its scratch alone exceeds the budget, CM_EAGAIN
 * if the queue is full.  Thread-safe. */
cm_status cm_submit(cm_ctx *ctx, const cm_request *req, uint64_t *ticket);

/* Wait up to timeout_ns for the request; CM_OK with *res filled once it is
 * done (the ticket is then released), CM_EAGAIN if it is not done yet,
 * CM_ENOTFOUND for an unknown or already collected ticket.  Thread-safe. */
cm_status cm_poll(cm_ctx *ctx, uint64_t ticket, cm_result *res, uint64_t timeout_ns);

/* Counters of the server (queue depth, waves, bytes in flight and their peak). */
cm_status cm_server_get_stats(cm_ctx *ctx, cm_server_stats *stats);

/* ----- tracing ----------------------------------------------------------- */

typedef struct {
    char name[40];     /* kernel name */
    uint64_t launches; /* launches since the last reset */
    double total_ms;   /* summed device time between the events around them */
} cm_profile_entry;

/* Turn per-kernel tracing on (1) or off (0).  When on, every kernel the
 * context enqueues is bracketed by two CUDA events recorded on the launching
 * stream. */
cm_status cm_profile_enable(cm_ctx *ctx, int on);

/* Wait for the traced launches, then copy up to `cap` per-kernel summaries
 * into out (sorted by name) and the number of distinct kernels into *count.
 * reset != 0 clears the summaries afterwards. */
cm_status cm_profile_read(cm_ctx *ctx, cm_profile_entry *out, uint32_t cap, uint32_t *count,
                          int reset);

/* ----- diagnostics ------------------------------------------------------ */

/* Field self-test on `device`: for `count` inputs (fixed edge values, then
 * SplitMix64 samples from `seed`) compares the device's Goldilocks add, sub,
 * multiply and multiply-by-2^s (s = 0..96), written as 32-bit carry chains,
 * with the plain 64-bit C forms of the same functions, and the 32-bit field's
 * add, subtract, Montgomery product and sub-transform twiddles (q = 3 * 2^30
 * + 1) and the lazily reduced field's (q = 5 * 2^25 + 1) reduction, canonical
 * form, add, subtract, Montgomery and Shoup products, values and output ranges
 * included, with plain 64-bit modular arithmetic; *mismatches receives the
 * number of disagreements (0 when correct).  Allocates and frees 8 bytes. */
cm_status cm_field_selftest(int device, uint64_t count, uint64_t seed, uint64_t *mismatches);

/* Modular-multiply rate of `device` for `field` (CM_FIELD_GOLDILOCKS: the
 * 64-bit product and reduction of the transforms; CM_FIELD_Q30: the 32-bit
 * Montgomery product; CM_FIELD_Q25: the Shoup product by a constant root with
 * its precomputed quotient, the product the transforms of the field of
 * 5 * 2^25 + 1 use for their roots), measured by a kernel of independent
 * register chains of
 * products on every SM (8 chains a thread, 4 CTAs of 256 threads per SM) and
 * timed with CUDA events: *per_second receives products per second.  The
 * integer-pipe bound of a path is its number of general multiplies divided by
 * this rate.  Allocates and frees 8 bytes; CM_EINVAL for another field. */
cm_status cm_modmul_rate(int device, uint32_t field, double *per_second);

/* ----- host helpers (no GPU work) --------------------------------------- */

/* 1 if P is prime and 2 is a primitive root modulo P (the set N_A of the
 * paper's footnote to Def. ext-circ), else 0.  Deterministic for P < 2^64. */
int cm_is_na_prime(uint64_t P);
/* Smallest member of N_A >= n (0 if none below 2^63). */
uint64_t cm_next_na_prime(uint64_t n);
/* Largest member of N_A <= n (0 if n < 3). */
uint64_t cm_prev_na_prime(uint64_t n);

/* How a single call of (kind, n, m) runs under the given options (the
 * planner of cm_toeplitz). */
typedef struct {
    uint64_t transform_length; /* the longest product's transform length L */
    uint64_t products;         /* middle products: input blocks x output windows */
    uint64_t windows;          /* output windows (one inverse transform each) */
    uint64_t scratch_bytes;    /* pool bytes the call holds */
    uint32_t launches;         /* kernel launches the call enqueues */
    uint32_t field;            /* the widest field of any product: CM_FIELD_GOLDILOCKS,
                                  else CM_FIELD_Q30, else CM_FIELD_Q25 */
    double est_ms;             /* the planner's GPU-time estimate (GB300) */
    uint64_t tail_terms;       /* terms t < tail_terms left out of the transforms
                                  and XORed in densely (0: none) */
    uint64_t reserved[3];
} cm_plan_info;

/* Fill *out with the plan of (kind, n, m) under opt (NULL: defaults, no
 * budget).  CM_EINVAL if the arguments or options are invalid, or the product
 * needs more than 65536 middle products. */
cm_status cm_plan_query(int kind, uint64_t n, uint64_t m, const cm_options *opt, cm_plan_info *out);

/* One middle product of a call's plan (cm_plan_products).  Its operands are
 * bit maps over x (a) and y (b): the value at transform position k in [0, L)
 * is 0 for k >= len, else the source bit at
 *   mode 0: k;   mode 1: (k + off) mod srclen;
 *   mode 2: off - k, or 0 when off - k is outside [0, srclen).
 * With c the cyclic convolution of length L of the two maps, output
 * zword * 64 + i (i < m) of the call is the parity of the sum of c[K - 1 + i]
 * over the product's sum group (sum 1 .. 3 in order, or the product alone,
 * sum 0), XORed over the window's groups.  A last entry with sum 4 (L = 0)
 * is the dense tail: every output i < m is XORed with the parity of
 * sum_{t < tail_terms} a(K - 1 - t) b(t + i) over its maps (the whole
 * product's). */
typedef struct {
    uint64_t K, m, L, zword;
    uint64_t a_len, a_srclen, a_off;
    uint64_t b_len, b_srclen, b_off;
    uint32_t a_mode, b_mode;
    uint32_t field;      /* CM_FIELD_GOLDILOCKS, CM_FIELD_Q30 or CM_FIELD_Q25 */
    int32_t sum;         /* 0 alone, 1 first of a sum group, 2 inner, 3 last, 4 tail */
    uint32_t xor_into;   /* this product's parities are XORed into z */
    uint32_t tail_terms; /* sum 4: the number of tail terms */
} cm_product_desc;

/* Write up to cap product descriptors of the plan of (kind, n, m) under opt
 * to out (may be NULL when cap is 0) and their number to *count.  CM_EINVAL
 * as cm_plan_query. */
cm_status cm_plan_products(int kind, uint64_t n, uint64_t m, const cm_options *opt, cm_product_desc *out,
                           uint64_t cap, uint64_t *count);

/*
 * Planner calibration on this context's GPU (the paper has no counterpart;
 * the planner's cost model is this library's).  Times one Toeplitz extraction
 * per transform length and field (K = L/2 + 1, m = L/4; one warm-up, the
 * median of three, L2 flushed before each): 5 * 2^25 + 1 over 2^9 .. 2^25
 * (2^14 .. 2^17 also as one cluster launch), 3 * 2^30 + 1 and Goldilocks from
 * 2^14, each up to max_lg (0: 2^30) and within the context's HBM budget; for
 * two-pass lengths it also picks the first column pass's length among the
 * default split and its two neighbours.  The figures replace the built-in
 * ones in this context's planner (single calls, batches, the server; not
 * cm_plan_query, which has no context).  cache_path (may be NULL): a text
 * file keyed by the device's name and SM count; when it exists and matches,
 * its figures are loaded instead of measured (unless flags has
 * CM_TUNE_FORCE), otherwise the new figures are written to it.  Runs
 * synchronously (seconds) and must not overlap other calls on the context.
 * CM_EINVAL for bad arguments or an unwritable cache file (the figures are in
 * force regardless), CM_ENOMEM, CM_EDEVICE.
 */
#define CM_TUNE_FORCE 0x1u
cm_status cm_calibrate(cm_ctx *ctx, const char *cache_path, uint32_t flags, uint32_t max_lg);

/* The calibrated figures of a context for field (CM_FIELD_GOLDILOCKS,
 * CM_FIELD_Q30, CM_FIELD_Q25) and transform length 2^lg: *ms the
 * column-pass form's time, *cluster_ms the cluster form's (5 * 2^25 + 1,
 * 2^14 .. 2^17), *split the first pass's log2 R of a two-pass plan; 0 where
 * none was taken (any pointer may be NULL).  CM_EINVAL for bad arguments. */
cm_status cm_tune_query(const cm_ctx *ctx, uint32_t field, uint32_t lg, double *ms, double *cluster_ms,
                        int32_t *split);

/* Transform length of the longest product of (kind, n, m) with default
 * options (cm_plan_query); 0 if the arguments are invalid for that kind. */
uint64_t cm_ntt_length(int kind, uint64_t n, uint64_t m);

/* Bytes of scratch one call of (kind, n, m) takes from the pool (default
 * options). */
uint64_t cm_scratch_bytes(int kind, uint64_t n, uint64_t m);

/* Number of kernel launches one call of (kind, n, m) enqueues (default
 * options). */
uint32_t cm_launch_count(int kind, uint64_t n, uint64_t m);

/* Number of middle products a call of (kind, n, m) runs when one transform
 * may be at most 2^max_transform_lg long (0 = 32), other options default; 0 if
 * invalid (including a max_transform_lg outside 8..32 or more than 65536
 * products). */
uint64_t cm_block_count(int kind, uint64_t n, uint64_t m, uint32_t max_transform_lg);

#ifdef __cplusplus
}
#endif

#endif /* CM_H */
