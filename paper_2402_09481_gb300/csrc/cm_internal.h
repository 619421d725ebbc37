// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "cm.h"
#include "ntt_device.cuh"

namespace cm {

constexpr uint32_t kFlagPrecond = CM_FLAG_PRECOND;
constexpr uint32_t kFlagTimeout = CM_FLAG_TIMEOUT;
constexpr size_t kTableWords = 8192 + 4 * 65536;  // resident root tables

// The unique id of the calling thread's current CUDA context (0 if there is
// none or the driver cannot tell): it changes when a device reset replaces the
// device's primary context, which drops every per-context setting.
uint64_t current_ctx_id();

// Raise KERN's dynamic shared-memory limit to `bytes` once per CUDA context
// instead of on every launch (the runtime call costs host time that a short
// extraction would wait for).  A new context (after a device reset) sets it
// again.
template <auto KERN>
inline cudaError_t smem_attr_once(int bytes) {
    static std::atomic<uint64_t> done_ctx{0};
    const uint64_t id = current_ctx_id();
    if (id && done_ctx.load(std::memory_order_acquire) == id) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && id) done_ctx.store(id, std::memory_order_release);
    return e;
}

// Transform fields (see ntt_device.cuh).
constexpr int kFieldGL = 0;   // Goldilocks, 64-bit elements, L <= 2^32
constexpr int kFieldF30 = 1;  // 3 * 2^30 + 1, 32-bit elements, L <= 2^30
constexpr int kFieldF25 = 2;  // 5 * 2^25 + 1, 32-bit elements, L <= 2^25, lazy reduction
constexpr int kF30MaxLg = 30;
constexpr int kF25MaxLg = 25;
constexpr size_t kTable30Words = 8192 + 4 * 32768 + 4096;  // resident F30 root tables + bit DFT table
// F25 root tables + bit DFT table + per-step tables of every on-chip length
constexpr size_t kTable25Words = 8192 + 2 * 8192 + 2 * 4096 + 4096 + 2 * 16384;

// Arguments of the single-CTA extraction (L <= 2^13).
struct Launch {
    BitMap amap, bmap;
    uint64_t lo, m, linv;  // linv in the field's product form
    uint64_t *z;
    const uint32_t *pre;
    uint32_t *status;
    int field;
    RootTables rt;
    RootTables30 rt30;
    RootTables25 rt25;
    cudaStream_t stream;
};

// Arguments of one column pass.  data: L elements of the field's word size;
// a forward pass may also take the second operand (data2, map2) in the same
// launch (data2 null: one operand).
struct PassArgs {
    void *data;
    BitMap map;
    void *data2;
    BitMap map2;
    int lgN, lgS;
    uint8_t *par;
    uint64_t lo, m;
    int field;
    RootTables rt;
    RootTables30 rt30;
    RootTables25 rt25;
    uint64_t L;
    bool inv, bits_in, parity_out;
};

cudaError_t launch_small(const Launch &q, int lg);
// Whole F25 extraction for 2^14 <= L <= 2^17 on one cluster of L / 2^13 CTAs
// (cm_cluster25.cu).  cluster25_prepare sets the kernel's attributes in the
// current CUDA context and reports whether one such cluster fits the device.
constexpr int kClusterMinLg = 14, kClusterMaxLg = 17;
cudaError_t cluster25_prepare(int lg, bool *fits);
cudaError_t launch_cluster25(const Launch &q, int lg);
cudaError_t launch_pass(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_fwd(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_inv(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_fwd30(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_inv30(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_fwd25(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_inv25(const PassArgs &a, int logr, cudaStream_t st);
// F25 passes: the fused column-pass kernels (cm_pass25.cu) for the single pass
// of a transform of 2^22 .. 2^25, else the generic k_pass.
cudaError_t launch_pass25(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_middle25(void *A, const void *B, void *C, int mode, uint64_t L, uint64_t linv,
                            const RootTables25 &rt, int nsm, cudaStream_t st);
// A, B: L elements of the field's word size.  C null: the product's
// row-transformed result goes to A.  Otherwise mode (MidSum) sums the scaled
// transform-domain products of a sum group in C (L elements): kMidFirst
// stores, kMidInner adds, kMidLast adds and writes the inverse row transform
// of the sum to A.
cudaError_t launch_middle(int field, void *A, const void *B, void *C, int mode, uint64_t L, uint64_t linv,
                          const RootTables &rt, const RootTables30 &rt30, const RootTables25 &rt25, int nsm,
                          cudaStream_t st);
cudaError_t launch_pack(const uint8_t *par, uint64_t m, uint64_t *z, const uint32_t *pre,
                        uint32_t *status, int nsm, cudaStream_t st);
cudaError_t launch_allsame(const uint64_t *x, uint64_t n, uint32_t *flags, int nsm, cudaStream_t st);
// z_i ^= sum_{t<T} amap(K-1-t) bmap(t+i) (mod 2), i < m, 1 <= T <= min(kTailMax, K);
// nothing when the Dodis et al. flags at pre (if any) report a constant x.
constexpr int kTailMax = 256;
cudaError_t launch_tail(const BitMap &amap, const BitMap &bmap, uint64_t K, uint32_t T, uint64_t m, uint64_t *z,
                        const uint32_t *pre, int nsm, cudaStream_t st);
// The dense tail of a one-window extraction, folded into the window's pack.
struct TailArgs {
    BitMap amap, bmap;
    uint64_t K;
    uint32_t T;
};
// launch_pack and launch_tail in one kernel: z = pack(par) ^ tail, words
// past m written 0, z zero (and the status flag set) for a constant Dodis et
// al. x.
cudaError_t launch_pack_tail(const uint8_t *par, uint64_t m, uint64_t *z, const uint32_t *pre, uint32_t *status,
                             const TailArgs &t, int nsm, cudaStream_t st);

// The plan of one extraction: the middle-product form of the extractor and the
// pass split of its transform.
struct Plan {
    int kind;
    uint64_t n, m;
    uint64_t K;      // length of a
    uint64_t L;      // transform length, power of two >= K + m - 1
    int lg;          // log2 L
    int amode, bmode;
    uint64_t alen, asrclen, aoff;
    uint64_t blen, bsrclen, boff;
    int npass;       // column passes before the on-chip block (0, 1 or 2)
    int pass_lg[2];  // log2 R_j, slowest dimension first
    uint64_t lo;     // window start K - 1
    uint64_t scratch_bytes;
    uint32_t launches;
    int field;       // kFieldGL, kFieldF30 or kFieldF25
    bool summed;     // one of several products summed before one inverse transform
    bool cluster;    // one launch on a thread-block cluster (F25, 2^14 .. 2^17, alone)
};

// Which fields a plan may take (cm_options.field):
//   kFieldsAll -- F25 for transforms of length <= 2^25, F30 up to 2^30,
//                 Goldilocks above;
//   kFieldsQ30 -- F30 up to 2^30, Goldilocks above;
//   kFieldsGL  -- Goldilocks throughout.
constexpr int kFieldsAll = 0;
constexpr int kFieldsQ30 = 1;
constexpr int kFieldsGL = 2;
// The field of a transform of length 2^lg under a field set.
inline int field_for(int fields, int lg) {
    if (fields == kFieldsAll && lg <= kF25MaxLg) return kFieldF25;
    if (fields != kFieldsGL && lg <= kF30MaxLg) return kFieldF30;
    return kFieldGL;
}

// Validate (kind, n, m) and fill the plan; false if invalid or if K + m - 1
// exceeds 2^32 (one transform).  fields: a field set (kFields*).
struct Tuning;  // planner figures taken on the device (below)
bool make_plan(int kind, uint64_t n, uint64_t m, Plan *out, int fields = kFieldsGL, const Tuning *tune = nullptr);
// (kind, n, m) satisfies the argument rules of the single calls.
bool valid_args(int kind, uint64_t n, uint64_t m);

// Longest bit string a blocked extraction takes (the paper's 2^40).
constexpr uint64_t kMaxBits = 1ull << 40;
constexpr uint64_t kMaxBlocks = 1u << 16;

// How a block's product joins the others of its output window.
enum SumMode : int {
    kSumNone = 0,   // a product on its own: inverse transform, parity, pack
    kSumFirst = 1,  // forward passes, middle: stores the scaled product to C
    kSumInner = 2,  // forward passes, middle: adds it into C
    kSumLast = 3,   // adds it into C, inverse row and column passes of the sum, parity, pack
    kSumTail = 4,   // not a transform: the dense tail (p: the whole product's maps)
};

// One product of a blocked extraction: plan p (a middle product over an input
// block and an output window) for the output words from zword on.  Input
// blocks of one window share the transform length and the window position, so
// their pointwise products are summed in the transform domain (in the middle
// kernel, before the inverse row transform) and one inverse transform serves
// the sum (the counts add; a sum group holds as many blocks as keep the total
// below the field's characteristic).  Packing blocks of later groups, and of windows of one-CTA
// plans (transform length <= 2^13, never summed), XOR their parities into z.
// A plan may also leave its first `tail` terms (t < tail <= kTailMax) out of
// the transforms: a last pseudo-block (kSumTail) XORs their dense GF(2)
// product into every output, so that the rest fits a shorter transform.
struct Block {
    Plan p;
    uint64_t zword;
    int sum;        // SumMode
    bool xor_into;  // this block packs to a temporary and XORs it into z
    uint32_t tail;  // kSumTail: the number of tail terms
};

// Split (kind, n, m) into middle products of transform length <= 2^max_lg
// (GF(2)-linearity: a window's output is the parity of the sum over its input
// blocks; output windows are independent), choosing among single transforms
// and block shapes by an estimate of GPU time; shapes whose scratch exceeds
// budget (0 = no limit) are taken only if none fits.  False if invalid.
// fields: the field set of the products (kFields*).
// Planner figures taken on the device (cm_calibrate): ms per extraction of
// each transform length and field (the column-pass form), of a product alone
// on a cluster (2^14 .. 2^17), and the first column pass's length log2 R of
// two-pass plans.  Zero entries fall back to the built-in tables.
struct Tuning {
    double cost[3][33];  // [kFieldGL, kFieldF30, kFieldF25][lg]
    double cluster[kClusterMaxLg - kClusterMinLg + 1];
    int8_t split[3][33];  // [field][lg]
};
struct PlanOptions {
    int max_lg = 32;          // longest transform of one product (log2), 8..32
    int fields = kFieldsAll;  // F25 up to 2^25, F30 up to 2^30, Goldilocks above
    uint64_t budget = 0;      // scratch cap for choosing a shape (0 = none)
    uint32_t max_sum = 0;     // cap on blocks per sum group (0 = the field's bound)
    bool single = false;      // one transform whenever it fits (no cost-based split)
    const Tuning *tune = nullptr;  // the context's calibration, if any
};
// PlanOptions from cm_options (NULL: defaults); false if a value is invalid.
bool plan_options(const cm_options *opt, PlanOptions *o);
// Batches and the server plan their instances like single calls, restricted
// to one transform for the work-list kernel (which runs every such instance
// over F25 whatever the plan's field tag); instances past the work list's
// lengths go through the single-call planner.
inline int worklist_fields(const PlanOptions &o) { return o.fields == kFieldsGL ? kFieldsGL : kFieldsQ30; }
bool make_blocks(int kind, uint64_t n, uint64_t m, const PlanOptions &o, std::vector<Block> *out);

// Estimated GPU time (ms) of a block list, from measured per-length times.
double blocks_cost_ms(const std::vector<Block> &bl, const Tuning *tune = nullptr);

// Scratch bytes of a block list: the largest block's scratch, then an XOR
// temporary at *tmp_off (when blocks XOR), then 256 bytes of Dodis et al.
// precondition flags at *pre_off.
uint64_t blocks_scratch(const std::vector<Block> &bl, uint64_t *tmp_off, uint64_t *pre_off);

// z[i] ^= t[i], i < words (stream-ordered).
cudaError_t launch_xor_into(uint64_t *z, const uint64_t *t, uint64_t words, int nsm, cudaStream_t st);

// N_A membership and search (host, deterministic).
bool is_na_prime(uint64_t P);
bool is_prime(uint64_t n);

}  // namespace cm
