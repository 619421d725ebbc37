// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "cm.h"
#include "ntt_device.cuh"

namespace cm {

constexpr uint32_t kFlagPrecond = CM_FLAG_PRECOND;
constexpr uint32_t kFlagTimeout = CM_FLAG_TIMEOUT;
constexpr size_t kTableWords = 8192 + 4 * 65536;  // resident root tables

// Transform fields (see ntt_device.cuh).
constexpr int kFieldGL = 0;   // Goldilocks, 64-bit elements, L <= 2^32
constexpr int kFieldF30 = 1;  // 3 * 2^30 + 1, 32-bit elements, L <= 2^30
constexpr int kF30MaxLg = 30;
constexpr size_t kTable30Words = 8192 + 4 * 32768;  // resident F30 root tables

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
    cudaStream_t stream;
};

// Arguments of one column pass.  data: L elements of the field's word size.
struct PassArgs {
    void *data;
    BitMap map;
    int lgN, lgS;
    uint8_t *par;
    uint64_t lo, m;
    int field;
    RootTables rt;
    RootTables30 rt30;
    uint64_t L;
    bool inv, bits_in, parity_out;
};

cudaError_t launch_small(const Launch &q, int lg);
cudaError_t launch_pass(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_fwd(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_inv(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_fwd30(const PassArgs &a, int logr, cudaStream_t st);
cudaError_t launch_pass_inv30(const PassArgs &a, int logr, cudaStream_t st);
// A, B: L elements of the field's word size.
cudaError_t launch_middle(int field, void *A, const void *B, uint64_t L, uint64_t linv, const RootTables &rt,
                          const RootTables30 &rt30, int nsm, cudaStream_t st);
cudaError_t launch_pack(const uint8_t *par, uint64_t m, uint64_t *z, const uint32_t *pre,
                        uint32_t *status, int nsm, cudaStream_t st);
cudaError_t launch_allsame(const uint64_t *x, uint64_t n, uint32_t *flags, int nsm, cudaStream_t st);

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
    int field;       // kFieldGL or kFieldF30
};

// Validate (kind, n, m) and fill the plan; false if invalid or if K + m - 1
// exceeds 2^32 (one transform).
// allow_f30: a transform of length <= 2^30 runs over the 32-bit field.
bool make_plan(int kind, uint64_t n, uint64_t m, Plan *out, bool allow_f30 = false);

// Longest bit string a blocked extraction takes (the paper's 2^40).
constexpr uint64_t kMaxBits = 1ull << 40;
constexpr uint64_t kMaxBlocks = 1u << 16;

// One product of a blocked extraction: plan p (a middle product over an
// input block and an output block), written to z + zword words; the first
// block of each output window writes, later ones XOR into it.
struct Block {
    Plan p;
    uint64_t zword;
    bool accumulate;
};

// Split (kind, n, m) into middle products of transform length <= 2^max_lg
// (GF(2)-linearity: the output is the XOR over input blocks; output blocks are
// independent).  One block when K + m - 1 <= 2^max_lg.  False if invalid.
// allow_f30: blocks whose transform fits 2^30 run over the 32-bit field.
bool make_blocks(int kind, uint64_t n, uint64_t m, int max_lg, bool allow_f30, std::vector<Block> *out);

// z[i] ^= t[i], i < words (stream-ordered).
cudaError_t launch_xor_into(uint64_t *z, const uint64_t *t, uint64_t words, int nsm, cudaStream_t st);

// N_A membership and search (host, deterministic).
bool is_na_prime(uint64_t P);
bool is_prime(uint64_t n);

}  // namespace cm
