// Work-list kernel interface shared by the batch planner and the server.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "cm.h"
#include "cm_internal.h"

namespace cm {

enum ItemType : uint16_t { kItSmall = 0, kItFwdA, kItFwdB, kItMiddle, kItInv, kItPack, kItCheck };
constexpr int kPackWordsPerItem = 1 << 16;

struct BatchInst {
    BitMap amap, bmap;
    void *A, *B;  // L elements each of the work list's field (32-bit words)
    uint8_t *par;
    uint64_t *z;
    uint32_t *pre;  // Dodis et al.: {any 1 bit, any 0 bit} of x, else null
    uint64_t lo, m, linv, nx;  // linv in the field's product form
    int32_t lg, logr, tile_lg, kind;
    uint32_t need[4];  // items per phase
};

struct WorkItem {
    uint32_t inst;
    uint16_t type;
    uint16_t phase;
    uint32_t idx;
    uint32_t pad;
};

// Instances with transforms up to 2^21 go on the work list; longer ones run
// the single-call kernels (column passes fused with the products over F25 up
// to 2^25), which are faster per element than the work list's runtime-size
// steps once a transform fills the GPU on its own.
constexpr int kWorklistMaxLg = 21;
inline bool on_worklist(const Plan &p) { return p.npass <= 1 && p.lg <= kWorklistMaxLg; }

// Scratch one work-list instance needs (0 for L <= 2^13): operands A and B
// (L elements each of the work list's field, 4 bytes) and the parity bytes of
// its window.
size_t worklist_scratch_bytes(const Plan &p);

// Bytes of one resident seed transform (operand B) of a work-list instance.
size_t worklist_seed_bytes(const Plan &p);

// Instance table and phase-ordered work list for the instances idx[0..n) of
// descs/plans.  Instance k's scratch starts at scratch + off[idx[k]]; Dodis
// et al. instances get precondition flags at pre + 2 k (pre may be null when
// none is Dodis et al.).  Within a phase, larger transforms come first.
// bext (may be null): per instance k, an external buffer for the transformed
// seed operand B; if bready[k] it already holds that transform (its forward
// tiles are skipped), otherwise the forward tiles write it there.
void build_worklist(const cm_desc *descs, const Plan *plans, const uint32_t *idx, uint32_t n,
                    uint8_t *scratch, const size_t *off, int tile_lg, uint32_t *pre,
                    std::vector<BatchInst> &insts, std::vector<WorkItem> &items,
                    void *const *bext = nullptr, const uint8_t *bready = nullptr, bool test_stall = false);

// Dynamic shared memory of the work-list kernel and its resident grid.
size_t batch_smem_bytes();
int batch_grid(int nsm);

// One launch of the work-list kernel; ctrl holds 2 + 4 n zeroed words.
cudaError_t launch_k_batch(const BatchInst *insts, const WorkItem *items, uint32_t nitems, uint32_t *ctrl,
                           uint32_t *status, const RootTables25 &rt, int grid, cudaStream_t st);

}  // namespace cm
