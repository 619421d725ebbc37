// cm_toeplitz_noalloc: the Toeplitz extraction with no device allocation.
//
// For callers that cannot allocate device memory (see include/cm.h).  The
// scratch of the multi-pass path (operands A and B, L u64 words each, and the
// parity bytes of the output window) and the root tables live in file-scope
// __device__ arrays of fixed size, so every GPU that loads the library holds
// them (about 19 MB) until the process exits.  Host code never dereferences or
// passes the arrays' names: their device addresses come from
// cudaGetSymbolAddress at set-up, once per device, with that device current.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "cm.h"
#include "cm_internal.h"

namespace cm {
namespace {

constexpr int kNoAllocMaxLg = 20;  // n + m - 1 <= 2^20
constexpr uint64_t kNoAllocMaxL = 1ull << kNoAllocMaxLg;
// A (8L) + B (8L) + parity bytes of the window (m <= L)
constexpr size_t kNoAllocScratchBytes = 2 * 8 * kNoAllocMaxL + kNoAllocMaxL;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ __align__(256) uint64_t g_noalloc_tables[kTableWords];
static __device__ __align__(256) uint32_t g_noalloc_status[64];

struct NoAllocDevice {
    bool ready;
    uint64_t ctx_id;  // the CUDA context the set-up ran in (current_ctx_id)
    unsigned char *scratch;
    uint64_t *tables;
    uint32_t *status;
    int nsm;
};

constexpr int kMaxDevices = 128;
static NoAllocDevice g_devices[kMaxDevices];
static std::mutex g_setup_mu;

__device__ uint64_t pow_dev(uint64_t a, uint32_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = gl_mul(r, a);
        a = gl_mul(a, a);
        e >>= 1;
    }
    return r;
}

// Same table layout as the context's: omega_8192^e (e < 8192), then g^e,
// g^(2^16 e), g^-e, g^-(2^16 e) for e < 2^16.
__global__ void k_noalloc_tables(uint64_t *t, uint64_t w, uint64_t g, uint64_t g16,
                                 uint64_t gi, uint64_t gi16) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 8192) t[e] = pow_dev(w, e);
    if (e < 65536) {
        uint64_t *base = t + 8192;
        base[e] = pow_dev(g, e);
        base[65536 + e] = pow_dev(g16, e);
        base[2 * 65536 + e] = pow_dev(gi, e);
        base[3 * 65536 + e] = pow_dev(gi16, e);
    }
}

// Set-up of device dev (current), once per CUDA context: a device reset
// replaces the primary context, whose __device__ arrays start over (addresses
// and root tables), so a new context runs the set-up again.
cm_status setup_device(int dev, NoAllocDevice **out) {
    if (dev < 0 || dev >= kMaxDevices) return CM_EDEVICE;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    NoAllocDevice &d = g_devices[dev];
    const uint64_t ctx = current_ctx_id();
    if (d.ready && (ctx == 0 || ctx != d.ctx_id)) d.ready = false;
    if (!d.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return CM_EDEVICE;
        d.scratch = static_cast<unsigned char *>(p);
        if (cudaGetSymbolAddress(&p, g_noalloc_tables) != cudaSuccess) return CM_EDEVICE;
        d.tables = static_cast<uint64_t *>(p);
        if (cudaGetSymbolAddress(&p, g_noalloc_status) != cudaSuccess) return CM_EDEVICE;
        d.status = static_cast<uint32_t *>(p);
        if (cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return CM_EDEVICE;
        const uint64_t g = gl_root_2_32_host(0), gi = gl_root_2_32_host(1);
        const uint64_t w = gl_pow_host(g, 1ull << (32 - kSmallLg));
        const uint64_t g16 = gl_pow_host(g, 65536), gi16 = gl_pow_host(gi, 65536);
        k_noalloc_tables<<<65536 / 256, 256, 0, 0>>>(d.tables, w, g, g16, gi, gi16);
        if (cudaGetLastError() != cudaSuccess) return CM_EDEVICE;
        if (cudaMemsetAsync(d.status, 0, sizeof(uint32_t) * 64, 0) != cudaSuccess) return CM_EDEVICE;
        if (cudaStreamSynchronize(0) != cudaSuccess) return CM_EDEVICE;
        d.ctx_id = ctx;
        d.ready = true;
    }
    *out = &d;
    return CM_OK;
}

cm_status status_of(cudaError_t e) { return e == cudaSuccess ? CM_OK : CM_EDEVICE; }

}  // namespace
}  // namespace cm

using namespace cm;

extern "C" cm_status cm_toeplitz_noalloc(const uint64_t *x, uint64_t n, const uint64_t *y, uint64_t m,
                                         uint64_t *z, cm_stream stream) {
    if (!x || !y || !z) return CM_EINVAL;
    Plan p;
    if (!make_plan(CM_TOEPLITZ, n, m, &p)) return CM_EINVAL;
    if (p.L > kNoAllocMaxL) return CM_EINVAL;  // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CM_EDEVICE;
    NoAllocDevice *d = nullptr;
    cm_status s = setup_device(dev, &d);
    if (s != CM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    RootTables rt{};
    rt.small = d->tables;
    rt.big_lo_fwd = d->tables + 8192;
    rt.big_hi_fwd = rt.big_lo_fwd + 65536;
    rt.big_lo_inv = rt.big_hi_fwd + 65536;
    rt.big_hi_inv = rt.big_lo_inv + 65536;

    BitMap am, bm;
    am.src = x; am.mode = p.amode; am.len = p.alen; am.srclen = p.asrclen; am.off = p.aoff;
    bm.src = y; bm.mode = p.bmode; bm.len = p.blen; bm.srclen = p.bsrclen; bm.off = p.boff;
    const uint64_t linv = gl_inv_pow2_host(p.L);

    if (p.npass == 0) {
        Launch q;
        q.amap = am;
        q.bmap = bm;
        q.lo = p.lo;
        q.m = p.m;
        q.linv = linv;
        q.z = z;
        q.pre = nullptr;
        q.status = d->status;
        q.field = kFieldGL;
        q.rt = rt;
        q.rt30 = RootTables30{};
        q.rt25 = RootTables25{};
        q.stream = st;
        return status_of(launch_small(q, p.lg));
    }
    // L <= 2^20: a single column pass (R = L / 2^13) around the on-chip middle.
    // Every word of A, B and the window's parity bytes is written before it is
    // read in this call, so nothing left by an earlier call is ever used.
    uint64_t *A = reinterpret_cast<uint64_t *>(d->scratch);
    uint64_t *B = A + p.L;
    uint8_t *par = reinterpret_cast<uint8_t *>(B + p.L);
    const int lgN = p.lg, lgS = p.lg - p.pass_lg[0];
    for (int op = 0; op < 2; ++op) {
        PassArgs a = {};
        a.data = op == 0 ? A : B;
        a.map = op == 0 ? am : bm;
        a.lgN = lgN;
        a.lgS = lgS;
        a.rt = rt;
        a.L = p.L;
        a.inv = false;
        a.bits_in = true;
        if ((s = status_of(launch_pass(a, p.pass_lg[0], st))) != CM_OK) return s;
    }
    if ((s = status_of(launch_middle(kFieldGL, A, B, nullptr, kMidAlone, p.L, linv, rt, RootTables30{}, RootTables25{},
                                         d->nsm, st))) != CM_OK)
        return s;
    PassArgs a = {};
    a.data = A;
    a.lgN = lgN;
    a.lgS = lgS;
    a.rt = rt;
    a.L = p.L;
    a.inv = true;
    a.parity_out = true;
    a.par = par;
    a.lo = p.lo;
    a.m = p.m;
    if ((s = status_of(launch_pass(a, p.pass_lg[0], st))) != CM_OK) return s;
    return status_of(launch_pack(par, p.m, z, nullptr, d->status, d->nsm, st));
}
