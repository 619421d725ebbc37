"""Batched extraction (one persistent work-list launch) vs the single calls and
the CPU oracle, bit for bit."""

import time

import numpy as np
import pytest
import torch

import oracle
from oracle import extractors as ex
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu
T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS


def ybits(kind, n, m):
    return n + m - 1 if kind == T else (n + 1 if kind == C else n)


def make_items(specs, stream0):
    items, host = [], []
    for j, (kind, n, m) in enumerate(specs):
        xw = inputs.bernoulli_half(stream0 + 2 * j, n)
        if kind == D:
            xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
        yw = inputs.bernoulli_half(stream0 + 2 * j + 1, ybits(kind, n, m))
        z = torch.full((native.words(m),), -1, dtype=torch.int64, device="cuda")
        items.append((kind, n, m, to_dev(xw), to_dev(yw), z))
        host.append((xw, yw))
    return items, host


def single(ctx, kind, n, m, x, y):
    if kind == T:
        return ctx.toeplitz(x, n, y, m)
    if kind == C:
        return ctx.circulant(x, n, y, m)
    return ctx.dodis(x, y, n, m)


def oracle_check(kind, n, m, xw, yw, z):
    zw = from_dev(z)
    if m <= 40000:
        ref = {T: oracle.toeplitz_packed, C: oracle.circulant_packed}.get(kind)
        want = ref(xw, n, yw, m) if ref else oracle.dodis_packed(xw, yw, n, m)
        assert (zw == want).all(), (kind, n, m)
    else:
        rows = np.unique(np.concatenate([np.arange(16), np.arange(m - 16, m),
                                         np.random.default_rng(m).integers(0, m, 48)]))
        got = ((zw[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
        fn = {T: lambda r: oracle.toeplitz_rows(xw, n, yw, m, r),
              C: lambda r: oracle.circulant_rows(xw, n, yw, m, r),
              D: lambda r: oracle.dodis_rows(xw, yw, n, m, r)}[kind]
        assert (got == fn(rows)).all(), (kind, n, m)


def mixed_specs():
    P = [oracle.next_na(v) for v in (600, 3000, 9000, 70000, 300000)]
    return [(T, 1000, 500), (T, 4096, 4097), (T, 5000, 4000), (T, 20000, 10000), (T, 2 ** 17, 2 ** 16),
            (C, P[0] - 1, P[0] // 2), (C, P[2] - 1, P[2] - 1), (C, P[3] - 1, P[3] // 2),
            (D, P[1], (2 * P[1]) // 5), (D, P[4], P[4] // 2), (T, 3, 2), (C, 10, 3),
            (T, 2 ** 21, 2 ** 20),  # L = 2^22: past the work list, the single-call kernels over F25
            (T, 2 ** 25, 2 ** 24)]  # L = 2^26: two column passes (single-call path)


def test_batch_mixed_matches_single_and_oracle(cm_ctx):
    specs = mixed_specs()
    items, host = make_items(specs, 900)
    b = cm_ctx.batch(items, autotune=True)
    b.launch()
    torch.cuda.synchronize()
    info = b.info()
    assert info["instances"] == len(specs) and info["solo_instances"] == 2 and info["graph"] == 1
    for (kind, n, m, x, y, z), (xw, yw) in zip(items, host):
        assert torch.equal(z, single(cm_ctx, kind, n, m, x, y)), (kind, n, m)
        oracle_check(kind, n, m, xw, yw, z)
    # replay: identical outputs after clearing them
    for it in items:
        it[5].fill_(-1)
    b.launch()
    torch.cuda.synchronize()
    for (kind, n, m, x, y, z), (xw, yw) in zip(items, host):
        assert torch.equal(z, single(cm_ctx, kind, n, m, x, y))
    assert cm_ctx.device_status() == (native.CM_OK, 0)
    b.close()


def test_batch_loguniform_toeplitz(cm_ctx):
    # the batched workload's shape at reduced count: n = floor(2^U), U ~ U[10, 18], m = n / 2
    ns = inputs.loguniform_lengths(1, 48, 10, 18)
    specs = [(T, int(n), int(n) // 2) for n in ns]
    items, host = make_items(specs, 5000)
    cm_ctx.batch_extract(items)
    for (kind, n, m, x, y, z), (xw, yw) in zip(items, host):
        assert torch.equal(z, cm_ctx.toeplitz(x, n, y, m)), (n, m)
    for (kind, n, m, x, y, z), (xw, yw) in list(zip(items, host))[::6]:
        oracle_check(kind, n, m, xw, yw, z)


def test_batch_dodis_precondition_isolated(cm_ctx):
    P = oracle.next_na(20000)
    Q = oracle.next_na(500)
    specs = [(D, P, P // 2), (D, Q, Q // 2), (T, 3000, 1000)]
    items, host = make_items(specs, 7000)
    bad_x = to_dev(ex.pack_bits(np.ones(P, dtype=np.uint8)))
    bad_small = to_dev(ex.pack_bits(np.zeros(Q, dtype=np.uint8)))
    items[0] = (D, P, P // 2, bad_x, items[0][4], items[0][5])
    items[1] = (D, Q, Q // 2, bad_small, items[1][4], items[1][5])
    cm_ctx.batch_extract(items)
    s, f = cm_ctx.device_status()
    assert s == native.CM_EPRECOND and f & native.FLAG_PRECOND
    assert not from_dev(items[0][5]).any() and not from_dev(items[1][5]).any()
    kind, n, m, x, y, z = items[2]
    assert torch.equal(z, cm_ctx.toeplitz(x, n, y, m))


def test_batch_invalid_descriptor(cm_ctx):
    items, _ = make_items([(T, 100, 50)], 8000)
    bad = (C, 6, 3, items[0][3], items[0][4], items[0][5])   # 7 not in N_A
    with pytest.raises(native.CMError):
        cm_ctx.batch([items[0], bad])
    # cm_batch_toeplitz refuses a batch with a non-Toeplitz descriptor
    kind, n, m, x, y, z = items[0]
    arr = cm_ctx._descs([(C, n, m, x, y, z)])   # n + 1 = 101 is in N_A: valid Circulant
    s = native.lib().cm_batch_toeplitz(cm_ctx.handle, native.ctypes.cast(arr, native.ctypes.c_void_p), 1,
                                       torch.cuda.current_stream().cuda_stream)
    assert s == native.CM_EINVAL


def test_batch_bounded_wait_times_out_and_context_survives(cm_ctx):
    # one instance waits for a forward-tile count that nothing will reach: the
    # bounded spin runs out, the kernel sets CM_FLAG_TIMEOUT and returns (no
    # trap, no hang), and the context keeps working
    specs = [(T, 20000, 10000), (T, 3000, 1000), (T, 70000, 30000)]
    items, _ = make_items(specs, 6100)
    b = cm_ctx.batch(items, test_stall=True)
    t0 = time.time()
    b.launch()
    torch.cuda.synchronize()
    elapsed = time.time() - t0
    s, f = cm_ctx.device_status()
    assert s == native.CM_ETIMEDOUT and f & native.FLAG_TIMEOUT
    assert elapsed < 60.0
    b.close()
    kind, n, m, x, y, z = items[1]
    z2 = cm_ctx.toeplitz(x, n, y, m)
    assert cm_ctx.device_status() == (native.CM_OK, 0)
    good = cm_ctx.batch(items)
    good.launch()
    torch.cuda.synchronize()
    assert cm_ctx.device_status() == (native.CM_OK, 0)
    assert torch.equal(items[1][5], z2)
    good.close()


def test_batch_workload_size_sampled(cm_ctx):
    # the batched (a) workload at full size, in the launch configuration the
    # bench times (autotuned plan, CUDA-graph replay): 4096 Toeplitz instances,
    # n = floor(2^U), U ~ U[10, 22), m = n / 2, the bench's seeds; every
    # instance's first and last 4 rows and 8 random ones (64 random ones for
    # the 24 longest instances) against the oracle; tails zero
    count = 4096
    ns = inputs.loguniform_lengths(1, count, 10, 22)
    ms = ns // 2
    items, host = [], []
    for j in range(count):
        n, m = int(ns[j]), int(ms[j])
        xw = inputs.bernoulli_half(10000 + 2 * j, n)
        yw = inputs.bernoulli_half(10001 + 2 * j, n + m - 1)
        z = torch.full((native.words(m),), -1, dtype=torch.int64, device="cuda")
        items.append((T, n, m, to_dev(xw), to_dev(yw), z))
        host.append((xw, yw))
    b = cm_ctx.batch(items, autotune=True, graph=True)
    b.launch()
    b.launch()  # a replay writes the same bits
    torch.cuda.synchronize()
    assert cm_ctx.device_status() == (native.CM_OK, 0)
    rng = np.random.default_rng(4096)
    longest = set(np.argsort(ns)[-24:].tolist())
    for j in range(count):
        n, m = int(ns[j]), int(ms[j])
        xw, yw = host[j]
        zw = from_dev(items[j][5])
        k = 64 if j in longest else 8
        rows = np.unique(np.concatenate([np.arange(min(4, m)), np.arange(max(0, m - 4), m),
                                         rng.integers(0, m, k)]))
        got = ((zw[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
        assert (got == oracle.toeplitz_rows(xw, n, yw, m, rows)).all(), (j, n, m)
        if m & 63:
            assert int(zw[-1]) >> (m & 63) == 0, (j, n, m)
    b.close()
