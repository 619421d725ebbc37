"""Von Neumann extraction on the GPU (cm_von_neumann) against the oracle.

Bit-exact parity (output bits and length m) on seeded inputs of several biases
at sizes from one pair to several 4096-word tiles with ragged tails; sparse
inputs whose few unequal pairs sit tiles apart (so the carried prefix crosses
runs of tiles with no output); the no-output case (Alg. vn's error); argument
checks; words past the output left untouched; the host-buffer form; and, at the
6.5e9-bit size of the paper's QRNG example, the length and sampled output bits
against the oracle's word counts.
"""

import numpy as np
import pytest
import torch

from oracle import von_neumann as vn
from oracle.extractors import pack_bits
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu
TILE_BITS = 4096 * 64


def thr(p):
    return int(round(p * 2 ** 32))


def gen(n, p, stream):
    if p == 0.5:
        return inputs.bernoulli_half(stream, n)
    return inputs.bernoulli(stream, n, thr(p))


def run(ctx, xw, n, sentinel=True):
    x = to_dev(xw)
    z = torch.full((max(1, native.words(n // 2)),), -1 if sentinel else 0, dtype=torch.int64, device="cuda")
    z, m = ctx.von_neumann(x, n, z)
    torch.cuda.synchronize()
    return from_dev(z), int(m.item())


def check(ctx, xw, n):
    z, m = run(ctx, xw, n)
    want, mw = vn.von_neumann_packed(xw, n)
    assert m == mw, (n, m, mw)
    k = native.words(m)
    assert (z[:k] == want[:k]).all(), n
    # later words are not written
    assert (z[k:] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    assert ctx.device_status()[0] == native.CM_OK


@pytest.mark.parametrize("n,p", [
    (2, 0.5), (3, 0.5), (64, 0.5), (65, 0.5), (127, 0.5), (128, 0.5), (129, 0.5),
    (TILE_BITS, 0.5), (TILE_BITS + 2, 0.5), (TILE_BITS - 1, 0.5),
    (3 * TILE_BITS + 4321, 0.5), (1_000_001, 0.8), (5_000_000, 0.5),
    (2_000_003, 0.1), (3_000_000, 0.99), (10_000_007, 0.5), (40 * TILE_BITS + 77, 0.7),
])
def test_parity_random(cm_ctx, n, p):
    xw = gen(n, p, 17 + n % 1000)
    if vn.von_neumann_count(xw, n) == 0:
        xw[0] = (xw[0] & ~np.uint64(3)) | np.uint64(1)
    check(cm_ctx, xw, n)


@pytest.mark.parametrize("positions", [
    [0],                                     # a single output bit
    [5 * TILE_BITS + 130],                   # one bit, deep in the input
    [3, 2 * TILE_BITS, 9 * TILE_BITS + 64, 30 * TILE_BITS - 2],
    list(range(0, 36 * TILE_BITS, TILE_BITS // 3))[:100],  # ~3 per tile, tails across tiles
])
def test_sparse_outputs_across_empty_tiles(cm_ctx, positions):
    # all pairs equal except unequal pairs at the given (even) bit positions,
    # alternating "10" and "01" so that output values vary
    n = 36 * TILE_BITS + 5
    b = np.zeros(n, dtype=np.uint8)
    for i, pos in enumerate(positions):
        pos -= pos % 2
        b[pos], b[pos + 1] = (1, 0) if i % 2 == 0 else (0, 1)
    check(cm_ctx, pack_bits(b), n)


def test_runs_of_ones_and_long_outputs(cm_ctx):
    # every pair unequal for whole tiles (the densest output: 32 bits a word)
    n = 6 * TILE_BITS + 66
    b = np.zeros(n, dtype=np.uint8)
    b[0:2 * TILE_BITS:2] = 1                      # pairs "10": output 1s
    b[2 * TILE_BITS + 1:4 * TILE_BITS:2] = 1      # pairs "01": output 0s
    rng = np.random.default_rng(5)
    b[4 * TILE_BITS:] = rng.integers(0, 2, n - 4 * TILE_BITS)
    check(cm_ctx, pack_bits(b), n)


def test_no_output_sets_precondition(cm_ctx):
    for n, fill in ((2, 0), (1000, 1), (3 * TILE_BITS + 9, 0)):
        b = np.full(n, fill, dtype=np.uint8)
        x = to_dev(pack_bits(b))
        z = torch.full((native.words(n // 2),), -1, dtype=torch.int64, device="cuda")
        _, m = cm_ctx.von_neumann(x, n, z)
        assert cm_ctx.device_status()[0] == native.CM_EPRECOND
        assert int(m.item()) == 0
        assert (from_dev(z) == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    # "0011" pairs are equal too
    b = np.tile(np.array([0, 0, 1, 1], dtype=np.uint8), 5000)
    _, m = cm_ctx.von_neumann(to_dev(pack_bits(b)), b.size)
    assert cm_ctx.device_status()[0] == native.CM_EPRECOND and int(m.item()) == 0


def test_argument_checks(cm_ctx):
    L = cm_ctx._L
    x = torch.zeros(64, dtype=torch.int64, device="cuda")
    z = torch.zeros(64, dtype=torch.int64, device="cuda")
    m = torch.zeros(2, dtype=torch.int64, device="cuda")
    h = cm_ctx.handle
    assert L.cm_von_neumann(h, x.data_ptr(), 1, z.data_ptr(), m.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_von_neumann(h, x.data_ptr(), 0, z.data_ptr(), m.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_von_neumann(h, None, 100, z.data_ptr(), m.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_von_neumann(h, x.data_ptr(), 100, None, m.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_von_neumann(h, x.data_ptr(), 100, z.data_ptr(), None, None) == native.CM_EINVAL
    # x must be 16-byte aligned
    assert L.cm_von_neumann(h, x.data_ptr() + 8, 100, z.data_ptr(), m.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_von_neumann(h, x.data_ptr(), 1 << 46, z.data_ptr(), m.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_von_neumann(None, x.data_ptr(), 100, z.data_ptr(), m.data_ptr(), None) == native.CM_EINVAL
    assert native.lib().cm_von_neumann_scratch_bytes(1) == 0
    assert native.lib().cm_von_neumann_scratch_bytes(TILE_BITS * 3) == 256 + 12 * 3 + 16 * 4096


def test_two_calls_in_a_row_and_streams(cm_ctx):
    n = 2 * TILE_BITS + 1000
    a, b = gen(n, 0.5, 301), gen(n, 0.3, 302)
    s = torch.cuda.Stream()
    xa, xb = to_dev(a), to_dev(b)
    za, ma = cm_ctx.von_neumann(xa, n)
    with torch.cuda.stream(s):
        zb, mb = cm_ctx.von_neumann(xb, n, stream=s)
    s.synchronize()
    torch.cuda.synchronize()
    for xw, z, m in ((a, za, ma), (b, zb, mb)):
        want, mw = vn.von_neumann_packed(xw, n)
        assert int(m.item()) == mw
        assert (from_dev(z)[:native.words(mw)] == want).all()


def test_host_buffers(cm_ctx):
    n = 3 * TILE_BITS + 12345
    xw = gen(n, 0.6, 77)
    xh = torch.from_numpy(xw.view(np.int64)).pin_memory()
    zh = torch.full((native.words(n // 2),), -1, dtype=torch.int64).pin_memory()
    s, m = cm_ctx.von_neumann_host(xh, n, zh)
    want, mw = vn.von_neumann_packed(xw, n)
    assert s == native.CM_OK and m == mw
    assert (zh.numpy().view(np.uint64)[:native.words(m)] == want).all()
    zero = torch.zeros(native.words(1000), dtype=torch.int64)
    s, m = cm_ctx.von_neumann_host(zero, 1000, torch.zeros(native.words(500), dtype=torch.int64))
    assert s == native.CM_EPRECOND and m == 0
    cm_ctx.device_status()  # clear the flag the kernel raised


@pytest.mark.slow
def test_qrng_size_sampled(cm_ctx):
    # n = 6.5e9 bits (the QRNG example's input length), Bernoulli(1/2): the
    # length and 400 sampled output bits against the oracle's word counts
    n = 6_500_000_000
    xw = inputs.bernoulli_half(2402, n)
    x = to_dev(xw)
    z, m = cm_ctx.von_neumann(x, n)
    torch.cuda.synchronize()
    m = int(m.item())
    rng = np.random.default_rng(1)
    pos = np.sort(rng.integers(0, m, 400))
    want, mw = vn.output_bits_at(xw, n, pos)
    assert m == mw
    zc = from_dev(z)
    got = ((zc[pos // 64] >> (pos % 64).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
    assert (got == want).all()
    # the last word's bits past m are zero
    if m % 64:
        assert zc[m // 64] >> np.uint64(m % 64) == 0
    assert cm_ctx.device_status()[0] == native.CM_OK
