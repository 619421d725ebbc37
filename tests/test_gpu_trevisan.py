"""Trevisan's one-bit step on the GPU (cm_trevisan_rsh, cm_trevisan) against
the oracle (oracle/trevisan.py), bit for bit: field sizes of one to four
64-bit words (l = 3 .. 256, including l a multiple of 64), ragged n and m
(output tails), an input shorter than one chunk, seeds gathered from a weak
design's sets, and argument errors."""

import numpy as np
import pytest
import torch

from oracle import extractors as ex
from oracle import trevisan as tv
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu


def bits_of(words, nbits):
    return ex.unpack_bits(words, nbits)


def run_rsh(ctx, xw, n, l, sw, m):
    return from_dev(ctx.trevisan_rsh(to_dev(xw), n, l, to_dev(sw), m))


def want_rsh(xw, n, l, sw, m):
    xb = bits_of(xw, n)
    sb = bits_of(sw, 2 * l * m)
    f = tv.rsh_modulus(l)
    z = [tv.rsh_onebit(xb, n, sb[2 * l * i: 2 * l * (i + 1)], l, f) for i in range(m)]
    return ex.pack_bits(np.array(z, dtype=np.uint8))


CASES = [
    # (n, l, m): W = 1 .. 4 words per element, delta = 0 at l = 64, 128, 256
    (1, 3, 5), (5, 3, 64), (200, 7, 65), (1000, 17, 130), (4097, 63, 64), (3000, 64, 100),
    (3001, 65, 33), (20000, 100, 96), (9000, 128, 70), (9001, 129, 40), (6000, 200, 37), (5000, 256, 31),
    (100, 121, 10),   # n < l: one chunk
    # few outputs: chunks shared by 8 or 32 threads per output, with leading
    # zero chunks padding s to a multiple of the group
    (60000, 64, 100), (200000, 30, 77), (150000, 129, 50), (300000, 256, 40),
    (100000, 100, 30), (400000, 150, 10), (600000, 256, 8),
]


@pytest.mark.parametrize("n,l,m", CASES)
def test_rsh_matches_oracle(cm_ctx, n, l, m):
    xw = inputs.bernoulli_half(1100 + n % 97, n)
    sw = inputs.bernoulli_half(1101 + l, 2 * l * m)
    got = run_rsh(cm_ctx, xw, n, l, sw, m)
    assert (got == want_rsh(xw, n, l, sw, m)).all(), (n, l, m)
    if m & 63:
        assert int(got[-1]) >> (m & 63) == 0


def test_rsh_linear_and_zero(cm_ctx):
    n, l, m = 5000, 90, 256
    a, b = inputs.bernoulli_half(1200, n), inputs.bernoulli_half(1201, n)
    sw = inputs.bernoulli_half(1202, 2 * l * m)
    za, zb = run_rsh(cm_ctx, a, n, l, sw, m), run_rsh(cm_ctx, b, n, l, sw, m)
    assert (run_rsh(cm_ctx, a ^ b, n, l, sw, m) == (za ^ zb)).all()
    assert not run_rsh(cm_ctx, np.zeros_like(a), n, l, sw, m).any()


def test_trevisan_sets(cm_ctx):
    rng = np.random.default_rng(12)
    n, l, d, m, t = 3000, 40, 700, 50, 83
    xw, yw = inputs.bernoulli_half(1300, n), inputs.bernoulli_half(1301, d)
    sets = np.stack([np.sort(rng.choice(d, t, replace=False)) for _ in range(m)]).astype(np.int32)
    z = from_dev(cm_ctx.trevisan(to_dev(xw), n, to_dev(yw), d, torch.from_numpy(sets).cuda(), t, m, l))
    want = tv.trevisan(bits_of(xw, n), n, bits_of(yw, d), [s[:2 * l] for s in sets], l)
    assert (z == ex.pack_bits(want)).all()


def test_argument_errors(cm_ctx):
    x = torch.zeros(4, dtype=torch.int64, device="cuda")
    s = torch.zeros(64, dtype=torch.int64, device="cuda")
    L = native.lib()
    h = cm_ctx.handle
    assert L.cm_trevisan_rsh(h, x.data_ptr(), 100, 1, s.data_ptr(), 1, x.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_trevisan_rsh(h, x.data_ptr(), 100, 257, s.data_ptr(), 1, x.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_trevisan_rsh(h, x.data_ptr(), 100, 8, s.data_ptr(), 0, x.data_ptr(), None) == native.CM_EINVAL
    assert L.cm_trevisan_rsh(h, x.data_ptr(), 0, 8, s.data_ptr(), 1, x.data_ptr(), None) == native.CM_EINVAL
    sets = torch.zeros(64, dtype=torch.int32, device="cuda")
    assert L.cm_trevisan(h, x.data_ptr(), 100, s.data_ptr(), 64, sets.data_ptr(), 15, 1, 8, x.data_ptr(),
                         None) == native.CM_EINVAL   # t < 2l


@pytest.mark.slow
def test_rsh_workload_size_sampled(cm_ctx):
    # the bench workload's input (n = 2^20, l = 121) on 1024 outputs; the
    # oracle checks outputs 0, 1, 511, 1022, 1023 (about 0.4 s each)
    n, m, l = 1 << 20, 1024, 121
    xw = inputs.bernoulli_half(1400, n)
    sw = inputs.bernoulli_half(1401, 2 * l * m)
    got = bits_of(run_rsh(cm_ctx, xw, n, l, sw, m), m)
    xb, sb = bits_of(xw, n), bits_of(sw, 2 * l * m)
    f = tv.rsh_modulus(l)
    for i in (0, 1, 511, 1022, 1023):
        assert got[i] == tv.rsh_onebit(xb, n, sb[2 * l * i: 2 * l * (i + 1)], l, f), i


def test_thread_groups_agree(cm_ctx):
    # the same seeds' outputs with one thread per output (many outputs) and
    # with 8 or 32 threads per output (few outputs)
    n, l = 1 << 18, 77
    big, small = 40000, 300
    xw = inputs.bernoulli_half(1500, n)
    sw = inputs.bernoulli_half(1501, 2 * l * big)
    zb = bits_of(run_rsh(cm_ctx, xw, n, l, sw, big), big)
    zs = bits_of(run_rsh(cm_ctx, xw, n, l, sw, small), small)
    assert (zb[:small] == zs).all()
