"""The allocation-free Toeplitz entry point, through the C ABI.

cm_toeplitz_noalloc serves callers that cannot allocate device memory: it
runs on fixed-size scratch compiled into the library.  This test checks, on
two calls in a row with different inputs (so stale scratch from the first call
would show in the second), that its output is bit-identical to that of the
ordinary cm_toeplitz entry point and, on sampled rows, to the oracle's, that
calls on two streams ordered by an event agree, and that sizes beyond its
static limit are refused.  The sizes cover the one-CTA path, the smallest
length with a column pass (2^14) and the largest (2^20).  It lives in its own
file so that it is collected last.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu

CASES = [(20000, 9001), (300000, 200000), (1000, 500), (9000, 7000), (2 ** 19, 2 ** 19 + 1)]


def test_noalloc_matches_toeplitz_two_calls_in_a_row(cm_ctx):
    L = native.lib()
    st = torch.cuda.current_stream().cuda_stream
    for n, m in CASES:
        outs = []
        for call in range(2):
            xw = to_dev(inputs.bernoulli_half(700 + 2 * call, n))
            yw = to_dev(inputs.bernoulli_half(701 + 2 * call, n + m - 1))
            z = torch.full((native.words(m),), -1, dtype=torch.int64, device="cuda")
            s = L.cm_toeplitz_noalloc(xw.data_ptr(), n, yw.data_ptr(), m, z.data_ptr(), st)
            assert s == native.CM_OK, native.STATUS.get(s)
            ref = cm_ctx.toeplitz(xw, n, yw, m)
            outs.append(z)
            assert torch.equal(z, ref), (n, m, call)
            rows = np.unique(np.concatenate([np.arange(8), np.arange(m - 8, m),
                                             np.random.default_rng(n + call).integers(0, m, 24)]))
            zw = from_dev(z)
            got = ((zw[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
            assert (got == oracle.toeplitz_rows(from_dev(xw), n, from_dev(yw), m, rows)).all()
        assert not torch.equal(outs[0], outs[1])


def test_noalloc_two_streams_ordered_by_an_event(cm_ctx):
    # calls on one device share the scratch: a second stream that waits on an
    # event recorded after the first call gets its own correct result
    L = native.lib()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    n, m = 40000, 30000
    res = [(to_dev(inputs.bernoulli_half(710 + k, n)), to_dev(inputs.bernoulli_half(711 + k, n + m - 1)),
            torch.full((native.words(m),), -1, dtype=torch.int64, device="cuda")) for k in range(2)]
    torch.cuda.synchronize()  # inputs in place before the side streams read them
    ev = torch.cuda.Event()
    for k, st in enumerate((s1, s2)):
        xw, yw, z = res[k]
        if k == 1:
            s2.wait_event(ev)  # the second call starts after the first ends
        s = L.cm_toeplitz_noalloc(xw.data_ptr(), n, yw.data_ptr(), m, z.data_ptr(), st.cuda_stream)
        assert s == native.CM_OK, native.STATUS.get(s)
        if k == 0:
            ev.record(s1)
    torch.cuda.synchronize()
    for xw, yw, z in res:
        assert torch.equal(z, cm_ctx.toeplitz(xw, n, yw, m))


def test_noalloc_rejects_beyond_limit():
    L = native.lib()
    st = torch.cuda.current_stream().cuda_stream
    d = to_dev(np.zeros(8, dtype=np.uint64))
    n, m = 2 ** 19, 2 ** 19 + 2          # n + m - 1 = 2^20 + 1
    assert L.cm_toeplitz_noalloc(d.data_ptr(), n, d.data_ptr(), m, d.data_ptr(), st) == native.CM_EINVAL
    assert L.cm_toeplitz_noalloc(None, 10, d.data_ptr(), 5, d.data_ptr(), st) == native.CM_EINVAL
    assert from_dev(d).sum() == 0
