"""The allocation-free Toeplitz entry point, through the C ABI.

cm_toeplitz_noalloc serves callers that cannot allocate device memory: it
runs on fixed-size scratch compiled into the library.  This test checks, on
two calls in a row with different inputs (so stale scratch from the first call
would show in the second), that its output is bit-identical to that of the
ordinary cm_toeplitz entry point, and that sizes beyond its static limit are
refused.  It lives in its own file so that it is collected last.
"""

import numpy as np
import pytest
import torch

from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu

CASES = [(20000, 9001), (300000, 200000), (1000, 500), (2 ** 19, 2 ** 19 + 1)]


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
        assert not torch.equal(outs[0], outs[1])


def test_noalloc_rejects_beyond_limit():
    L = native.lib()
    st = torch.cuda.current_stream().cuda_stream
    d = to_dev(np.zeros(8, dtype=np.uint64))
    n, m = 2 ** 19, 2 ** 19 + 2          # n + m - 1 = 2^20 + 1
    assert L.cm_toeplitz_noalloc(d.data_ptr(), n, d.data_ptr(), m, d.data_ptr(), st) == native.CM_EINVAL
    assert L.cm_toeplitz_noalloc(None, 10, d.data_ptr(), 5, d.data_ptr(), st) == native.CM_EINVAL
    assert from_dev(d).sum() == 0
