"""Many inputs under one Toeplitz seed: the three dense engines (INT8 and
binary tensor cores, GF(2) CUDA cores) vs the single-call NTT path and the CPU
oracle."""

import numpy as np
import pytest
import torch

import oracle
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu


def run_case(ctx, n, m, count, engine, seed):
    wx, wz = native.words(n), native.words(m)
    yw = inputs.bernoulli_half(seed, n + m - 1)
    X = np.concatenate([inputs.bernoulli_half(seed + 1 + c, n) for c in range(count)])
    Xd, yd = to_dev(X), to_dev(yw)
    # dirty tails in every input: the product must ignore them
    if n % 64:
        Xd.view(-1, wx)[:, -1] |= torch.tensor(-(1 << 62), dtype=torch.int64, device="cuda")
    Z = ctx.toeplitz_shared_seed(yd, n, m, Xd, count, engine=engine)
    Zh = from_dev(Z).reshape(count, wz)
    for c in range(count):
        ref = from_dev(ctx.toeplitz(Xd[c * wx:(c + 1) * wx], n, yd, m))
        assert (Zh[c] == ref).all(), (engine, c)
    for c in (0, count // 2, count - 1):
        assert (Zh[c] == oracle.toeplitz_packed(X[c * wx:(c + 1) * wx], n, yw, m)).all()
    if m % 64:
        assert not (Zh[:, -1] >> np.uint64(m % 64)).any()
    return Zh


@pytest.mark.parametrize("engine", [native.ENGINE_IMMA, native.ENGINE_GF2, native.ENGINE_BMMA])
def test_engines_config_shape(cm_ctx, engine):
    run_case(cm_ctx, 4096, 2048, 300, engine, 11)


@pytest.mark.parametrize("engine", [native.ENGINE_IMMA, native.ENGINE_GF2, native.ENGINE_BMMA])
@pytest.mark.parametrize("n,m,count", [(1000, 333, 257), (77, 1, 3), (1, 65, 129), (5000, 4000, 9)])
def test_engines_ragged(cm_ctx, engine, n, m, count):
    run_case(cm_ctx, n, m, count, engine, 21)


def test_auto_engine_agrees(cm_ctx):
    a = run_case(cm_ctx, 3000, 1500, 200, native.ENGINE_AUTO, 31)
    b = run_case(cm_ctx, 3000, 1500, 200, native.ENGINE_GF2, 31)
    assert (a == b).all()
    assert native.lib().cm_shared_seed_engine(3000, 1500) in (native.ENGINE_IMMA, native.ENGINE_GF2,
                                                              native.ENGINE_BMMA)


def test_shared_seed_invalid(cm_ctx):
    L = native.lib()
    d = to_dev(np.zeros(8, dtype=np.uint64))
    p = d.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    h = cm_ctx.handle
    assert L.cm_batch_toeplitz_shared_seed(h, p, 0, 5, p, 1, p, 0, s) == native.CM_EINVAL
    assert L.cm_batch_toeplitz_shared_seed(h, p, 5, 5, p, 0, p, 0, s) == native.CM_EINVAL
    assert L.cm_batch_toeplitz_shared_seed(h, p, 5, 5, p, 1, p, 7, s) == native.CM_EINVAL
    assert L.cm_batch_toeplitz_shared_seed(h, p, 1 << 20, 1 << 20, p, 1, p, 0, s) == native.CM_EINVAL


def test_engines_full_count_sampled(cm_ctx):
    # the shared-seed workload at full size: 65536 inputs of 4096 bits under one
    # 2048 x 4096 Toeplitz seed.  The three engines and the auto choice agree on
    # every output bit; 50 inputs against the oracle.
    n, m, count = 4096, 2048, 65536
    wx, wz = native.words(n), native.words(m)
    yw = inputs.bernoulli_half(4096, n + m - 1)
    X = inputs.bernoulli_half(4097, n * count)
    Xd, yd = to_dev(X), to_dev(yw)
    Zg = from_dev(cm_ctx.toeplitz_shared_seed(yd, n, m, Xd, count, engine=native.ENGINE_GF2)).reshape(count, wz)
    Zi = from_dev(cm_ctx.toeplitz_shared_seed(yd, n, m, Xd, count, engine=native.ENGINE_IMMA)).reshape(count, wz)
    Zb = from_dev(cm_ctx.toeplitz_shared_seed(yd, n, m, Xd, count, engine=native.ENGINE_BMMA)).reshape(count, wz)
    Za = from_dev(cm_ctx.toeplitz_shared_seed(yd, n, m, Xd, count)).reshape(count, wz)
    assert (Zg == Zi).all() and (Zg == Zb).all() and (Zg == Za).all()
    picks = [0, count - 1] + np.random.default_rng(4098).choice(count, 48, replace=False).tolist()
    for c in picks:
        assert (Zg[c] == oracle.toeplitz_packed(X[c * wx:(c + 1) * wx], n, yw, m)).all(), c
