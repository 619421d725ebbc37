"""The continuous-batching server (cm_submit / cm_poll) on the GPU.

Each result must equal what the same extraction gives alone (the single call)
and the oracle, whatever else shares its wave; admission respects the HBM
budget; the queue, poll timeout and unknown-ticket paths return their codes.
"""

import threading
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


def make(kind, n, m, s0, const_x=None):
    if const_x is None:
        xw = inputs.bernoulli_half(s0, n)
        if kind == D:
            xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    else:
        xw = ex.pack_bits(np.full(n, const_x, dtype=np.uint8))
    yw = inputs.bernoulli_half(s0 + 1, ybits(kind, n, m))
    z = torch.full((native.words(m),), -1, dtype=torch.int64, device="cuda")
    return dict(kind=kind, n=n, m=m, xw=xw, yw=yw, x=to_dev(xw), y=to_dev(yw), z=z)


def alone(ctx, r):
    k, n, m, x, y = r["kind"], r["n"], r["m"], r["x"], r["y"]
    if k == T:
        return ctx.toeplitz(x, n, y, m)
    if k == C:
        return ctx.circulant(x, n, y, m)
    return ctx.dodis(x, y, n, m)


@pytest.fixture
def sctx():
    ctx = native.Context(0)
    yield ctx
    ctx.close()


def submit(ctx, r):
    return ctx.submit(r["kind"], r["n"], r["m"], r["x"], r["y"], r["z"])


def wait(ctx, t, timeout=60.0):
    s, res = ctx.poll(t, timeout)
    assert s == native.CM_OK, native.STATUS.get(s)
    return res


def test_server_mix_same_alone_and_in_mix(sctx, cm_ctx):
    P = [oracle.next_na(v) for v in (300, 5000, 40000, 200000)]
    specs = []
    rng = np.random.default_rng(4)
    for j in range(36):
        kind = (T, T, C, D)[j % 4]
        if kind == T:
            n = int(2 ** rng.uniform(8, 20))
            specs.append((T, n, max(1, n // 2)))
        elif kind == C:
            p = P[j % 4]
            specs.append((C, p - 1, (p - 1) // 2))
        else:
            p = P[(j // 4) % 4]
            specs.append((D, p, (2 * p) // 5))
    specs.append((T, 2 ** 25, 2 ** 24))   # two column passes: the single-call kernels inside a wave
    reqs = [make(k, n, m, 300 + 10 * j) for j, (k, n, m) in enumerate(specs)]
    sctx.server_start(slots=2)
    tickets = [None] * len(reqs)

    def client():
        # Poisson-like arrivals so that requests arrive while others run
        for j, r in enumerate(reqs):
            tickets[j] = submit(sctx, r)
            time.sleep(float(rng.exponential(0.0004)))

    th = threading.Thread(target=client)
    th.start()
    th.join()
    results = [wait(sctx, t) for t in tickets]
    torch.cuda.synchronize()
    st = sctx.server_stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0
    assert st["waves"] >= 2
    for r, res in zip(reqs, results):
        assert res["status"] == native.CM_OK
        assert res["t_submit_ns"] <= res["t_admit_ns"] <= res["t_done_ns"]
        assert torch.equal(r["z"], alone(cm_ctx, r)), (r["kind"], r["n"], r["m"])
    for r in reqs[:12]:
        k, n, m = r["kind"], r["n"], r["m"]
        want = {T: lambda: oracle.toeplitz_packed(r["xw"], n, r["yw"], m),
                C: lambda: oracle.circulant_packed(r["xw"], n, r["yw"], m),
                D: lambda: oracle.dodis_packed(r["xw"], r["yw"], n, m)}[k]()
        assert (from_dev(r["z"]) == want).all()
    sctx.server_stop()


def test_server_admission_by_footprint(sctx, cm_ctx):
    # L = 2^20 needs 8 MiB of transform scratch (two operands of 32-bit field
    # elements) + window bytes; a 40 MiB budget fits four at a time
    budget = 40 << 20
    sctx.server_start(hbm_budget_bytes=budget, slots=3)
    reqs = [make(T, 600000, 300000, 700 + 3 * j) for j in range(8)]
    tickets = [submit(sctx, r) for r in reqs]
    for t in tickets:
        assert wait(sctx, t)["status"] == native.CM_OK
    st = sctx.server_stats()
    assert 0 < st["max_inflight_bytes"] <= budget
    for r in reqs:
        assert torch.equal(r["z"], alone(cm_ctx, r))
    # L = 2^23 alone needs 64 MiB: the single-call planner splits it into
    # summed blocks that fit the budget
    big = make(T, 2 ** 22, 2 ** 22, 999)
    assert wait(sctx, submit(sctx, big))["status"] == native.CM_OK
    assert sctx.server_stats()["max_inflight_bytes"] <= budget
    assert torch.equal(big["z"], alone(cm_ctx, big))
    sctx.server_stop()
    # nothing fits 64 KiB: refused at submission
    sctx.server_start(hbm_budget_bytes=64 << 10, slots=1)
    s, _ = sctx.submit_raw(T, big["n"], big["m"], big["x"].data_ptr(), big["y"].data_ptr(), big["z"].data_ptr())
    assert s == native.CM_ENOMEM
    sctx.server_stop()


def test_server_express_slot(sctx, cm_ctx):
    # one normal stream: a long request holds it; short requests that arrive
    # meanwhile finish first through the express slot (high stream priority),
    # and without it they wait behind the long one (queued on its stream)
    big = make(T, 2 ** 26, 2 ** 25, 801)     # L = 2^27: milliseconds
    smalls = [make(T, 3000 + 100 * j, 1500, 810 + 2 * j) for j in range(6)]
    for express in (0, native.SERVER_NO_EXPRESS):
        sctx.server_start(slots=1, express_slots=express)
        tb = submit(sctx, big)
        time.sleep(0.002)
        ts = [submit(sctx, r) for r in smalls]
        rs = [wait(sctx, t) for t in ts]
        rb = wait(sctx, tb)
        assert rb["status"] == native.CM_OK and all(r["status"] == native.CM_OK for r in rs)
        if express == 0:
            assert all(r["t_done_ns"] < rb["t_done_ns"] for r in rs)
        else:
            assert all(r["t_done_ns"] >= rb["t_done_ns"] for r in rs)
        st = sctx.server_stats()
        assert st["slots"] == (3 if express == 0 else 2)   # two wave slots on the stream, and the express one
        sctx.server_stop()
        for r in smalls + [big]:
            assert torch.equal(r["z"], alone(cm_ctx, r))


def test_server_queue_full_poll_timeout_unknown(sctx):
    a = make(T, 2 ** 25, 2 ** 25, 41)     # L = 2^26: about 0.5 GiB of scratch, over a millisecond
    b = make(T, 2 ** 25, 2 ** 25, 43)
    c = make(T, 1000, 500, 45)
    one = native.plan_query(T, 2 ** 25, 2 ** 25)["scratch_bytes"]
    foot = one + 4096                     # room for one of them (the planner keeps one product)
    assert native.plan_query(T, 2 ** 25, 2 ** 25, hbm_budget_bytes=foot)["scratch_bytes"] == one
    sctx.server_start(hbm_budget_bytes=foot, slots=2, max_queue=1)
    ta = submit(sctx, a)                  # admitted at once
    time.sleep(0.0005)
    tb = submit(sctx, b)                  # waits for a's memory: the queue holds it
    s, _ = sctx.submit_raw(T, c["n"], c["m"], c["x"].data_ptr(), c["y"].data_ptr(), c["z"].data_ptr())
    assert s == native.CM_EAGAIN          # queue full
    s, _ = sctx.poll(tb, 0.0)
    assert s == native.CM_EAGAIN          # not done yet
    assert sctx.poll(987654321, 0.0)[0] == native.CM_ENOTFOUND
    assert wait(sctx, ta)["status"] == native.CM_OK
    res_b = wait(sctx, tb)
    assert res_b["status"] == native.CM_OK and res_b["wave"] != 0
    assert sctx.poll(ta, 0.0)[0] == native.CM_ENOTFOUND   # collected once
    sctx.server_stop()
    assert sctx._L.cm_submit(sctx.handle, None, None) == native.CM_EINVAL


def test_server_dodis_precondition_per_request(sctx, cm_ctx):
    # work-list requests and, past the work list's 2^25 (P about 2^25 + 2^24:
    # the single-call planner inside the wave), requests of both paths
    P, Q, B = oracle.next_na(70000), oracle.next_na(700), oracle.next_na(3 << 24)
    reqs = [make(D, P, P // 2, 51, const_x=1), make(D, Q, Q // 2, 53, const_x=0),
            make(D, P, P // 3, 55), make(T, 5000, 2500, 57),
            make(D, B, B // 2, 59, const_x=0), make(D, B, B // 3, 61)]
    assert native.plan_query(D, B, B // 2)["transform_length"] > 2 ** 25 or \
        native.plan_query(D, B, B // 2)["products"] > 1
    sctx.server_start()
    tickets = [submit(sctx, r) for r in reqs]
    res = [wait(sctx, t) for t in tickets]
    assert [r["status"] for r in res] == [native.CM_EPRECOND, native.CM_EPRECOND, native.CM_OK, native.CM_OK,
                                           native.CM_EPRECOND, native.CM_OK]
    assert not from_dev(reqs[0]["z"]).any() and not from_dev(reqs[1]["z"]).any()
    assert not from_dev(reqs[4]["z"]).any()
    for r in reqs[2:4] + reqs[5:]:
        assert torch.equal(r["z"], alone(cm_ctx, r))
    sctx.server_stop()


def test_server_seed_transform_resident(sctx, cm_ctx):
    # several inputs under one seed: the seed's transform is computed once and
    # reused; every output still equals its single call
    sctx.server_start(seed_cache_bytes=1 << 30)
    P = oracle.next_na(200000)
    groups = [(T, 150000, 60000), (C, P - 1, (P - 1) // 2), (D, P, P // 3)]
    reqs = []
    for g, (k, n, m) in enumerate(groups):
        base = make(k, n, m, 1000 + 100 * g)
        for j in range(4):
            r = make(k, n, m, 1000 + 100 * g + 2 * j + 2)
            r["y"], r["yw"] = base["y"], base["yw"]
            reqs.append((r, 77 + g))
    first = [sctx.submit(r["kind"], r["n"], r["m"], r["x"], r["y"], r["z"], seed_id=sid)
             for r, sid in reqs[::4]]
    for t in first:
        assert wait(sctx, t)["status"] == native.CM_OK
    rest = [sctx.submit(r["kind"], r["n"], r["m"], r["x"], r["y"], r["z"], seed_id=sid)
            for i, (r, sid) in enumerate(reqs) if i % 4]
    for t in rest:
        assert wait(sctx, t)["status"] == native.CM_OK
    st = sctx.server_stats()
    assert st["seed_cache_misses"] == 3 and st["seed_cache_hits"] == 9 and st["seed_cache_entries"] == 3
    for r, _ in reqs:
        assert torch.equal(r["z"], alone(cm_ctx, r)), (r["kind"], r["n"])
    r0 = reqs[0][0]
    assert (from_dev(r0["z"]) == oracle.toeplitz_packed(r0["xw"], r0["n"], r0["yw"], r0["m"])).all()
    sctx.server_stop()
