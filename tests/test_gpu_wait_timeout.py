"""Failure detection on the GPU: a bounded device wait made to run out.

Every pipeline wait of the tensor-core kernels has a clock budget. When it runs
out, the kernel raises its abort flag, lets its copies in flight land, finishes
the MMAs it issued, frees its tensor memory and returns; the entry point turns
the kernel's error word into DL_ETIMEOUT, and the server marks the batch's
requests DL_EFAILED so they can be resubmitted. Here the budget is shortened to
one clock (dl_debug_set_wait_budget), so a healthy join's first wait runs out:
no fault, no trap, no unbounded spin. Each failure is followed by the same call
with the default budget in the same process, which must return the oracle's
exact answer (the context stays usable).
"""

import math
import time

import numpy as np
import pytest

import oracle
from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import torch
    from paper_1812_07607_gb300 import build as B, dl as D
    assert torch.cuda.is_available()
    B.build()
    D.load()
    yield D
    D.set_wait_budget(0)


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.fixture(scope="module")
def data(dl):
    import torch
    wl = W.rxs_histograms_2k()
    Rs = dl.Store(torch.from_numpy(wl.r_ids).cuda(), torch.from_numpy(wl.R).cuda())
    Ss = dl.Store(torch.from_numpy(wl.s_ids).cuda(), torch.from_numpy(wl.S).cuda())
    return wl, Rs, Ss


def _want(orc, wl):
    p = orc.join(wl.R, wl.S, wl.eps, oracle.MODE_RXS)
    return set(zip(wl.r_ids[p[:, 0]].tolist(), wl.s_ids[p[:, 1]].tolist()))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_eps_join_wait_expires_then_exact(dl, orc, data, prec):
    wl, Rs, Ss = data
    dl.set_wait_budget(1)
    try:
        with pytest.raises(dl.DLError) as ei:
            dl.sim_join(Rs, Ss, wl.eps, precision=prec)
        assert ei.value.status == dl.DL_ETIMEOUT
        assert "bounded device wait" in dl.last_error()
    finally:
        dl.set_wait_budget(0)
    res = dl.sim_join(Rs, Ss, wl.eps, precision=prec)
    a, b = res.pairs_host()
    res.free()
    assert set(zip(a.tolist(), b.tolist())) == _want(orc, wl) and len(a) == len(_want(orc, wl))


def test_topk_and_batch_wait_expires_then_exact(dl, orc, data):
    import torch
    wl, Rs, Ss = data
    Q = wl.R[:300]
    Qs = dl.Store(torch.from_numpy(wl.r_ids[:300]).cuda(), torch.from_numpy(Q).cuda())
    reqs = [{"kind": "eps", "q_begin": 0, "nq": 200, "eps": wl.eps},
            {"kind": "topk", "q_begin": 200, "nq": 100, "k": 10}]
    dl.set_wait_budget(1)
    try:
        with pytest.raises(dl.DLError) as ei:
            dl.topk_join(Qs, Ss, 10, precision="bf16")
        assert ei.value.status == dl.DL_ETIMEOUT
        with pytest.raises(dl.DLError) as ei:
            dl.batch_join(Ss, wl.r_ids[:300], Q, reqs)
        assert ei.value.status == dl.DL_ETIMEOUT
    finally:
        dl.set_wait_budget(0)
    res = dl.topk_join(Qs, Ss, 10, precision="bf16")
    ids, d2 = res.topk_host()
    res.free()
    oi, od = orc.topk(Q, wl.S, 10)
    assert (ids == wl.s_ids[oi]).all() and (d2 == od).all()
    br = dl.batch_join(Ss, wl.r_ids[:300], Q, reqs)
    a, b = br.request_pairs(0)
    p = orc.join(Q[:200], wl.S, wl.eps, oracle.MODE_RXS)
    assert set(zip(a.tolist(), b.tolist())) == set(zip(wl.r_ids[p[:, 0]].tolist(), wl.s_ids[p[:, 1]].tolist()))
    ids, d2 = br.request_topk(1)
    oi, od = orc.topk(Q[200:], wl.S, 10)
    assert (ids == wl.s_ids[oi]).all() and (d2 == od).all()
    br.free()


def test_server_marks_failed_then_resubmit_exact(dl, orc, data):
    wl, _, Ss = data
    sv = dl.Server(Ss, mem_budget_bytes=1 << 30, slots=2, max_batch_rows=4096)
    Q, qid = wl.R[:150], wl.r_ids[:150]

    def finish(t):
        for _ in range(600):
            rc, res = sv.poll_status(t, timeout_us=100_000)
            if rc not in (dl.DL_EAGAIN, dl.DL_ETIMEOUT):
                return rc, res
        raise AssertionError("request did not finish")

    dl.set_wait_budget(1)
    try:
        tickets = [sv.submit(qid, Q, "eps", eps=wl.eps), sv.submit(qid, Q, "topk", k=5)]
        outcomes = [finish(t) for t in tickets]
    finally:
        dl.set_wait_budget(0)
    for rc, res in outcomes:
        assert rc == dl.DL_EFAILED and res is None
    assert sv.stats()["failed"] == 2
    rc, res = finish(sv.submit(qid, Q, "eps", eps=wl.eps))
    assert rc == dl.DL_OK
    a, b = res.pairs_host()
    res.free()
    p = orc.join(Q, wl.S, wl.eps, oracle.MODE_RXS)
    assert set(zip(a.tolist(), b.tolist())) == set(zip(qid[p[:, 0]].tolist(), wl.s_ids[p[:, 1]].tolist()))
    rc, res = finish(sv.submit(qid, Q, "topk", k=5))
    assert rc == dl.DL_OK
    ids, d2 = res.topk_host()
    res.free()
    oi, od = orc.topk(Q, wl.S, 5)
    assert (ids == wl.s_ids[oi]).all() and (d2 == od).all()
    sv.close()
