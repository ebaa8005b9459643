"""The serving loop: continuous batching, admission by memory, polling, cancel.

Requests are submitted one at a time while earlier batches are on the GPU; each
result must equal the FP64 oracle's answer for that request alone.
"""

import math
import threading
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
    return D


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def test_server_results_equal_oracle_alone(dl, orc):
    import torch
    g = W.rng(61)
    S, _ = W.clustered_histograms(g, 8000, 64, 500, 0.01)
    sid = np.arange(8000, dtype=np.int64) * 11 + 2
    Ss = dl.Store(torch.from_numpy(sid).cuda(), torch.from_numpy(S).cuda())
    sv = dl.Server(Ss, mem_budget_bytes=2 << 30, slots=3, max_batch_rows=4096)
    reqs = W.request_mix(g, 60, 3.0, 1.2, 400, topk_frac=0.3, ks=(1, 10, 100))
    pending = []
    for i, r in enumerate(reqs):
        Q, _ = W.clustered_histograms(g, r["nq"], 64, 500, 0.012)
        qid = np.arange(r["nq"], dtype=np.int64) + 1000 * i
        if r["kind"] == "eps":
            D = np.sort(orc.dist_block(Q[:1], S)[0])
            r["eps"] = math.sqrt(D[int(r["selectivity"] * 4 * len(D))]) * (1 + 1e-9)
            t = sv.submit(qid, Q, "eps", eps=r["eps"])
        else:
            t = sv.submit(qid, Q, "topk", k=r["k"])
        pending.append((t, r, Q, qid))
        if i % 7 == 0:
            time.sleep(0.002)   # let batches start while later requests arrive
    for t, r, Q, qid in pending:
        res = None
        for _ in range(600):
            res = sv.poll(t, timeout_us=100_000)
            if res is not None:
                break
        assert res is not None, "request did not finish"
        if r["kind"] == "eps":
            a, b = res.pairs_host()
            p = orc.join(Q, S, r["eps"], oracle.MODE_RXS)
            want = set(zip(qid[p[:, 0]].tolist(), sid[p[:, 1]].tolist()))
            assert set(zip(a.tolist(), b.tolist())) == want and len(a) == len(want)
        else:
            ids, d2 = res.topk_host()
            oi, od = orc.topk(Q, S, r["k"])
            assert (ids == sid[oi]).all() and (d2 == od).all()
        res.free()
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert st["batches"] >= 2
    sv.close()


def test_server_admission_and_cancel(dl):
    import torch
    g = W.rng(62)
    S = W.dirichlet_histograms(g, 3000, 32)
    Ss = dl.Store(torch.arange(3000, device="cuda"), torch.from_numpy(S).cuda())
    sv = dl.Server(Ss, mem_budget_bytes=64 << 20, slots=1, max_batch_rows=2000)
    Q = W.dirichlet_histograms(g, 3000, 32)
    with pytest.raises(dl.DLError) as ei:          # more rows than a batch may hold
        sv.submit(np.arange(3000), Q, "eps", eps=0.1)
    assert ei.value.status == dl.DL_ENOMEM_ADMIT
    with pytest.raises(dl.DLError) as ei:          # can never fit the memory budget
        sv.submit(np.arange(1500), Q[:1500], "topk", k=1000)
    assert ei.value.status == dl.DL_ENOMEM_ADMIT
    with pytest.raises(dl.DLError) as ei:
        sv.submit(np.arange(5), Q[:5], "eps", eps=-1.0)
    assert ei.value.status == dl.DL_EINVAL
    tickets = [sv.submit(np.arange(1500), Q[:1500], "eps", eps=0.15) for _ in range(4)]
    last = tickets[-1]
    rc = sv.cancel(last)
    if rc == dl.DL_OK:
        st, res = sv.poll_status(last, 0)
        assert st == dl.DL_ECANCELED and res is None
    else:
        assert rc == dl.DL_EAGAIN
    for t in tickets[:-1]:
        for _ in range(600):
            res = sv.poll(t, timeout_us=100_000)
            if res is not None:
                break
        assert res is not None and res.count() > 0
        res.free()
    sv.close()
