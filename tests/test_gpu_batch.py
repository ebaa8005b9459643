"""dl_batch_join: many eps-join and top-k requests of uneven sizes in one call.

Each request's result must equal the FP64 oracle's result for that request
alone, and equal the single-request entry point's result (alone vs in the mix).
"""

import math

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


def _mix(seed, n_req, store_n, d, mu, sigma, qmax):
    g = W.rng(seed)
    S, _ = W.clustered_histograms(g, store_n, d, max(1, store_n // 16), 0.01)
    sid = np.arange(store_n, dtype=np.int64) * 13 + 5
    reqs = W.request_mix(g, n_req, mu, sigma, qmax, topk_frac=0.3, ks=(1, 10, 100))
    nq_total = sum(r["nq"] for r in reqs)
    Q, _ = W.clustered_histograms(g, nq_total, d, max(1, store_n // 16), 0.012)
    qid = np.arange(nq_total, dtype=np.int64) * 3 + 7
    off = 0
    for r in reqs:
        r["q_begin"] = off
        off += r["nq"]
    return S, sid, Q, qid, reqs


def _eps_for(orc, Q, S, sel):
    """eps at the requested selectivity of the request's first query row (test-side calibration)."""
    D = np.sort(orc.dist_block(Q[:1], S)[0])
    i = max(0, min(len(D) - 1, int(sel * len(D))))
    return math.sqrt(D[i]) * (1 + 1e-9)


def test_batch_mixed_requests_match_oracle_and_alone(dl, orc):
    import torch
    S, sid, Q, qid, reqs = _mix(51, 40, 6000, 64, 3.0, 1.2, 300)
    for r in reqs:
        if r["kind"] == "eps":
            r["eps"] = _eps_for(orc, Q[r["q_begin"]:r["q_begin"] + r["nq"]], S, r["selectivity"] * 4)
    reqs.append({"kind": "eps", "q_begin": 5, "nq": 0, "eps": 0.1})            # empty request
    reqs.append({"kind": "topk", "q_begin": 3, "nq": 2, "k": 7})               # overlapping rows
    Ss = dl.Store(torch.from_numpy(sid).cuda(), torch.from_numpy(S).cuda())
    res = dl.batch_join(Ss, qid, Q, reqs)
    st = res.stats()
    for i, r in enumerate(reqs):
        q0, nq = r["q_begin"], r["nq"]
        Qr = Q[q0:q0 + nq]
        if r["kind"] == "eps":
            a, b = res.request_pairs(i)
            got = set(zip(a.tolist(), b.tolist()))
            assert len(got) == len(a)
            p = orc.join(Qr, S, r["eps"], oracle.MODE_RXS) if nq else np.empty((0, 2), np.int64)
            want = set(zip(qid[q0 + p[:, 0]].tolist(), sid[p[:, 1]].tolist()))
            assert got == want, (i, r, len(got ^ want), st)
            if nq and i % 5 == 0:   # alone through the single-request call
                one = dl.sim_join(dl.Store(torch.from_numpy(qid[q0:q0 + nq]).cuda(), torch.from_numpy(Qr).cuda()),
                                  Ss, r["eps"])
                x, y = one.pairs_host()
                one.free()
                assert set(zip(x.tolist(), y.tolist())) == got
        else:
            ids, d2 = res.request_topk(i)
            oi, od = orc.topk(Qr, S, r["k"])
            want = np.where(oi >= 0, sid[np.clip(oi, 0, None)], -1)
            assert (ids == want).all() and (d2 == od).all(), (i, r)
            if i % 3 == 0:
                one = dl.topk_join(dl.Store(torch.from_numpy(qid[q0:q0 + nq]).cuda(),
                                            torch.from_numpy(Qr).cuda()), Ss, r["k"])
                x, y = one.topk_host()
                one.free()
                assert (x == ids).all() and (y == d2).all()
    res.free()


def test_batch_host_inputs_and_rejects(dl):
    import torch
    g = W.rng(52)
    S = W.dirichlet_histograms(g, 500, 32)
    Ss = dl.Store(torch.arange(500, device="cuda"), torch.from_numpy(S).cuda())
    Q = W.dirichlet_histograms(g, 50, 32)
    qid = np.arange(50, dtype=np.int64)
    res = dl.batch_join(Ss, qid, Q, [{"kind": "eps", "q_begin": 0, "nq": 50, "eps": 0.2},
                                     {"kind": "topk", "q_begin": 10, "nq": 20, "k": 4}])
    a, _ = res.request_pairs(0)
    ids, _ = res.request_topk(1)
    assert ids.shape == (20, 4) and (ids >= 0).all() and len(a) > 0
    res.free()
    with pytest.raises(dl.DLError) as ei:
        dl.batch_join(Ss, qid, Q, [{"kind": "eps", "q_begin": 40, "nq": 20, "eps": 0.2}])
    assert ei.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as ei:
        dl.batch_join(Ss, qid, Q, [{"kind": "topk", "q_begin": 0, "nq": 5, "k": 0}])
    assert ei.value.status == dl.DL_EINVAL
