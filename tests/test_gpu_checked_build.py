"""The bounds-checked build (-DDL_CHECKED) on the GPU.

The checked library guards the computed shared- and global-memory indices of the hot
kernels (the tensor-core join's candidate staging, column data and per-row parameters; the
band recheck's and the batch decision's candidate rows; the top-k finalize's columns). A
failed check skips its access and records (site << 40) | index; nothing traps. This test
builds that library, runs a battery of small joins through it -- BF16, FP8 and exact FP32,
R x S and both self-join modes with ragged tails, an SM-pair join, top-k and a mixed batch --
checks every result against the oracle and requires that no check failed. The recording
itself is shown by a self-test that fails a check of a constant-false condition (guarding no
access). The normal library is restored for the tests that follow.
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
    path = B.build(checked=True)
    D.load(path)
    assert D.check_word() == 0
    yield D
    D.load(D.LIB_PATH)


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def _store(dl, ids, X):
    import torch
    return dl.Store(torch.from_numpy(np.ascontiguousarray(ids)).cuda(),
                    torch.from_numpy(np.ascontiguousarray(X)).cuda())


def _want(orc, R, S, eps, mode, rid, sid):
    p = orc.join(R, S, eps, mode)
    return set(zip(rid[p[:, 0]].tolist(), sid[p[:, 1]].tolist()))


def test_check_recording_selftest(dl):
    assert dl.load().dl_debug_check_selftest(12345) == dl.DL_OK
    assert dl.check_word() == (99 << 40) | 12345
    assert dl.check_word() == 0   # reading clears the record


@pytest.mark.parametrize("nR,nS,d", [(1, 300, 7), (129, 255, 64), (300, 257, 128), (200, 700, 200), (130, 390, 512)])
def test_checked_joins_exact_and_clean(dl, orc, nR, nS, d):
    g = W.rng(9100 + nR + d)
    R = W.dirichlet_histograms(g, nR, d)
    S = W.dirichlet_histograms(g, nS, d)
    eps = math.sqrt(float(np.quantile(orc.dist_block(R, S), 0.02)))
    rid = np.arange(nR, dtype=np.int64) + 1
    sid = np.arange(nS, dtype=np.int64) + (1 << 40)
    Rs, Ss = _store(dl, rid, R), _store(dl, sid, S)
    want = _want(orc, R, S, eps, oracle.MODE_RXS, rid, sid)
    for prec, pair in (("bf16", 1), ("fp8", 1), ("fp32", 0), ("bf16", 2)):
        res = dl.sim_join(Rs, Ss, eps, precision=prec, cta_pair=pair)
        a, b = res.pairs_host()
        res.free()
        assert set(zip(a.tolist(), b.tolist())) == want, (prec, pair)
    for mode, om in (("upper", oracle.MODE_SELF_UPPER), ("full", oracle.MODE_SELF_FULL)):
        res = dl.sim_join(Rs, None, eps, precision="bf16", self_mode=mode)
        a, b = res.pairs_host()
        res.free()
        assert set(zip(a.tolist(), b.tolist())) == _want(orc, R, None, eps, om, rid, rid), mode
    assert dl.check_word() == 0


def test_checked_topk_and_batch_exact_and_clean(dl, orc):
    g = W.rng(9200)
    S = W.dirichlet_histograms(g, 3000, 64)
    Q = W.dirichlet_histograms(g, 333, 64)
    sid = np.arange(3000, dtype=np.int64) * 3
    Ss = _store(dl, sid, S)
    res = dl.topk_join(_store(dl, np.arange(333), Q), Ss, 10, precision="bf16")
    ids, d2 = res.topk_host()
    res.free()
    oi, od = orc.topk(Q, S, 10)
    assert (ids == sid[oi]).all() and (d2 == od).all()
    eps = math.sqrt(float(np.quantile(orc.dist_block(Q[:50], S), 0.01)))
    reqs = [{"kind": "eps", "q_begin": 0, "nq": 200, "eps": eps}, {"kind": "topk", "q_begin": 200, "nq": 133, "k": 5}]
    br = dl.batch_join(Ss, np.arange(333), Q, reqs)
    a, b = br.request_pairs(0)
    p = orc.join(Q[:200], S, eps, oracle.MODE_RXS)
    assert set(zip(a.tolist(), b.tolist())) == set(zip(p[:, 0].tolist(), sid[p[:, 1]].tolist()))
    ids, d2 = br.request_topk(1)
    oi, od = orc.topk(Q[200:], S, 5)
    assert (ids == sid[oi]).all() and (d2 == od).all()
    br.free()
    assert dl.check_word() == 0
