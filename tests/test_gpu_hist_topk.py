"""Parity of the top-k join under the L1 and chi-square histogram distances with the FP64 oracle.

For every query row, the k store rows with the smallest canonical distance (k ascending, every
operation rounded to nearest), ordered by (distance, caller's store row); unused slots are -1.
The bar is bit-exact ids and distances against `oracle.hist_topk` (Sec. 6.2 q1 with the
colour-histogram distances of Sec. 4.1): Dirichlet histograms, clustered histograms with exact
duplicates (ties broken by the store row), a store smaller than k, ragged d, and the refusals.
"""

import numpy as np
import pytest

import oracle
from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu

METRICS = {"l1": oracle.METRIC_L1, "chi2": oracle.METRIC_CHI2}


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


def _store(dl, ids, X):
    import torch
    return dl.Store(torch.from_numpy(np.ascontiguousarray(ids)).cuda(), torch.from_numpy(np.ascontiguousarray(X)).cuda())


def check(dl, orc, Q, S, k, metric):
    qid = np.arange(Q.shape[0], dtype=np.int64) * 3 + 1
    sid = np.arange(S.shape[0], dtype=np.int64) * 5 + 1_000_000
    res = dl.topk_join(_store(dl, qid, Q), _store(dl, sid, S), k, metric=metric)
    ids, dist = res.topk_host()
    res.free()
    oi, od = orc.hist_topk(Q, S, k, METRICS[metric])
    want = np.where(oi >= 0, sid[np.clip(oi, 0, None)], -1)
    bad = np.nonzero((ids != want).any(axis=1) | (dist != od).any(axis=1))[0]
    assert bad.size == 0, (metric, k, bad[:5].tolist(), ids[bad[0]][:6].tolist(), want[bad[0]][:6].tolist())


@pytest.mark.parametrize("metric", ["l1", "chi2"])
@pytest.mark.parametrize("nQ,nS,d,k", [(1, 1, 1, 1), (5, 3, 7, 4), (64, 500, 32, 1), (129, 1000, 128, 10),
                                       (40, 2000, 64, 100), (33, 300, 200, 17)])
def test_hist_topk_exact(dl, orc, metric, nQ, nS, d, k):
    g = W.rng(9700 + nQ + nS + d + k)
    check(dl, orc, W.dirichlet_histograms(g, nQ, d), W.dirichlet_histograms(g, nS, d), k, metric)


@pytest.mark.parametrize("metric", ["l1", "chi2"])
def test_hist_topk_duplicates_tie_by_store_row(dl, orc, metric):
    g = W.rng(9800)
    X, _ = W.clustered_histograms(g, 1500, 64, 100, 0.01)
    S = np.concatenate([X, X[:400]])   # exact duplicates: equal distances, ranked by store row
    check(dl, orc, X[:200], S, 12, metric)


def test_hist_topk_refusals(dl):
    g = W.rng(9900)
    X = W.dirichlet_histograms(g, 50, 16)
    Xs = _store(dl, np.arange(50), X)
    with pytest.raises(dl.DLError) as ei:
        dl.topk_join(Xs, Xs, 5, precision="bf16", metric="l1")
    assert ei.value.status == dl.DL_EUNSUPPORTED
    Y = X.copy()
    Y[3, 2] = -0.25
    Ys = _store(dl, np.arange(50), Y)
    with pytest.raises(dl.DLError) as ei:
        dl.topk_join(Ys, Xs, 5, metric="chi2")
    assert ei.value.status == dl.DL_EINVAL
