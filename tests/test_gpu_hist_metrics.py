"""L1 and chi-square histogram joins (a further metric family) on the GPU against the oracle.

Exact set equality with the canonical FP64 nested loop, including thresholds placed
exactly on a realised distance, histograms with exact zero bins (chi-square skips
bins where both are zero), both self-join modes, ragged sizes, a 256-row sample of a
65,536-row clustered store, and the rejections (tensor-core precisions, negative
features for chi-square).
"""

import numpy as np
import pytest

import oracle
from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MET = {"l1": oracle.METRIC_L1, "chi2": oracle.METRIC_CHI2}


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
    return dl.Store(torch.from_numpy(np.ascontiguousarray(ids)).cuda(),
                    torch.from_numpy(np.ascontiguousarray(X)).cuda())


def _pairs(res):
    a, b = res.pairs_host()
    res.free()
    got = set(zip(a.tolist(), b.tolist()))
    assert len(got) == len(a)
    return got


def _data(kind, g, n, d):
    if kind == "dirichlet":
        return W.dirichlet_histograms(g, n, d)
    if kind == "clustered":        # clipped jitter: many exact zeros
        return W.clustered_histograms(g, n, d, max(1, n // 16), 0.02)[0]
    return np.abs(W.mixed_magnitude_rows(g, n, d)).astype(np.float32)


@pytest.mark.parametrize("metric", ["l1", "chi2"])
@pytest.mark.parametrize("kind,nR,nS,d", [("dirichlet", 300, 257, 64), ("clustered", 129, 400, 128),
                                          ("mixed", 90, 130, 33), ("clustered", 1, 1000, 7),
                                          ("dirichlet", 255, 1, 300)])
def test_rxs_equals_oracle(dl, orc, metric, kind, nR, nS, d):
    g = W.rng(8100 + nR + d)
    R, S = _data(kind, g, nR, d), _data(kind, g, nS, d)
    rid = np.arange(nR, dtype=np.int64) * 3 + 5
    sid = np.arange(nS, dtype=np.int64) * 7 + 1
    Rs, Ss = _store(dl, rid, R), _store(dl, sid, S)
    D = orc.hist_dist_block(R, S, MET[metric])
    flat = np.sort(D.ravel())
    thrs = [float(np.quantile(flat, q)) for q in (0.0005, 0.01, 0.3)]
    thrs += [float(flat[min(len(flat) - 1, len(flat) // 40)])]     # exactly a realised distance
    for t in thrs:
        want = {(int(rid[i]), int(sid[j])) for i, j in orc.hist_join(R, S, t, MET[metric], oracle.MODE_RXS).tolist()}
        for prec in ("auto", "fp32"):
            got = _pairs(dl.sim_join(Rs, Ss, t, precision=prec, metric=metric))
            assert got == want, (metric, kind, t, prec, len(got ^ want))
    dl.sim_join(Rs, Ss, thrs[1], precision="fp32_plain", metric=metric).free()


@pytest.mark.parametrize("metric", ["l1", "chi2"])
def test_self_join_modes(dl, orc, metric):
    g = W.rng(8200)
    X = W.clustered_histograms(g, 700, 96, 40, 0.01)[0]
    ids = np.arange(700, dtype=np.int64) + 100
    Xs = _store(dl, ids, X)
    D = orc.hist_dist_block(X[:100], X, MET[metric])
    t = float(np.quantile(D[D > 0], 0.02))
    for mode, om in (("upper", oracle.MODE_SELF_UPPER), ("full", oracle.MODE_SELF_FULL)):
        want = {(int(ids[i]), int(ids[j])) for i, j in orc.hist_join(X, None, t, MET[metric], om).tolist()}
        assert _pairs(dl.sim_join(Xs, None, t, self_mode=mode, metric=metric)) == want, mode


@pytest.mark.parametrize("metric", ["l1", "chi2"])
def test_sampled_rows_of_the_64k_bench_store(dl, orc, metric):
    """The benchmark's hist_clustered_64k self-join at its calibrated threshold, in the launch
    the benchmark times, with 256 sampled rows against the oracle over the whole store."""
    X, thr = W.hist_clustered_64k()
    t = thr[metric]
    g = W.rng(8300)
    ids = np.arange(65536, dtype=np.int64)
    rows = np.sort(g.choice(65536, 256, replace=False))
    D = orc.hist_dist_block(X[rows], X, MET[metric])
    D[np.arange(256), rows] = np.inf
    Xs = _store(dl, ids, X)
    a, b = dl.sim_join(Xs, None, t, self_mode="full", metric=metric).pairs_host()
    sel = np.isin(a, rows) & (a != b)
    got = set(zip(a[sel].tolist(), b[sel].tolist()))
    want = {(int(rows[i]), int(j)) for i, j in zip(*np.nonzero(D <= t))}
    assert got == want, (metric, len(got ^ want))


def test_rejections(dl):
    g = W.rng(8400)
    X = W.dirichlet_histograms(g, 50, 16)
    Xs = _store(dl, np.arange(50), X)
    for prec in ("bf16", "fp8"):
        with pytest.raises(dl.DLError) as ei:
            dl.sim_join(Xs, None, 0.5, precision=prec, metric="l1")
        assert ei.value.status == dl.DL_EUNSUPPORTED
    with pytest.raises(dl.DLError) as ei:
        dl.sim_join(Xs, None, -1.0, metric="chi2")
    assert ei.value.status == dl.DL_EINVAL
    Y = X.copy()
    Y[3, 2] = -1e-3
    Ys = _store(dl, np.arange(50), Y)
    with pytest.raises(dl.DLError) as ei:
        dl.sim_join(Ys, None, 0.5, metric="chi2")
    assert ei.value.status == dl.DL_EINVAL
    dl.sim_join(Ys, None, 0.5, metric="l1").free()      # L1 takes signed features
    dl.topk_join(Xs, Xs, 3, metric="l1").free()   # served by the histogram top-k (test_gpu_hist_topk.py)
    with pytest.raises(dl.DLError) as ei:
        dl.topk_join(Ys, Xs, 3, metric="chi2")
    assert ei.value.status == dl.DL_EINVAL
