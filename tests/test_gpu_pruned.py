"""The exact pruned epsilon-join (tile-pair pruning by bounding balls, Sec. 5 / Sec. 7.3) and
the clustered store order, on the GPU against the oracle.

Pruning must never change the result: every configuration below equals the oracle's
nested loop exactly, whatever the store order (clustered or plain norm order), the
precision, the self-join mode or eps (0, a realised distance, infinity). The full-size
tracked-objects store also checks that pruning actually skips most tile pairs.
"""

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


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_pruned_equals_oracle_small(dl, orc, prec):
    g = W.rng(9600)
    X, _ = W.clustered_histograms(g, 3000, 64, 24, 0.004)
    Y, _ = W.clustered_histograms(W.rng(9601), 1700, 64, 24, 0.004)
    ids = np.arange(3000, dtype=np.int64) * 5 + 3
    yid = np.arange(1700, dtype=np.int64) * 7 + 1
    Xs = _store(dl, ids, X)
    Xc = Xs.clustered(32, iters=3)
    Ys = _store(dl, yid, Y).clustered(16, iters=2)
    D = orc.dist_block(X[:300], X)
    realised = float(np.sort(D[D > 0])[D.size // 200])
    for eps in (0.0, float(np.sqrt(realised)), float(np.sqrt(np.quantile(D[D > 0], 0.01))), float("inf")):
        for mode, om in (("upper", oracle.MODE_SELF_UPPER), ("full", oracle.MODE_SELF_FULL)):
            want = {(int(ids[i]), int(ids[j])) for i, j in orc.join(X, None, eps, om).tolist()}
            for S in (Xc, Xs):
                res = dl.sim_join(S, None, eps, precision=prec, self_mode=mode, prune=True)
                assert _pairs(res) == want, (prec, eps, mode)
        want = {(int(ids[i]), int(yid[j])) for i, j in orc.join(X, Y, eps, oracle.MODE_RXS).tolist()}
        assert _pairs(dl.sim_join(Xc, Ys, eps, precision=prec, prune=True)) == want, (prec, eps)


def test_cluster_store_keeps_rows_and_edges(dl, orc):
    g = W.rng(9700)
    X, _ = W.clustered_histograms(g, 500, 32, 10, 0.01)
    ids = np.arange(500, dtype=np.int64) + 40
    Xs = _store(dl, ids, X)
    eps = float(np.sqrt(np.quantile(orc.dist_block(X[:50], X), 0.05)))
    want = {(int(ids[i]), int(ids[j])) for i, j in orc.join(X, None, eps, oracle.MODE_SELF_UPPER).tolist()}
    for k, it in ((1, 0), (7, 1), (600, 2), (500, 0)):
        Xc = Xs.clustered(k, iters=it)
        assert Xc.n == 500 and Xc.d == 32
        # upper mode writes (lower caller row, higher caller row): the clustered store keeps caller rows
        assert _pairs(dl.sim_join(Xc, None, eps, precision="bf16", prune=True)) == want, (k, it)
        assert _pairs(dl.sim_join(Xc, None, eps, precision="bf16")) == want, (k, it)
    with pytest.raises(dl.DLError):
        Xs.clustered(0)


def test_full_size_tracked_objects(dl, orc):
    wl = W.tracked_objects_262k()
    S = _store(dl, wl.r_ids, wl.R)
    C = S.clustered(1024, iters=5)
    res = dl.sim_join(C, None, wl.eps, precision="bf16", self_mode="full", prune=True, timing=True)
    st = res.stats()
    a, b = res.pairs_host()
    res.free()
    assert st["tile_pairs"] > 0 and st["tile_pairs_kept"] < 0.2 * st["tile_pairs"], st
    dense = dl.sim_join(S, None, wl.eps, precision="bf16", self_mode="full")
    da, db = dense.pairs_host()
    dense.free()
    assert len(a) == len(da)
    key = lambda x, y: np.sort(x.astype(np.int64) * (1 << 40) + y)   # noqa: E731
    assert np.array_equal(key(a, b), key(da, db))
    rows = np.sort(W.rng(9800).choice(wl.R.shape[0], 64, replace=False))
    D = orc.dist_block(wl.R[rows], wl.R)
    e2 = wl.eps * wl.eps
    pos = {int(v): i for i, v in enumerate(wl.r_ids)}
    got = {}
    for x, y in zip(a.tolist(), b.tolist()):
        got.setdefault(pos[x], set()).add(pos[y])
    for i, r in enumerate(rows):
        assert got.get(int(r), set()) == set(np.flatnonzero(D[i] <= e2).tolist()), r
