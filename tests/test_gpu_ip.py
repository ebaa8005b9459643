"""Parity of the inner-product threshold join (DL_METRIC_IP) with the FP64 oracle.

A pair matches iff its canonical FP64 dot product (k ascending, exact products, every addition
rounded to nearest) is >= t (Sec. 3.2: threshold the similarity). The GPU screens pairs on the
BF16 tensor cores with a bound that includes the canonical dot's own error, then settles the
band with an FP32 dot and its bound, else the canonical FP64 dot. The bar is exact set
equality with the oracle: rows of very different norms, signed and non-negative features,
ragged shapes, thresholds at quantiles, at a realised canonical dot (a tie, which matches) and
one ulp above it, near-copies that put many pairs in the band, -inf and +inf, the upper
self-join, and the modes the path refuses.
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


def _store(dl, ids, X):
    import torch
    return dl.Store(torch.from_numpy(np.ascontiguousarray(ids)).cuda(), torch.from_numpy(np.ascontiguousarray(X)).cuda())


def _rows(g, n, d, spread=3.0):
    """Signed rows whose norms span 2^-spread .. 2^spread."""
    X = g.standard_normal((n, d))
    X *= 2.0 ** g.uniform(-spread, spread, (n, 1))
    return X.astype(np.float32)


def _gpu(dl, R, S, t, rid, sid, **kw):
    res = dl.sim_join(_store(dl, rid, R), None if S is None else _store(dl, sid, S), t, metric="ip", **kw)
    a, b = res.pairs_host()
    st = res.stats()
    res.free()
    got = list(zip(a.tolist(), b.tolist()))
    assert len(set(got)) == len(got), "duplicate pair in output"
    return set(got), st


def _want(orc, R, S, t, mode, rid, sid):
    p = orc.ip_join(R, S, t, mode)
    return set(zip(rid[p[:, 0]].tolist(), sid[p[:, 1]].tolist()))


@pytest.mark.parametrize("nR,nS,d", [(1, 1, 4), (129, 257, 16), (300, 700, 64), (257, 513, 128), (200, 300, 200),
                                     (130, 390, 512)])
@pytest.mark.parametrize("q", [0.5, 0.99, 0.999])
def test_ip_rxs_quantiles_exact(dl, orc, nR, nS, d, q):
    g = W.rng(9000 + nR + 3 * nS + 7 * d)
    R, S = _rows(g, nR, d), _rows(g, nS, d)
    t = float(np.quantile(R.astype(np.float64) @ S.astype(np.float64).T, q))
    rid = np.arange(nR, dtype=np.int64) * 3 + 1
    sid = np.arange(nS, dtype=np.int64) + (1 << 35)
    got, st = _gpu(dl, R, S, t, rid, sid)
    assert got == _want(orc, R, S, t, oracle.MODE_RXS, rid, sid)


def test_ip_tie_and_one_ulp_above(dl, orc):
    g = W.rng(9100)
    R, S = _rows(g, 150, 96, 2.0), _rows(g, 220, 96, 2.0)
    rid, sid = np.arange(150, dtype=np.int64), np.arange(220, dtype=np.int64) + 10_000
    for i, j in ((3, 7), (140, 219), (0, 0)):
        t = orc.dot(R[i], S[j])
        got, _ = _gpu(dl, R, S, t, rid, sid)
        want = _want(orc, R, S, t, oracle.MODE_RXS, rid, sid)
        assert got == want and (int(rid[i]), int(sid[j])) in got
        t1 = float(np.nextafter(t, math.inf))
        got1, _ = _gpu(dl, R, S, t1, rid, sid)
        assert got1 == _want(orc, R, S, t1, oracle.MODE_RXS, rid, sid)
        assert (int(rid[i]), int(sid[j])) not in got1


def test_ip_band_heavy_near_copies(dl, orc):
    """S holds near-copies of R's rows, and t sits among their squared norms, so many pairs fall
    in the BF16 band and the FP32 / FP64 stages decide them."""
    g = W.rng(9200)
    R = _rows(g, 600, 64, 0.5)
    S = (R * (1.0 + 1e-4 * g.standard_normal(R.shape))).astype(np.float32)
    t = float(np.median(np.einsum("ij,ij->i", R.astype(np.float64), S.astype(np.float64))))
    rid, sid = np.arange(600, dtype=np.int64) * 2, np.arange(600, dtype=np.int64) * 2 + 1
    got, st = _gpu(dl, R, S, t, rid, sid)
    assert got == _want(orc, R, S, t, oracle.MODE_RXS, rid, sid)
    assert st["band_pairs"] > 0


def test_ip_nonnegative_histograms(dl, orc):
    g = W.rng(9300)
    R, S = W.dirichlet_histograms(g, 400, 128), W.dirichlet_histograms(g, 900, 128)
    t = float(np.quantile(R.astype(np.float64) @ S.astype(np.float64).T, 0.995))
    rid, sid = np.arange(400, dtype=np.int64) + 5, np.arange(900, dtype=np.int64) + 5_000
    got, _ = _gpu(dl, R, S, t, rid, sid)
    assert got == _want(orc, R, S, t, oracle.MODE_RXS, rid, sid)


@pytest.mark.parametrize("n", [2, 255, 700])
def test_ip_self_upper_exact(dl, orc, n):
    g = W.rng(9400 + n)
    X = _rows(g, n, 72)
    t = float(np.quantile(X.astype(np.float64) @ X.astype(np.float64).T, 0.98))
    xid = np.arange(n, dtype=np.int64) * 7 + 2
    got, _ = _gpu(dl, X, None, t, xid, xid, self_mode="upper")
    assert got == _want(orc, X, None, t, oracle.MODE_SELF_UPPER, xid, xid)


def test_ip_infinite_thresholds(dl, orc):
    g = W.rng(9500)
    R, S = _rows(g, 40, 32), _rows(g, 70, 32)
    rid, sid = np.arange(40, dtype=np.int64), np.arange(70, dtype=np.int64) + 100
    got, _ = _gpu(dl, R, S, -math.inf, rid, sid)
    assert len(got) == 40 * 70
    got, _ = _gpu(dl, R, S, math.inf, rid, sid)
    assert got == set()


def test_ip_refusals(dl):
    g = W.rng(9600)
    X = _rows(g, 50, 32)
    Xs = _store(dl, np.arange(50), X)
    for kw in ({"precision": "fp32"}, {"precision": "fp8"}, {"self_mode": "full"}, {"prune": True}):
        with pytest.raises(dl.DLError) as ei:
            dl.sim_join(Xs, None, 0.5, metric="ip", **kw)
        assert ei.value.status == dl.DL_EUNSUPPORTED, kw
    with pytest.raises(dl.DLError) as ei:
        dl.sim_join(Xs, None, math.nan, metric="ip")
    assert ei.value.status == dl.DL_EINVAL
