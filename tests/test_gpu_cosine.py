"""The cosine metric (a further metric, on unit-normalized stores) against the oracle.

dl_store_normalize must produce the oracle's normalized rows bit for bit (each row's norm is
a canonical FP64 sum), so every cosine join and top-k equals the oracle's on those rows,
including thresholds placed exactly on a realised distance.
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
    return dl.Store(torch.from_numpy(ids).cuda(), torch.from_numpy(X).cuda())


def _pairs(res):
    a, b = res.pairs_host()
    res.free()
    got = set(zip(a.tolist(), b.tolist()))
    assert len(got) == len(a)
    return got


@pytest.mark.parametrize("kind,d", [("signed", 96), ("signed", 300), ("hist", 64)])
@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
def test_cosine_join_equals_oracle(dl, orc, kind, d, prec):
    g = W.rng(9100 + d)
    if kind == "signed":
        R, c0 = W.unit_mixture(g, 500, d, 40, 0.3)
        S, _ = W.unit_mixture(g, 700, d, 40, 0.3, centroids=c0)
        R = (R * g.uniform(0.5, 4.0, size=(500, 1))).astype(np.float32)   # not unit: the store normalizes
    else:
        R = W.dirichlet_histograms(g, 500, d)
        S = W.dirichlet_histograms(g, 700, d)
    rid = np.arange(500, dtype=np.int64) * 3 + 1
    sid = np.arange(700, dtype=np.int64) * 5 + 2
    Rn, Sn = _store(dl, rid, R).normalized(), _store(dl, sid, S).normalized()
    Ro, So = orc.normalize(R), orc.normalize(S)
    D = orc.dist_block(Ro, So)
    cs = [1.0 - float(np.quantile(D, q)) / 2.0 for q in (0.001, 0.02, 0.2)]
    # a threshold on a realised distance: 2 - 2c equals a canonical D exactly (inclusive)
    t = float(np.sort(D.ravel())[D.size // 50])
    c_on = 1.0 - t / 2.0
    if 2.0 - 2.0 * c_on == t:
        cs.append(c_on)
    for c in cs:
        want = {(int(rid[i]), int(sid[j])) for i, j in orc.cosine_join(Ro, So, c, oracle.MODE_RXS).tolist()}
        got = _pairs(dl.sim_join(Rn, Sn, c, precision=prec, metric="cosine"))
        assert got == want, (prec, c, len(got ^ want))


def test_cosine_self_join_and_topk(dl, orc):
    g = W.rng(9200)
    X, _ = W.unit_mixture(g, 800, 128, 50, 0.25)
    X = (X * g.uniform(0.1, 10.0, size=(800, 1))).astype(np.float32)
    ids = np.arange(800, dtype=np.int64) + 10
    Xn = _store(dl, ids, X).normalized()
    Xo = orc.normalize(X)
    for mode, omode in (("upper", oracle.MODE_SELF_UPPER), ("full", oracle.MODE_SELF_FULL)):
        want = {(int(ids[i]), int(ids[j])) for i, j in orc.cosine_join(Xo, None, 0.9, omode).tolist()}
        assert _pairs(dl.sim_join(Xn, None, 0.9, self_mode=mode, metric="cosine")) == want, mode
    Q = X[:100] * np.float32(0.5)
    Qn = _store(dl, np.arange(100, dtype=np.int64), Q).normalized()
    res = dl.topk_join(Qn, Xn, 10, metric="cosine")
    got_ids, got_d2 = res.topk_host()
    res.free()
    oi, od = orc.topk(orc.normalize(Q), Xo, 10)
    assert np.array_equal(got_ids, ids[oi]) and np.array_equal(got_d2, od)


def test_cosine_rejections(dl):
    import torch
    X = torch.rand(20, 16, device="cuda")
    ids = torch.arange(20, device="cuda")
    S = dl.Store(ids, X)
    with pytest.raises(dl.DLError) as ei:      # not normalized
        dl.sim_join(S, None, 0.5, metric="cosine")
    assert ei.value.status == dl.DL_EINVAL
    Sn = S.normalized()
    with pytest.raises(dl.DLError) as ei:      # threshold outside [-1, 1]
        dl.sim_join(Sn, None, 1.5, metric="cosine")
    assert ei.value.status == dl.DL_EINVAL
    Z = X.clone()
    Z[7] = 0.0
    with pytest.raises(dl.DLError) as ei:      # a zero row has no direction
        dl.Store(ids, Z).normalized()
    assert ei.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as ei:
        dl.topk_join(S, Sn, 3, metric="cosine")
    assert ei.value.status == dl.DL_EINVAL
