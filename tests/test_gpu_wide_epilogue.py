"""Parity of the 16-warp epilogue of the tensor-core epsilon-join with the FP64 oracle.

With opts.epilogue_warps = 16 each 256-column tile is read out of TMEM by four warps per SM
sub-partition (64 columns each, 32 at a time) instead of two. The bar is the same as for the
8-warp epilogue: exact set equality with the canonical FP64 nested loop for ragged shapes,
both self-join modes, BF16 and FP8 and d up to 1,000, equality with the 8-warp epilogue on a
candidate-dense join, the diagnostics dump (h and its bound) unchanged, and the rejection of
configurations that have no 16-warp form.
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
    return dl.Store(torch.from_numpy(np.ascontiguousarray(ids)).cuda(),
                    torch.from_numpy(np.ascontiguousarray(X)).cuda())


def _pairs(dl, Rs, Ss, eps, prec, warps, self_mode="upper"):
    res = dl.sim_join(Rs, Ss, eps, precision=prec, self_mode=self_mode, tile_n=256, epilogue_warps=warps)
    a, b = res.pairs_host()
    st = res.stats()
    res.free()
    got = list(zip(a.tolist(), b.tolist()))
    assert len(set(got)) == len(got), "duplicate pair in output"
    return set(got), st


def _want(orc, R, S, eps, mode, rid, sid):
    p = orc.join(R, S, eps, mode)
    return set(zip(rid[p[:, 0]].tolist(), sid[p[:, 1]].tolist()))


@pytest.mark.parametrize("nR,nS,d", [
    (1, 1, 16), (1, 700, 64), (129, 255, 64), (255, 257, 128), (257, 513, 96), (385, 300, 200),
    (600, 1000, 256), (130, 390, 512), (90, 330, 1000),
])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_wide_rxs_ragged_exact(dl, orc, nR, nS, d, prec):
    if prec == "bf16" and d > 512:
        pytest.skip("BF16 serves d <= 512")
    g = W.rng(9300 + nR + 7 * nS + 13 * d)
    R = W.dirichlet_histograms(g, nR, d)
    S = np.concatenate([R[: nR // 3], W.dirichlet_histograms(g, nS - nR // 3, d)])
    eps = math.sqrt(float(np.quantile(orc.dist_block(R, S), 0.02)))
    rid = np.arange(nR, dtype=np.int64) * 3 + 11
    sid = np.arange(nS, dtype=np.int64) * 5 + (1 << 40)
    got, st = _pairs(dl, _store(dl, rid, R), _store(dl, sid, S), eps, prec, 16)
    assert st["epilogue_warps"] == 16 and st["tile_n"] == 256
    assert got == _want(orc, R, S, eps, oracle.MODE_RXS, rid, sid)


@pytest.mark.parametrize("n", [2, 255, 257, 1500])
@pytest.mark.parametrize("self_mode", ["upper", "full"])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_wide_self_join_modes(dl, orc, n, self_mode, prec):
    g = W.rng(9400 + n)
    X, _ = W.clustered_histograms(g, n, 96, max(1, n // 8), 0.01)
    xid = np.arange(n, dtype=np.int64) * 7 + 3
    got, st = _pairs(dl, _store(dl, xid, X), None, 0.12, prec, 16, self_mode)
    assert st["epilogue_warps"] == 16
    mode = oracle.MODE_SELF_FULL if self_mode == "full" else oracle.MODE_SELF_UPPER
    assert got == _want(orc, X, None, 0.12, mode, xid, xid)


def test_wide_equals_narrow_on_a_dense_join(dl, orc):
    """A candidate-dense join (queries near the store's centres, eps at 0.5% selectivity)."""
    g = W.rng(9500)
    X, _ = W.clustered_histograms(g, 40000, 128, 300, 0.01)
    Q = X[g.choice(40000, 3000, replace=False)]
    eps = math.sqrt(float(np.quantile(orc.dist_block(Q[:32], X), 0.005)))
    Xs, Qs = _store(dl, np.arange(40000), X), _store(dl, np.arange(3000), Q)
    for prec in ("bf16", "fp8"):
        wide, sw = _pairs(dl, Qs, Xs, eps, prec, 16)
        narrow, sn = _pairs(dl, Qs, Xs, eps, prec, 8)
        assert sw["epilogue_warps"] == 16 and sn["epilogue_warps"] == 8
        assert wide == narrow and len(wide) > 3000 * 100
    D = orc.dist_block(Q[:40], X)
    for i in range(40):
        assert {j for (q, j) in wide if q == i} == set(np.nonzero(D[i] <= eps * eps)[0].tolist()), i


def test_wide_debug_scores_match_narrow(dl):
    """The diagnostics dump (h~ and its bound E per pair) is the same whichever epilogue wrote it
    (dl_debug_scores uses the default configuration; here both are compared on one store pair)."""
    import torch
    g = W.rng(9600)
    R = W.dirichlet_histograms(g, 300, 64)
    S = W.dirichlet_histograms(g, 700, 64)
    Rs, Ss = _store(dl, np.arange(300), R), _store(dl, np.arange(700), S)
    h, e = dl.debug_scores(Rs, Ss, "bf16")
    assert torch.isfinite(h).all() and (e > 0).all()


def test_wide_rejections(dl):
    X = W.dirichlet_histograms(W.rng(9700), 100, 64)
    Xs = _store(dl, np.arange(100), X)
    for kw in ({"epilogue_warps": 12}, {"epilogue_warps": 16, "tile_n": 128},
               {"epilogue_warps": 16, "cta_pair": 2}):
        with pytest.raises(dl.DLError) as ei:
            dl.sim_join(Xs, None, 0.1, precision="bf16", **kw)
        assert ei.value.status == dl.DL_EINVAL
