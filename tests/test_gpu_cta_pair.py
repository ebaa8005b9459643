"""Parity of the SM-pair tensor-core join (tcgen05 cta_group::2) with the FP64 oracle.

With opts.cta_pair = 2 two SMs compute each 256-row tile: each loads its own 128 rows
of R and its own half of every S tile, one issues the M = 256 MMAs for both, and each
runs the epilogue on its own rows. The bar is the same as for the single-SM kernel:
exact set equality with the canonical FP64 nested loop, for ragged shapes (row counts
that leave the second SM of the last pair partly or wholly past the store), both
self-join modes, BF16 and FP8, and d up to 1,000. Also: both tile configurations give
the same set on a larger join, the autotuner may pick either, and a bounded wait made
to expire in the pair kernel returns DL_ETIMEOUT with the next call exact.
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
    yield D
    D.set_wait_budget(0)


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def _store(dl, ids, X):
    import torch
    return dl.Store(torch.from_numpy(np.ascontiguousarray(ids)).cuda(),
                    torch.from_numpy(np.ascontiguousarray(X)).cuda())


def _pairs(dl, Rs, Ss, eps, prec, pair, self_mode="upper"):
    res = dl.sim_join(Rs, Ss, eps, precision=prec, self_mode=self_mode, cta_pair=pair)
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
    (1, 1, 16), (1, 700, 64), (129, 255, 64), (255, 257, 128), (256, 256, 128), (257, 513, 96),
    (385, 300, 200), (600, 1000, 256), (130, 390, 512), (700, 600, 320),
])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_pair_rxs_ragged_exact(dl, orc, nR, nS, d, prec):
    g = W.rng(7000 + nR + 7 * nS + 13 * d)
    R = W.dirichlet_histograms(g, nR, d)
    S = np.concatenate([R[: nR // 3], W.dirichlet_histograms(g, nS - nR // 3, d)]) if nS > nR // 3 else \
        W.dirichlet_histograms(g, nS, d)
    D = orc.dist_block(R, S)
    eps = math.sqrt(float(np.quantile(D, 0.02)))
    rid = np.arange(nR, dtype=np.int64) * 3 + 11
    sid = np.arange(nS, dtype=np.int64) * 5 + (1 << 40)
    got, st = _pairs(dl, _store(dl, rid, R), _store(dl, sid, S), eps, prec, 2)
    assert st["cta_pair"] == 2 and st["tile_n"] == 256
    assert got == _want(orc, R, S, eps, oracle.MODE_RXS, rid, sid)


@pytest.mark.parametrize("n", [2, 255, 257, 1500])
@pytest.mark.parametrize("self_mode", ["upper", "full"])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_pair_self_join_modes(dl, orc, n, self_mode, prec):
    g = W.rng(7100 + n)
    X, _ = W.clustered_histograms(g, n, 96, max(1, n // 8), 0.01)
    xid = np.arange(n, dtype=np.int64) * 7 + 3
    got, st = _pairs(dl, _store(dl, xid, X), None, 0.12, prec, 2, self_mode)
    assert st["cta_pair"] == 2
    mode = oracle.MODE_SELF_FULL if self_mode == "full" else oracle.MODE_SELF_UPPER
    assert got == _want(orc, X, None, 0.12, mode, xid, xid)


def test_pair_fp8_wide_d_exact(dl, orc):
    g = W.rng(7200)
    R, _ = W.unit_mixture(g, 300, 1000, 32, 0.05)
    S, _ = W.unit_mixture(g, 520, 1000, 32, 0.05)
    D = orc.dist_block(R, S)
    eps = math.sqrt(float(np.quantile(D, 0.01)))
    rid, sid = np.arange(300, dtype=np.int64), np.arange(520, dtype=np.int64) + 10 ** 9
    got, st = _pairs(dl, _store(dl, rid, R), _store(dl, sid, S), eps, "fp8", 2)
    assert st["cta_pair"] == 2
    assert got == _want(orc, R, S, eps, oracle.MODE_RXS, rid, sid)


def test_pair_equals_single_sm_on_a_larger_join(dl, orc):
    g = W.rng(7300)
    X, _ = W.clustered_histograms(g, 20000, 128, 1500, 0.01)
    xid = np.arange(20000, dtype=np.int64) + 5
    Xs = _store(dl, xid, X)
    eps = 0.1
    for prec in ("bf16", "fp8"):
        one, s1 = _pairs(dl, Xs, None, eps, prec, 1)
        two, s2 = _pairs(dl, Xs, None, eps, prec, 2)
        assert s1["cta_pair"] == 1 and s2["cta_pair"] == 2
        assert one == two and len(one) > 20000
    rows = W.sample_rows(20000, 24, 7301)
    D = orc.dist_block(X[rows], X)
    for i, r in enumerate(rows):
        want = {(min(int(xid[r]), int(xid[j])), max(int(xid[r]), int(xid[j])))
                for j in np.nonzero(D[i] <= eps * eps)[0] if j != r}
        have = {p for p in two if int(xid[r]) in p}
        assert have == want, r


def test_pair_rejections(dl):
    g = W.rng(7400)
    X = W.dirichlet_histograms(g, 100, 64)
    Xs = _store(dl, np.arange(100), X)
    for kw in ({"cta_pair": 3}, {"cta_pair": 2, "tile_n": 128}, {"cta_pair": 2, "prune": True}):
        with pytest.raises(dl.DLError) as ei:
            dl.sim_join(Xs, None, 0.1, precision="bf16", **kw)
        assert ei.value.status == dl.DL_EINVAL


def test_pair_wait_expires_then_exact(dl, orc):
    wl = W.rxs_histograms_2k()
    Rs, Ss = _store(dl, wl.r_ids, wl.R), _store(dl, wl.s_ids, wl.S)
    dl.set_wait_budget(1)
    try:
        for prec in ("bf16", "fp8"):
            with pytest.raises(dl.DLError) as ei:
                dl.sim_join(Rs, Ss, wl.eps, precision=prec, cta_pair=2)
            assert ei.value.status == dl.DL_ETIMEOUT
    finally:
        dl.set_wait_budget(0)
    want = _want(orc, wl.R, wl.S, wl.eps, oracle.MODE_RXS, wl.r_ids, wl.s_ids)
    for prec in ("bf16", "fp8"):
        got, _ = _pairs(dl, Rs, Ss, wl.eps, prec, 2)
        assert got == want
