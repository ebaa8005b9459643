"""Parity of the CUDA top-k join (through the C ABI) with the FP64 CPU oracle.

Exact bar: for every query row the ids, their order (canonical distance, then
store row) and the canonical FP64 distances must equal the oracle's bit for bit.
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


def check_topk(dl, orc, Q, S, k, precision="auto", epilogue_warps=0):
    qid = np.arange(Q.shape[0], dtype=np.int64) * 5 + 3
    sid = np.arange(S.shape[0], dtype=np.int64) * 7 + 1_000_000
    Qs, Ss = _store(dl, qid, Q), _store(dl, sid, S)
    res = dl.topk_join(Qs, Ss, k, precision=precision, epilogue_warps=epilogue_warps)
    ids, d2 = res.topk_host()
    st = res.stats()
    res.free()
    oi, od = orc.topk(Q, S, k)
    want_ids = np.where(oi >= 0, sid[np.clip(oi, 0, None)], -1)
    bad = np.nonzero((ids != want_ids).any(axis=1) | (d2 != od).any(axis=1))[0]
    assert bad.size == 0, (f"{bad.size} rows differ, first {bad[:5].tolist()}; stats={st}; "
                           f"got {ids[bad[0]][:8].tolist()} {d2[bad[0]][:4].tolist()} "
                           f"want {want_ids[bad[0]][:8].tolist()} {od[bad[0]][:4].tolist()}")
    return st


@pytest.mark.parametrize("k", [1, 10, 100])
def test_topk_histograms_2k(dl, orc, k):
    wl = W.rxs_histograms_2k()
    check_topk(dl, orc, wl.R[:700], wl.S, k)


@pytest.mark.parametrize("nQ,nS,d,k", [
    (1, 1, 1, 1), (3, 2, 5, 4), (130, 257, 16, 7), (257, 1000, 64, 33), (129, 3000, 128, 10),
    (64, 500, 200, 5), (40, 700, 512, 3),
])
def test_topk_ragged(dl, orc, nQ, nS, d, k):
    g = W.rng(4000 + nQ + nS + d + k)
    Q = W.dirichlet_histograms(g, nQ, d)
    S = W.dirichlet_histograms(g, nS, d)
    check_topk(dl, orc, Q, S, k)


@pytest.mark.parametrize("nQ,nS0,d,k", [(330000, 150, 8, 1), (60000, 1000, 16, 3), (60000, 1000, 16, 12),
                                         (60000, 1000, 16, 40)])
def test_topk_many_rows_per_warp_exact(dl, orc, nQ, nS0, d, k):
    """Enough query rows that each finalize warp takes several: rows with few columns left
    queue them and share lane-parallel passes of canonical FP64 distances (k = 1 with 34 rows
    per warp fills the queue's 32 row slots; k = 12 fills its 64 columns), and rows with more
    take the direct path after the queue is flushed (k = 40). A quarter of the store rows are
    duplicated, so distances tie and the rank falls back to the store row."""
    g = W.rng(4300 + k)
    S0 = W.dirichlet_histograms(g, nS0, d)
    S = np.concatenate([S0, S0[: nS0 // 4]])
    Q = W.dirichlet_histograms(g, nQ, d)
    check_topk(dl, orc, Q, S, k)


def test_topk_clustered_self(dl, orc):
    """Queries are the store itself: each row's nearest is itself at distance 0."""
    g = W.rng(41)
    X, _ = W.clustered_histograms(g, 2500, 96, 200, 0.01)
    st = check_topk(dl, orc, X[:600], X, 10)
    assert st["pairs_out"] == 600 * 10


def test_topk_ties_and_duplicates(dl, orc):
    """Exact duplicate store rows: ties broken by the smaller store row."""
    g = W.rng(42)
    base = W.grid_points(g, 60, 24, levels=3)
    S = np.concatenate([base, base, base[:20], W.grid_points(g, 300, 24, levels=3)])
    Q = np.concatenate([base[:30], W.grid_points(g, 30, 24, levels=3)])
    for k in (1, 5, 40):
        check_topk(dl, orc, Q, S, k)


def test_topk_overflow_fallback(dl, orc):
    """Hundreds of exact duplicates of a query overflow the candidate lists; the exact scan answers."""
    g = W.rng(43)
    Q = W.dirichlet_histograms(g, 8, 32)
    S = np.concatenate([np.repeat(Q[:2], 400, axis=0), W.dirichlet_histograms(g, 3000, 32)])
    st = check_topk(dl, orc, Q, S, 10)
    assert st["band_pairs"] >= 2   # rows re-solved by the exact scan


def test_topk_k_exceeds_store_and_wide_d(dl, orc):
    g = W.rng(44)
    Q = W.dirichlet_histograms(g, 9, 16)
    S = W.dirichlet_histograms(g, 5, 16)
    check_topk(dl, orc, Q, S, 8)
    Q = W.dirichlet_histograms(g, 12, 700)
    S = W.dirichlet_histograms(g, 300, 700)
    check_topk(dl, orc, Q, S, 6)          # d > 512: exact scan path


def test_topk_empty_store(dl):
    import torch
    Q = dl.Store(torch.arange(4, device="cuda"), torch.rand(4, 8, device="cuda"))
    E = dl.Store(torch.empty(0, dtype=torch.int64, device="cuda"), torch.empty(0, 8, device="cuda"))
    res = dl.topk_join(Q, E, 3)
    ids, d2 = res.topk_host()
    assert (ids == -1).all() and (d2 == -1.0).all()
    res.free()


@pytest.mark.parametrize("k", [4, 10, 100])
def test_topk_large_store_with_ties_exact(dl, orc, k):
    """A 70,000-row store split over ten S splits per query row (many slots per row share the
    row threshold). Ids and distances must equal the oracle's bit for bit, including exact ties
    at the k-th distance (600 planted duplicate rows) and query rows that are store rows."""
    g = W.rng(8800 + k)
    S, _ = W.clustered_histograms(g, 70_000, 64, 900, 0.01)
    dup_src = g.choice(70_000, size=600, replace=False)
    dup_dst = g.choice(np.setdiff1d(np.arange(70_000), dup_src), size=600, replace=False)
    S[dup_dst] = S[dup_src]
    Q, _ = W.clustered_histograms(g, 260, 64, 900, 0.012)
    Q = np.concatenate([Q, S[dup_src[:40]]])
    st = check_topk(dl, orc, Q, S, k)
    assert st["band_pairs"] < Q.shape[0]   # rows re-solved by the exact scan stay rare


@pytest.mark.parametrize("k", [1, 10, 100])
def test_topk_wide_epilogue_exact(dl, orc, k):
    """The 16-warp epilogue (slots per row, split and quarter of a tile): ids and distances equal
    the oracle's, with exact ties at the k-th distance and ragged store sizes."""
    g = W.rng(8900 + k)
    S, _ = W.clustered_histograms(g, 20_011, 64, 400, 0.01)
    S[g.choice(20_011, 300, replace=False)] = S[g.choice(20_011, 300, replace=False)]
    Q, _ = W.clustered_histograms(g, 333, 64, 400, 0.012)
    st = check_topk(dl, orc, Q, S, k, precision="bf16", epilogue_warps=16)
    assert st["epilogue_warps"] == 16
