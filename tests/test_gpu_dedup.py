"""q4 deduplication on the GPU against the oracle: connected components (bit-exact
smallest-row labels and counts) and the three plans of dl_dedup."""

import numpy as np
import pytest

import oracle
from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PLANS = {"all": oracle.DEDUP_ALL, "filter_match": oracle.DEDUP_FILTER_MATCH,
         "match_filter": oracle.DEDUP_MATCH_FILTER}


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


def _graph(g, n, m, loops=True):
    p = g.integers(0, n, size=(m, 2))
    if loops and m:
        p = np.concatenate([p, p[: m // 4], np.stack([p[:5, 0], p[:5, 0]], 1)])
    return p.astype(np.int64)


@pytest.mark.parametrize("n,m", [(1, 0), (5, 0), (40, 10), (1000, 700), (1000, 3000), (100000, 60000),
                                 (100000, 300000)])
def test_components_equal_oracle(dl, orc, n, m):
    import torch
    g = W.rng(9300 + n + m)
    p = _graph(g, n, m)
    want, wc = orc.components(n, p)
    t = torch.from_numpy(p).cuda()
    lab, c = dl.components(n, t[:, 0], t[:, 1])
    assert c == wc and np.array_equal(lab.cpu().numpy(), want)


def test_components_paths_and_rejection(dl, orc):
    import torch
    n = 5000
    g = W.rng(9400)
    perm = g.permutation(n)
    p = np.stack([perm[:-1], perm[1:]], 1).astype(np.int64)[g.permutation(n - 1)]   # one long shuffled path
    t = torch.from_numpy(p).cuda()
    lab, c = dl.components(n, t[:, 0], t[:, 1])
    assert c == 1 and bool((lab == 0).all())
    bad = torch.tensor([[0, n]], dtype=torch.int64, device="cuda")
    with pytest.raises(dl.DLError) as ei:
        dl.components(n, bad[:, 0], bad[:, 1])
    assert ei.value.status == dl.DL_EINVAL


def test_dedup_hand_example(dl):
    import torch
    X = np.array([[0.0], [1.0], [2.0], [10.0], [20.0], [21.0]], dtype=np.float32)
    lab = torch.tensor([1, 2, 1, 1, 2, 2], dtype=torch.int32, device="cuda")
    S = dl.Store(torch.arange(6, device="cuda") * 11, torch.from_numpy(X).cuda())
    comp, c = dl.dedup(S, 1.0, plan="all", precision="fp32")
    assert c == 3 and comp.cpu().tolist() == [0, 0, 0, 3, 4, 4]
    comp, c = dl.dedup(S, 1.0, lab, 1, plan="filter_match", precision="fp32")
    assert c == 3 and comp.cpu().tolist() == [0, -1, 2, 3, -1, -1]
    comp, c = dl.dedup(S, 1.0, lab, 1, plan="match_filter", precision="fp32")
    assert c == 2 and comp.cpu().tolist() == [0, 0, 0, 3, 4, 4]
    comp, c = dl.dedup(S, 1.0, lab, 7, plan="filter_match", precision="fp32")
    assert c == 0 and bool((comp == -1).all())


@pytest.mark.parametrize("plan", sorted(PLANS))
@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_dedup_clustered_equals_oracle(dl, orc, plan, prec):
    import torch
    g = W.rng(9500)
    X, groups = W.clustered_histograms(g, 3000, 64, 300, 0.01)
    labels = W.object_labels(g, groups, 300)
    perm = g.permutation(3000)       # rows out of group order
    X, groups, labels = X[perm], groups[perm], labels[perm]
    D = orc.dist_block(X[:200], X)
    eps = float(np.sqrt(np.quantile(D[D > 0], 0.004)))
    S = dl.Store(torch.arange(3000, device="cuda") * 3 + 1, torch.from_numpy(X).cuda())
    want, wc = orc.dedup(X, eps, labels, 0, PLANS[plan])
    comp, c = dl.dedup(S, eps, torch.from_numpy(labels).cuda(), 0, plan=plan, precision=prec)
    assert c == wc and np.array_equal(comp.cpu().numpy(), want), (plan, c, wc)
