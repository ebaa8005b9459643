"""Edge cases at the domain limits and a seeded randomized sweep, all against the oracle.

* Features near the largest admitted magnitude (|x| up to 2^39): the FP32 squared norms and
  accumulators stay far from overflow and every precision still returns the oracle's set.
* A value past 2^40 is rejected at store creation (DL_EINVAL).
* 24 seeded configurations drawn at random: n, m in [1, 700], d in [1, 300], R x S or a
  self-join in either mode, eps at a random distance quantile, BF16 / FP8 / exact FP32 / AUTO.
"""

import math

import numpy as np
import pytest

import oracle
from paper_1812_07607_gb300 import workloads as W
from test_gpu_join import check  # noqa: F401  (shared helpers)

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


def test_large_magnitudes_near_domain_limit(dl, orc):
    g = W.rng(8100)
    base = W.dirichlet_histograms(g, 200, 48).astype(np.float64)
    R = (base * 2.0 ** 39).astype(np.float32)
    S = np.concatenate([R[:60] * np.float32(1.0000002), (W.dirichlet_histograms(g, 140, 48) * 2.0 ** 39)])
    S = S.astype(np.float32)
    D = orc.dist_block(R, S)
    for q in (0.002, 0.05):
        check(dl, orc, R, S, math.sqrt(float(np.quantile(D, q))), precs=("bf16", "fp8", "fp32"))


def test_value_past_domain_limit_is_rejected(dl):
    import torch
    X = torch.rand(16, 8, device="cuda")
    X[5, 3] = 2.0 ** 41
    with pytest.raises(dl.DLError) as ei:
        dl.Store(torch.arange(16, device="cuda"), X)
    assert ei.value.status == dl.DL_EINVAL


def _draw(g, n, d):
    kind = int(g.integers(0, 3))
    if kind == 0:
        return W.dirichlet_histograms(g, n, d)
    if kind == 1:
        return W.grid_points(g, n, d, levels=3, dup_frac=0.2)
    return W.mixed_magnitude_rows(g, n, d) if d <= 64 else W.dirichlet_histograms(g, n, d)


@pytest.mark.parametrize("case", range(24))
def test_randomized_configurations(dl, orc, case):
    g = W.rng(8200 + case)
    n = int(g.integers(1, 701))
    m = int(g.integers(1, 701))
    d = int(g.integers(1, 301))
    prec = ["bf16", "fp8", "fp32", "auto"][case % 4]
    self_join = bool(g.integers(0, 3) == 0)
    R = _draw(g, n, d)
    S = None if self_join else _draw(g, m, d)
    D = orc.dist_block(R, R if S is None else S)
    q = float(g.choice([0.0, 0.001, 0.02, 0.2]))
    eps = math.sqrt(float(np.quantile(D, q))) if D.size else 0.1
    mode = ["upper", "full"][int(g.integers(0, 2))]
    check(dl, orc, R, S, eps, self_mode=mode, precs=(prec,))


@pytest.mark.parametrize("case", range(12))
def test_randomized_topk(dl, orc, case):
    """12 seeded top-k configurations: ids and canonical distances equal the oracle's."""
    import torch
    g = W.rng(8300 + case)
    n = int(g.integers(1, 400))
    m = int(g.integers(1, 900))
    d = int(g.integers(1, 300))
    k = int(g.choice([1, 2, 7, 10, 33, 100, 200]))
    Q, S = _draw(g, n, d), _draw(g, m, d)
    sid = np.arange(m, dtype=np.int64) * 7 + 1
    Qs = dl.Store(torch.arange(n).cuda(), torch.from_numpy(Q).cuda())
    Ss = dl.Store(torch.from_numpy(sid).cuda(), torch.from_numpy(S).cuda())
    res = dl.topk_join(Qs, Ss, k)
    ids, d2 = res.topk_host()
    res.free()
    oi, od = orc.topk(Q, S, k)
    want_ids = np.where(oi >= 0, sid[np.maximum(oi, 0)], -1)
    assert np.array_equal(ids, want_ids), (n, m, d, k)
    assert np.array_equal(d2, np.where(oi >= 0, od, -1.0)), (n, m, d, k)
