"""FP8 e4m3 precision: the same exactness bar as BF16 (set equality with the FP64 oracle).

e4m3 keeps 3 mantissa bits, so its error bound is wide and many more pairs fall
in the band that the exact recheck settles; the returned set must not change.
"""

import math

import numpy as np
import pytest

import oracle
from paper_1812_07607_gb300 import workloads as W
from test_gpu_join import check, gpu_pairs, oracle_pairs  # noqa: F401  (shared helpers)

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


def test_fp8_histograms_2k(dl, orc):
    wl = W.rxs_histograms_2k()
    check(dl, orc, wl.R, wl.S, wl.eps, precs=("fp8",), rid=wl.r_ids, sid=wl.s_ids)


@pytest.mark.parametrize("nR,nS,d", [(1, 1, 1), (127, 129, 16), (300, 257, 64), (513, 300, 128),
                                     (130, 390, 512), (64, 200, 1000)])
def test_fp8_ragged(dl, orc, nR, nS, d):
    g = W.rng(7000 + nR + nS + d)
    R = W.dirichlet_histograms(g, nR, d)
    S = W.dirichlet_histograms(g, nS, d)
    D = orc.dist_block(R, S)
    check(dl, orc, R, S, math.sqrt(float(np.quantile(D, 0.02))), precs=("fp8",))


@pytest.mark.parametrize("self_mode", ["upper", "full"])
def test_fp8_self_join(dl, orc, self_mode):
    g = W.rng(7100)
    X, _ = W.clustered_histograms(g, 1500, 96, 150, 0.01)
    check(dl, orc, X, None, 0.12, self_mode=self_mode, precs=("fp8",))


def test_fp8_adversarial_and_mixed(dl, orc):
    g = W.rng(7200)
    R = W.dirichlet_histograms(g, 150, 64)
    S = np.concatenate([R + g.normal(0, 2e-4, size=R.shape).astype(np.float32),
                        W.dirichlet_histograms(g, 80, 64)]).astype(np.float32)
    D = orc.dist_block(R, S)
    for t in np.sort(D.ravel())[[40, 400]]:
        base = math.sqrt(float(t))
        for step in (-2, 0, 2):
            eps = base
            for _ in range(abs(step)):
                eps = float(np.nextafter(eps, math.inf if step > 0 else 0.0))
            check(dl, orc, R, S, eps, precs=("fp8",))
    M = W.mixed_magnitude_rows(g, 120, 32)
    N = np.concatenate([M[:30] * np.float32(1.0000001), W.mixed_magnitude_rows(g, 70, 32)])
    D = orc.dist_block(M, N)
    check(dl, orc, M, N, math.sqrt(float(np.quantile(D, 0.01))), precs=("fp8",))
    G = W.grid_points(g, 200, 24, levels=4)
    base = G[g.integers(0, 200, size=150)]
    step = g.integers(-3, 4, size=base.shape) * (g.uniform(size=base.shape) < 0.15)
    H = (base + step.astype(np.float32) / 8.0).astype(np.float32)
    check(dl, orc, G, H, 3.0 / 8.0, precs=("fp8",))


def test_fp8_bench_workload_equals_bf16(dl):
    """Full-size 262,144-row self-join: the FP8 set equals the BF16 set (both exact)."""
    import torch
    wl = W.self_clustered_262k()
    S = dl.Store(torch.from_numpy(wl.r_ids).cuda(), torch.from_numpy(wl.R).cuda())
    a = dl.sim_join(S, None, wl.eps, precision="bf16")
    b = dl.sim_join(S, None, wl.eps, precision="fp8")
    ra, sa = a.pairs_host()
    rb, sb = b.pairs_host()
    stb = b.stats()
    a.free()
    b.free()
    assert set(zip(ra.tolist(), sa.tolist())) == set(zip(rb.tolist(), sb.tolist()))
    print("fp8 band pairs", stb["band_pairs"], "fp64", stb["fp64_pairs"])


def test_fp8_signed_multichunk_equals_exact_fp32(dl):
    """Signed unit-norm embeddings at d = 256 / 512 / 1024 (2-8 FP8 K chunks): FP8 set == exact FP32 set."""
    import torch
    g = W.rng(7300)
    for d, n in ((256, 6000), (512, 6000), (1024, 3000)):
        # jitter of norm ~0.15: same-centroid pairs sit near 0.21 apart, right at eps
        sig = 0.15 / np.sqrt(d)
        R, c = W.unit_mixture(g, n, d, 256, sig)
        S, _ = W.unit_mixture(g, n, d, 256, sig, centroids=c)
        Rs = dl.Store(torch.arange(n).cuda(), torch.from_numpy(R).cuda())
        Ss = dl.Store(torch.arange(n).cuda() + 10**9, torch.from_numpy(S).cuda())
        sets = {}
        for prec in ("fp8", "fp32"):
            r = dl.sim_join(Rs, Ss, 0.21, precision=prec)
            a, b = r.pairs_host()
            r.free()
            sets[prec] = set(zip(a.tolist(), b.tolist()))
        assert len(sets["fp32"]) > 100 and sets["fp8"] == sets["fp32"], (d, len(sets["fp8"] ^ sets["fp32"]))


def test_auto_precision_uses_fp8_above_512(dl, orc):
    """d in (512, 1024]: the BF16 R tile does not fit in shared memory, so AUTO takes FP8 (still exact)."""
    g = W.rng(7400)
    R = W.dirichlet_histograms(g, 300, 768)
    S = W.dirichlet_histograms(g, 700, 768)
    D = orc.dist_block(R, S)
    eps = math.sqrt(float(np.quantile(D, 0.01)))
    got, st, rid, sid = gpu_pairs(dl, R, S, eps, "auto")
    assert st["precision"] == dl.DL_PREC_FP8E4M3
    want = oracle_pairs(orc, R, S, eps, oracle.MODE_RXS, rid, sid)
    assert got == want
