"""Bound validity of the low-precision stage: |h~ - h| <= E for every pair.

The tensor-core kernel decides most pairs from h~ (an approximation of
h = q.x - ||x||^2/2, so D = ||q||^2 - 2h) and a per-pair bound E. The bound's
encoding part is proven; its accumulation part rests on an ASSUMED tensor-core
accumulation error gamma = d_p * 2^-20 (the hardware's summation order and
rounding are not documented). This test dumps h~ and E for many random pairs --
non-negative histograms and signed unit-norm embeddings, d from 64 to 1024, one
to eight K chunks -- and checks
  (1) |h~ - h| <= E against h in FP64 (the whole bound), and
  (2) the accumulation error alone, |h~ - (q~.x~ - beta~)| with q~, x~ the
      encoded rows rebuilt on the host, stays below 5% of gamma ||q~|| ||x~||.
"""

import numpy as np
import pytest

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


def enc_bf16(X):
    import torch
    return torch.from_numpy(X).to(torch.bfloat16).to(torch.float64).numpy()


def enc_fp8(X):
    """Host rebuild of the library's FP8 copy: power-of-two scale s with max|x|/s <= 448, RN e4m3.

    The library shares one scale per 32-row chunk (the largest row scale of the chunk); the FP8
    cases below give every row max|x| = 1, so every row scale, hence every chunk scale, is 2^-8
    and the per-row rebuild here is exact.
    """
    import torch
    mx = np.abs(X).max(axis=1, keepdims=True).astype(np.float32)
    m, e = np.frexp(mx / np.float32(448.0))
    s = np.ldexp(np.float32(1.0), np.where(m == 0.5, e - 1, e)).astype(np.float32)
    s = np.where(mx > 0, s, np.float32(1.0))
    while ((mx / s) > 448).any():
        s = np.where((mx / s) > 448, s * 2, s)
    q = torch.from_numpy((X / s).astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    return q * s.astype(np.float64)


def _data(kind, d, n, g):
    if kind == "hist":
        return W.dirichlet_histograms(g, n, d)
    X, _ = W.unit_mixture(g, n, d, 64, 0.05)
    return X


CASES = [("bf16", d) for d in (64, 128, 256, 512)] + [("fp8", d) for d in (64, 128, 256, 512, 1024)]


@pytest.mark.parametrize("prec,d", CASES)
@pytest.mark.parametrize("kind", ["hist", "signed"])
def test_bound_and_accumulation_margin(dl, prec, d, kind):
    import torch
    g = W.rng(9000 + d + (kind == "signed") + 17 * (prec == "fp8"))
    R, S = _data(kind, d, 320, g), _data(kind, d, 2500, g)
    if prec == "fp8":   # one scale for every row (see enc_fp8)
        R = (R / np.abs(R).max(axis=1, keepdims=True)).astype(np.float32)
        S = (S / np.abs(S).max(axis=1, keepdims=True)).astype(np.float32)
    Rs = dl.Store(torch.arange(R.shape[0]).cuda(), torch.from_numpy(R).cuda())
    Ss = dl.Store(torch.arange(S.shape[0]).cuda(), torch.from_numpy(S).cuda())
    h, e = dl.debug_scores(Rs, Ss, prec)
    h, e = h.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
    R64, S64 = R.astype(np.float64), S.astype(np.float64)
    beta = 0.5 * (S64 * S64).sum(axis=1)
    hx = R64 @ S64.T - beta[None, :]
    ratio = np.abs(h - hx) / e
    # (2): accumulation error against the assumed gamma
    enc = enc_bf16 if prec == "bf16" else enc_fp8
    Rq, Sq = enc(R), enc(S)
    beta32 = beta.astype(np.float32).astype(np.float64)
    acc = np.abs(h - (Rq @ Sq.T - beta32[None, :]))
    dp = (d + 63) // 64 * 64 if prec == "bf16" else (d + 127) // 128 * 128
    gamma = dp * 2.0 ** -20
    acc_ratio = acc / (gamma * np.linalg.norm(Rq, axis=1)[:, None] * np.linalg.norm(Sq, axis=1)[None, :])
    print(f"{prec} d={d} {kind}: max |h~-h|/E {ratio.max():.3f}; max accumulation / assumed {acc_ratio.max():.2e}")
    assert ratio.max() <= 1.0
    assert acc_ratio.max() < 0.05
