"""Bound validity of the low-precision stage: |h~ - h| <= E for every pair.

The tensor-core kernel decides most pairs from h~ (an approximation of
h = q.x - ||x||^2/2, so D = ||q||^2 - 2h) and a per-pair bound E. The bound's
encoding part is proven; its accumulation part rests on an ASSUMED tensor-core
accumulation error gamma = d_p * 2^-20 (the hardware's summation order and
rounding are not documented). This test dumps h~ and E for 10,240 x 10,240 = 1.05e8 random pairs per case --
non-negative histograms and signed unit-norm embeddings, d from 64 to 1024, one
to eight K chunks -- and checks
  (1) |h~ - h| <= E against h in FP64 (the whole bound), and
  (2) the accumulation error alone, |h~ - (q~.x~ - beta~)| with q~, x~ the
      encoded rows rebuilt on the host, stays below 5% of gamma ||q~|| ||x~||.
The reference values are FP64 matrix products on the device (their own error,
about d 2^-53 ||q|| ||x||, is far below E). The largest ratio of each case is
appended to the file named by DL_BOUNDS_LOG, when that variable is set.
"""

import json
import os

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


N_ROWS = 10240   # 10,240^2 = 1.05e8 pairs per (precision, d, data) case


@pytest.mark.parametrize("prec,d", CASES)
@pytest.mark.parametrize("kind", ["hist", "signed"])
def test_bound_and_accumulation_margin(dl, prec, d, kind):
    import torch
    g = W.rng(9000 + d + (kind == "signed") + 17 * (prec == "fp8"))
    R, S = _data(kind, d, N_ROWS, g), _data(kind, d, N_ROWS, g)
    if prec == "fp8":   # one scale for every row (see enc_fp8)
        R = (R / np.abs(R).max(axis=1, keepdims=True)).astype(np.float32)
        S = (S / np.abs(S).max(axis=1, keepdims=True)).astype(np.float32)
    Rd, Sd = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    Rs = dl.Store(torch.arange(R.shape[0]).cuda(), Rd)
    Ss = dl.Store(torch.arange(S.shape[0]).cuda(), Sd)
    h, e = dl.debug_scores(Rs, Ss, prec)
    h, e = h.double(), e.double()
    R64, S64 = Rd.double(), Sd.double()
    beta = 0.5 * (S64 * S64).sum(dim=1)
    ratio = float(((h - (R64 @ S64.T - beta[None, :])).abs() / e).max())
    # (2): accumulation error against the assumed gamma
    enc = enc_bf16 if prec == "bf16" else enc_fp8
    Rq, Sq = torch.from_numpy(enc(R)).cuda(), torch.from_numpy(enc(S)).cuda()
    beta32 = beta.float().double()
    acc = (h - (Rq @ Sq.T - beta32[None, :])).abs()
    dp = (d + 63) // 64 * 64 if prec == "bf16" else (d + 127) // 128 * 128
    gamma = dp * 2.0 ** -20
    acc_ratio = float((acc / (gamma * Rq.norm(dim=1)[:, None] * Sq.norm(dim=1)[None, :])).max())
    pairs = R.shape[0] * S.shape[0]
    print(f"{prec} d={d} {kind}: {pairs} pairs; max |h~-h|/E {ratio:.3f}; max accumulation / assumed {acc_ratio:.2e}")
    if os.environ.get("DL_BOUNDS_LOG"):
        with open(os.environ["DL_BOUNDS_LOG"], "a") as f:
            f.write(json.dumps({"prec": prec, "d": d, "kind": kind, "pairs": pairs, "bound_ratio": ratio,
                                "acc_ratio": acc_ratio}) + "\n")
    assert pairs >= 10 ** 8
    assert ratio <= 1.0
    assert acc_ratio < 0.05
