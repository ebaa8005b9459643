"""Full-size parity of the 1,048,576 x 1,048,576 d=512 unit-norm join (BF16 and FP8).

The oracle cannot run the whole join, so its exact pair set for a seeded sample of
16,384 R rows against ALL of S is stored as a digest in
tests/golden/unit_mixture_1m_sample16k.json (written by the committed script beside
it, which calls only the oracle). Here the GPU path computes

  * the sample rows x S join, in BF16 and FP8 (the digest must match exactly), and
  * the whole 1M x 1M join in one launch, in BF16 and in FP8, restricted afterwards to the
    sample rows (the digest must match again: the full-size launch decides those rows
    exactly).

The input generator's output is pinned by hashes in the same file, so a platform
whose generator draws differ is reported as such and not as a join mismatch.
"""

import base64
import hashlib
import json
import os
import zlib

import numpy as np
import pytest

from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "unit_mixture_1m_sample16k.json")


@pytest.fixture(scope="module")
def dl():
    import torch
    from paper_1812_07607_gb300 import build as B, dl as D
    assert torch.cuda.is_available()
    B.build()
    D.load()
    return D


@pytest.fixture(scope="module")
def c3():
    with open(GOLDEN) as f:
        gold = json.load(f)
    wl = W.rxs_unit_mixture_1m()
    rows = W.sample_rows(wl.R.shape[0], gold["sample_rows"], gold["sample_seed"])
    Rs = np.ascontiguousarray(wl.R[rows])
    assert hashlib.sha256(Rs.astype("<f4").tobytes()).hexdigest() == gold["r_sample_sha256"], \
        "generator output differs from the one the golden digest was written for"
    assert hashlib.sha256(np.ascontiguousarray(wl.S, dtype="<f4").tobytes()).hexdigest() == gold["s_sha256"], \
        "generator output differs from the one the golden digest was written for"
    assert wl.eps == gold["eps"]
    return wl, rows, Rs, gold


def _digest(pos, srow):
    P = np.stack([np.asarray(pos, np.int64), np.asarray(srow, np.int64)], axis=1)
    P = P[np.lexsort((P[:, 1], P[:, 0]))]
    return P, hashlib.sha256(np.ascontiguousarray(P, dtype="<i8").tobytes()).hexdigest()


def _check(P, digest, gold, what):
    counts = np.frombuffer(zlib.decompress(base64.b64decode(gold["counts_zlib_b64"])), dtype="<u2")
    got = np.bincount(P[:, 0], minlength=gold["sample_rows"])
    bad = np.nonzero(got != counts)[0]
    assert bad.size == 0, f"{what}: per-row counts differ at sample rows {bad[:10].tolist()}"
    assert P.shape[0] == gold["pairs"] and digest == gold["pairs_sha256"], what


def test_unit_mixture_1m_sample_rows_bf16_fp8(dl, c3):
    import torch
    wl, rows, Rs, gold = c3
    n = wl.S.shape[0]
    S = dl.Store(torch.arange(n).cuda(), torch.from_numpy(wl.S).cuda())
    R = dl.Store(torch.arange(Rs.shape[0]).cuda(), torch.from_numpy(Rs).cuda())
    for prec in ("bf16", "fp8"):
        res = dl.sim_join(R, S, wl.eps, precision=prec)
        a, b = res.pairs_host()
        res.free()
        P, dg = _digest(a, b)
        _check(P, dg, gold, prec)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_unit_mixture_1m_full_launch(dl, c3, prec):
    import torch
    wl, rows, Rs, gold = c3
    n = wl.R.shape[0]
    S = dl.Store(torch.arange(n).cuda(), torch.from_numpy(wl.S).cuda())
    R = dl.Store(torch.arange(n).cuda(), torch.from_numpy(wl.R).cuda())
    res = dl.sim_join(R, S, wl.eps, precision=prec)
    a, b = res.pairs_host()
    st = res.stats()
    res.free()
    assert st["pairs_evaluated"] == n * n
    pos = np.full(n, -1, dtype=np.int64)
    pos[rows] = np.arange(rows.shape[0])
    keep = pos[a] >= 0
    P, dg = _digest(pos[a[keep]], b[keep])
    _check(P, dg, gold, f"full launch {prec}")
    # the whole result: about 10 matches per row, no duplicates
    assert 5 * n < a.shape[0] < 20 * n
    key = a * n + b
    assert np.unique(key).shape[0] == key.shape[0]
