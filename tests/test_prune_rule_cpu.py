"""Soundness of the pruned join's tile-pair rule, checked on the CPU against the oracle.

The rule (prune.cu): each tile run gets a centre c = fl32(mean) and a radius r >= max
||x - c|| (FP64, widened by 1e-9, rounded up to FP32); a tile pair is skipped when, for
every pair of balls, lower = fl32(||c1 - c2||) * (1 - 1e-4) - r1 - r2 > 0 and lower^2 >
fl32_up(eps^2 (1 + 1e-6)). Here the rule is evaluated in numpy on many seeded inputs -- tight
clusters, near-duplicate rows, thresholds placed at and just below the closest cross-tile
distance -- and every skipped tile pair is checked to hold no pair with canonical D <= eps^2.
"""

import numpy as np
import pytest

import oracle
from paper_1812_07607_gb300 import workloads as W

ORC = oracle.default()


def _f32_up(x: float) -> np.float32:
    f = np.float32(x)
    return f if float(f) >= x else np.nextafter(f, np.float32(np.inf))


def _balls(X, labels, rows):
    out = []
    for t0 in range(0, len(X), rows):
        lab = labels[t0:t0 + rows]
        cuts = [0] + [i for i in range(1, len(lab)) if lab[i] != lab[i - 1]] + [len(lab)]
        if len(cuts) - 1 > 4:
            cuts = [0, len(lab)]
        bl = []
        for a, b in zip(cuts[:-1], cuts[1:]):
            xs = X[t0 + a:t0 + b].astype(np.float64)
            c = xs.mean(axis=0).astype(np.float32)
            r = np.sqrt(((xs - c.astype(np.float64)) ** 2).sum(axis=1).max())
            bl.append((c, _f32_up(r * (1 + 1e-9) + 1e-30)))
        out.append(bl)
    return out


def _skipped(bR, bS, e2):
    e2_up = _f32_up(e2 * (1 + 1e-6) + 1e-37)
    skip = np.zeros((len(bR), len(bS)), dtype=bool)
    for i, a in enumerate(bR):
        for j, b in enumerate(bS):
            ok = True
            for ca, ra in a:
                for cb, rb in b:
                    w = (ca - cb).astype(np.float32)
                    s = np.float32(0)
                    for v in w:   # an FP32 sum of squares (the kernel fuses each step; either is within the margin)
                        s = np.float32(s + np.float32(v * v))
                    lower = np.float32(np.float32(np.sqrt(s)) * np.float32(1 - 1e-4)) - ra - rb
                    if not (lower > 0 and np.float32(lower * lower) > e2_up):
                        ok = False
            skip[i, j] = ok
    return skip


@pytest.mark.parametrize("seed", range(6))
def test_skipped_tile_pairs_hold_no_pair(seed):
    g = W.rng(4200 + seed)
    n_obj, d = int(g.integers(3, 9)), int(g.integers(2, 17))
    X, groups = W.clustered_histograms(g, 96 * n_obj, d, n_obj, float(g.choice([0.001, 0.004, 0.02])))
    if seed % 2:   # planted near-duplicates across objects
        X[5] = X[-7] + np.float32(1e-4)
    order = np.argsort(groups, kind="stable")
    X, groups = X[order], groups[order]
    D = ORC.dist_block(X, X)
    rows_r, rows_s = 32, 64
    bR, bS = _balls(X, groups, rows_r), _balls(X, groups, rows_s)
    # thresholds: at the closest distance between rows of different objects, just below it,
    # and at a small quantile
    cross = D[groups[:, None] != groups[None, :]]
    dmin = float(cross.min())
    for e2 in (dmin, float(np.nextafter(dmin, 0)), float(np.quantile(cross, 0.01)), 0.0):
        eps = float(np.sqrt(e2))
        e2r = eps * eps
        skip = _skipped(bR, bS, e2r)
        for i in range(len(bR)):
            for j in range(len(bS)):
                if skip[i, j]:
                    blk = D[i * rows_r:(i + 1) * rows_r, j * rows_s:(j + 1) * rows_s]
                    assert float(blk.min()) > e2r, (seed, e2r, i, j, float(blk.min()))
        assert skip.sum() > 0 or e2r > 0.01   # the rule does skip something on tight data
