"""Pins that tie the CPU oracle to the paper and to mathematics, not to itself.

Each pin takes an `oracle.Oracle` and raises AssertionError when the oracle
disagrees with something the paper or the mathematics fixes:

  * exact rational arithmetic (fractions.Fraction) on tiny inputs -- the join
    set of Sec. 5's nested loop under Sec. 3.2's Euclidean threshold, with no
    rounding at all;
  * the hand-derived integer fixture in tests/golden/grid_join_small.txt;
  * closed forms: one-hot histograms (distinct rows are sqrt(2) apart) and
    integer grids scaled by 2^-3 (exact in every format);
  * invariants: self-join symmetry, zero self-distance, monotonicity in eps,
    eps=0 gives exact duplicates, eps=inf gives every pair, permutation and
    union laws, top-k ordering and top-k/join consistency;
  * the cosine metric: the normalized rows against exact rational arithmetic
    (round-to-nearest quotients, unit norm within the rounding bound, invariance
    under power-of-two scaling) and the cosine join against the exact cosine;
  * the L1 and chi-square histogram distances against exact rationals, their
    one-hot and histogram-intersection closed forms, symmetry and chi2 <= L1;
  * the colour-histogram transformer against the hand-derived fixture
    tests/golden/color_hist_small.txt, the uniform-binning definition at every
    8-bit value, count conservation, box additivity and pixel-order invariance;
  * connected components against scipy's graph routine and closed forms (paths,
    isolated rows), and the q4 plans on a hand-built example.

The same suite runs against deliberately broken copies of the oracle
(tests/test_oracle_mutants.py) to show that a plausible slip fails a pin.
"""

from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np

import oracle
from oracle import MODE_RXS, MODE_SELF_FULL, MODE_SELF_UPPER
from paper_1812_07607_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grid_join_small.txt")


# ----------------------------------------------------------------------------------------
# exact helpers (plain definitions, written independently of oracle.c)
# ----------------------------------------------------------------------------------------

def exact_d2(q, x) -> Fraction:
    """Exact squared Euclidean distance of two float32 rows, as a rational."""
    s = Fraction(0)
    for a, b in zip(q.tolist(), x.tolist()):
        t = Fraction(a) - Fraction(b)
        s += t * t
    return s


def exact_matrix(R, S):
    return [[exact_d2(R[i], S[j]) for j in range(S.shape[0])] for i in range(R.shape[0])]


def pair_set(p):
    return set(map(tuple, np.asarray(p).reshape(-1, 2).tolist()))


def eps_between(values, lo_rank: int):
    """An eps whose square (in FP64) lies strictly inside a wide gap of `values`.

    Sorts the distinct exact distances, picks the first gap at or after rank
    `lo_rank` that is wider than 1e-6 relative, and returns eps with
    fl(eps*eps) inside it, so that no distance is near the threshold.
    """
    vals = sorted(set(values))
    for r in range(max(0, lo_rank), len(vals) - 1):
        a, b = vals[r], vals[r + 1]
        if b - a > Fraction(1, 10**6) * max(b, Fraction(1, 10**30)):
            mid = (a + b) / 2
            eps = math.sqrt(float(mid))
            e2 = Fraction(eps * eps)
            if a < e2 < b:
                return eps, e2
    raise AssertionError("no usable gap")


def _g(seed):
    return W.rng(seed)


# ----------------------------------------------------------------------------------------
# pins
# ----------------------------------------------------------------------------------------

def pin_sqdist_within_rounding_of_exact(orc):
    """|D64 - D| <= (d+3) 2^-53 D for the canonical FP64 sum (standard error bound)."""
    g = _g(11)
    for d in (1, 2, 3, 7, 16, 33):
        for gen in (W.mixed_magnitude_rows, lambda g, n, d: W.dirichlet_histograms(g, n, d)):
            X = gen(g, 6, d)
            for i in range(X.shape[0]):
                for j in range(X.shape[0]):
                    D = exact_d2(X[i], X[j])
                    got = orc.sqdist(X[i], X[j])
                    if D == 0:
                        assert got == 0.0, (d, i, j, got)
                    else:
                        err = abs(Fraction(got) - D)
                        assert err <= Fraction(d + 3, 2**53) * D, (d, i, j, got, float(D))


def pin_join_matches_exact_rational(orc):
    """All three join modes equal the exact-rational nested loop on tiny inputs."""
    g = _g(12)
    for d, nR, nS in ((1, 9, 11), (5, 23, 31), (12, 17, 13)):
        R = W.mixed_magnitude_rows(g, nR, d) if d != 12 else W.dirichlet_histograms(g, nR, d)
        S = W.mixed_magnitude_rows(g, nS, d) if d != 12 else W.dirichlet_histograms(g, nS, d)
        M = exact_matrix(R, S)
        vals = [v for row in M for v in row]
        for rank in (0, len(vals) // 7, len(vals) // 2):
            eps, e2 = eps_between(vals, rank)
            want = {(i, j) for i in range(nR) for j in range(nS) if M[i][j] <= e2}
            assert pair_set(orc.join(R, S, eps, MODE_RXS)) == want, (d, rank)
        MS = exact_matrix(R, R)
        svals = [MS[i][j] for i in range(nR) for j in range(nR) if i != j]
        eps, e2 = eps_between(svals, len(svals) // 3)
        up = {(i, j) for i in range(nR) for j in range(i + 1, nR) if MS[i][j] <= e2}
        full = {(i, j) for i in range(nR) for j in range(nR) if MS[i][j] <= e2}
        assert pair_set(orc.join(R, None, eps, MODE_SELF_UPPER)) == up, d
        assert pair_set(orc.join(R, None, eps, MODE_SELF_FULL)) == full, d


def read_golden(path=GOLDEN):
    R, S, T, Q = [], [], [], []
    entries = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "d":
                continue
            if tok[0] in ("R", "S"):
                (R if tok[0] == "R" else S).append([float(v) for v in tok[1:]])
            elif tok[0] == "topk_ties" and tok[1] in ("Q", "T"):
                (Q if tok[1] == "Q" else T).append([float(v) for v in tok[2:]])
            else:
                key, val = line.split(":")
                entries[key.strip()] = val.split()
    f32 = lambda a: np.asarray(a, dtype=np.float32)
    return f32(R), f32(S), f32(Q), f32(T), entries


def _pairs_tok(toks):
    return {tuple(int(v) for v in t.split(",")) for t in toks}


def pin_golden_fixture(orc):
    """The hand-derived integer fixture (tests/golden/grid_join_small.txt)."""
    R, S, Q, T, e = read_golden()
    for key, toks in e.items():
        parts = key.split()
        if parts[0] == "join_rxs":
            assert pair_set(orc.join(R, S, float(parts[1]), MODE_RXS)) == _pairs_tok(toks), key
        elif parts[0] == "join_self_upper":
            assert pair_set(orc.join(R, None, float(parts[1]), MODE_SELF_UPPER)) == _pairs_tok(toks), key
    idx, d2 = orc.topk(R, S, 1)
    assert idx[:, 0].tolist() == [int(v) for v in e["top1"]]
    assert d2[:, 0].tolist() == [float(v) for v in e["top1_d2"]]
    idx, d2 = orc.topk(R, S, 2)
    assert [tuple(r) for r in idx.tolist()] == [tuple(int(v) for v in t.split(",")) for t in e["top2"]]
    assert [tuple(r) for r in d2.tolist()] == [tuple(float(v) for v in t.split(",")) for t in e["top2_d2"]]
    idx, d2 = orc.topk(Q, T, 3)
    assert idx[0].tolist() == [int(v) for v in e["topk_ties top3"]]
    assert d2[0].tolist() == [float(v) for v in e["topk_ties top3_d2"]]


def pin_boundary_closed_forms(orc):
    """Inclusive threshold at exact distances: one-hot rows and 2^-3 grids."""
    g = _g(13)
    X = W.one_hot_rows(g, 40, 16)
    same = {(i, j) for i in range(40) for j in range(40) if (X[i] == X[j]).all()}
    # fl(sqrt(2))^2 rounds to just above 2, so every distinct pair (D = 2) is kept.
    assert pair_set(orc.join(X, None, math.sqrt(2.0), MODE_SELF_FULL)) == \
        {(i, j) for i in range(40) for j in range(40)}
    assert pair_set(orc.join(X, None, 1.414, MODE_SELF_FULL)) == same
    # 1-D grid 0, 3/8, 6/8: eps = 3/8 exactly -> eps^2 = 9/64 exactly, neighbours kept.
    P = np.array([[0.0], [0.375], [0.75]], dtype=np.float32)
    assert pair_set(orc.join(P, None, 0.375, MODE_SELF_UPPER)) == {(0, 1), (1, 2)}
    assert pair_set(orc.join(P, None, float(np.nextafter(0.375, 0.0)), MODE_SELF_UPPER)) == set()
    # d-dim grid: eps^2 set exactly equal to one realised distance
    G = W.grid_points(g, 30, 6)
    M = exact_matrix(G, G)
    # pick a realised distance m/64 with m a perfect square, so eps = sqrt(m)/8 is exact
    hit = next((i, j) for i in range(30) for j in range(i + 1, 30)
               if M[i][j] > 0 and math.isqrt(int(M[i][j] * 64)) ** 2 == M[i][j] * 64)
    target = M[hit[0]][hit[1]]
    eps = math.isqrt(int(target * 64)) / 8.0
    assert Fraction(eps * eps) == target
    want = {(i, j) for i in range(30) for j in range(i + 1, 30) if M[i][j] <= target}
    assert hit in want
    assert pair_set(orc.join(G, None, eps, MODE_SELF_UPPER)) == want
    just_below = float(np.nextafter(eps, 0.0))
    assert hit not in pair_set(orc.join(G, None, just_below, MODE_SELF_UPPER))


def pin_self_join_symmetry_and_diagonal(orc):
    """Full mode is symmetric and holds every (i, i); upper mode is its i<j half."""
    g = _g(14)
    X = W.dirichlet_histograms(g, 120, 8)
    eps = 0.25
    full = pair_set(orc.join(X, None, eps, MODE_SELF_FULL))
    assert all((j, i) in full for (i, j) in full)
    assert all((i, i) in full for i in range(120))
    up = pair_set(orc.join(X, None, eps, MODE_SELF_UPPER))
    assert up == {(i, j) for (i, j) in full if i < j}
    assert pair_set(orc.join(X, X, eps, MODE_RXS)) == full


def pin_monotone_in_eps(orc):
    """eps1 < eps2 implies J(eps1) is a subset of J(eps2); eps=0 and eps=inf limits."""
    g = _g(15)
    R = W.grid_points(g, 50, 5, levels=4, dup_frac=0.2)
    S = np.concatenate([R[:10], W.grid_points(g, 30, 5, levels=4)])
    prev = None
    for eps in (0.0, 0.1, 0.2, 0.25, 0.3, 0.45, 0.6, 1.0):
        cur = pair_set(orc.join(R, S, eps, MODE_RXS))
        if prev is not None:
            assert prev <= cur, eps
        prev = cur
    dup = {(i, j) for i in range(R.shape[0]) for j in range(S.shape[0]) if (R[i] == S[j]).all()}
    assert pair_set(orc.join(R, S, 0.0, MODE_RXS)) == dup
    assert len(dup) >= 10
    assert pair_set(orc.join(R, S, math.inf, MODE_RXS)) == \
        {(i, j) for i in range(R.shape[0]) for j in range(S.shape[0])}


def pin_permutation_and_union(orc):
    """Row permutations map the result; J(R, S1 u S2) = J(R, S1) u J(R, S2)."""
    g = _g(16)
    R = W.dirichlet_histograms(g, 70, 6)
    S = W.dirichlet_histograms(g, 90, 6)
    eps = 0.3
    base = pair_set(orc.join(R, S, eps))
    pr = g.permutation(70)
    ps = g.permutation(90)
    perm = pair_set(orc.join(R[pr], S[ps], eps))
    assert {(int(pr[i]), int(ps[j])) for (i, j) in perm} == base
    a = pair_set(orc.join(R, S[:40], eps))
    b = {(i, j + 40) for (i, j) in pair_set(orc.join(R, S[40:], eps))}
    assert a | b == base


def pin_topk_matches_exact_order(orc):
    """Top-k equals the exact-rational order (distance, then index) on tiny inputs."""
    g = _g(17)
    Q = W.dirichlet_histograms(g, 9, 7)
    S = np.concatenate([W.dirichlet_histograms(g, 25, 7), W.dirichlet_histograms(g, 1, 7)])
    S = np.concatenate([S, S[3:6]])  # exact duplicates: ties broken by the smaller index
    M = exact_matrix(Q, S)
    for k in (1, 4, 11):
        idx, d2 = orc.topk(Q, S, k)
        for i in range(Q.shape[0]):
            order = sorted(range(S.shape[0]), key=lambda j: (M[i][j], j))[:k]
            assert idx[i].tolist() == order, (k, i)
            for t, j in enumerate(order):
                assert d2[i, t] == orc.sqdist(Q[i], S[j])
                assert abs(Fraction(float(d2[i, t])) - M[i][j]) <= Fraction(10, 2**53) * M[i][j]


def pin_topk_small_store_and_join_consistency(orc):
    """k >= |S| returns every row sorted; top-k rows lie inside the join at eps_k."""
    g = _g(18)
    Q = W.dirichlet_histograms(g, 6, 5)
    S = W.dirichlet_histograms(g, 7, 5)
    idx, d2 = orc.topk(Q, S, 10)
    D = orc.dist_block(Q, S)
    for i in range(6):
        order = sorted(range(7), key=lambda j: (D[i, j], j))
        assert idx[i, :7].tolist() == order
        assert (idx[i, 7:] == -1).all() and (d2[i, 7:] == -1.0).all()
    S2 = W.dirichlet_histograms(g, 60, 5)
    k = 5
    idx, d2 = orc.topk(Q, S2, k)
    for i in range(6):
        kth = d2[i, k - 1]
        eps = math.sqrt(kth)
        while eps * eps < kth:
            eps = float(np.nextafter(eps, math.inf))
        row = {j for (r, j) in pair_set(orc.join(Q[i:i + 1], S2, eps)) if r == 0}
        assert set(idx[i].tolist()) <= row


def _rn32(q: Fraction) -> Fraction:
    """The float32 nearest to the rational q (ties to even), as a rational (exact search)."""
    f = np.float32(float(q))   # within an ulp; then step to the exact nearest
    best = None
    for cand in (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))):
        c = Fraction(float(cand))
        key = (abs(c - q), int(np.frombuffer(np.float32(cand).tobytes(), dtype=np.uint32)[0]) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


def pin_normalize_exact_properties(orc):
    """Unit-normalized rows: RN quotients, unit norm within 5u, power-of-two scaling, zero rows."""
    # rows whose norm is exact (Pythagorean), so each output is the RN of an exact quotient
    X = np.array([[3, 4, 0], [0, -5, 12], [8, 0, 15], [-2, 3, 6]], dtype=np.float32)
    N = orc.normalize(X)
    for i, norm in enumerate((5, 13, 17, 7)):
        for k in range(3):
            assert Fraction(float(N[i, k])) == _rn32(Fraction(int(X[i, k]), norm)), (i, k)
    g = _g(19)
    for d in (1, 2, 5, 16, 77):
        Y = W.mixed_magnitude_rows(g, 20, d) if d < 77 else W.dirichlet_histograms(g, 20, d)
        Y = Y[np.abs(Y).max(axis=1) > 0]
        M = orc.normalize(Y)
        for i in range(M.shape[0]):
            s = sum(Fraction(float(v)) ** 2 for v in M[i].tolist())
            assert abs(s - 1) <= Fraction(5, 2**24), (d, i, float(s))
        for e in (-20, 3, 17):   # scaling by 2^e changes nothing
            assert np.array_equal(orc.normalize((Y.astype(np.float64) * 2.0 ** e).astype(np.float32)), M), (d, e)
    one_hot = W.one_hot_rows(g, 10, 6) * np.float32(-3.5)
    assert np.array_equal(orc.normalize(one_hot), -np.abs(one_hot) / np.float32(3.5))
    try:
        orc.normalize(np.zeros((2, 4), np.float32))
        raise AssertionError("a zero row must be rejected")
    except ValueError:
        pass


def pin_cosine_join_matches_exact(orc):
    """The cosine join equals the exact set on its rows, and agrees with the exact cosine."""
    g = _g(20)
    checked = 0
    for d, nR, nS in ((3, 15, 19), (8, 21, 17)):
        R = orc.normalize(W.mixed_magnitude_rows(g, nR, d))
        S = orc.normalize(W.mixed_magnitude_rows(g, nS, d))
        M = exact_matrix(R, S)
        vals = sorted({v for row in M for v in row})
        for rank in (len(vals) // 5, len(vals) // 2):
            a, b = vals[rank], vals[rank + 1]
            c = (2.0 - float((a + b) / 2)) / 2.0
            t = Fraction(2.0 - 2.0 * c)
            if not (a < t < b):
                continue
            want = {(i, j) for i in range(nR) for j in range(nS) if M[i][j] <= t}
            assert pair_set(orc.cosine_join(R, S, c, MODE_RXS)) == want, (d, rank)
            checked += 1
    assert checked >= 2
    # against the exact cosine of the raw rows (margin for the normalization rounding)
    Rraw = W.dirichlet_histograms(g, 30, 6)
    Sraw = W.dirichlet_histograms(g, 40, 6)
    c = 0.8
    got = pair_set(orc.cosine_join(orc.normalize(Rraw), orc.normalize(Sraw), c, MODE_RXS))
    margin = Fraction(1, 10**5)
    for i in range(30):
        for j in range(40):
            q = [Fraction(v) for v in Rraw[i].astype(np.float64).tolist()]
            x = [Fraction(v) for v in Sraw[j].astype(np.float64).tolist()]
            dot = sum(a * b for a, b in zip(q, x))
            nq, nx = sum(a * a for a in q), sum(b * b for b in x)
            hi, lo = (Fraction(c) + margin) ** 2, (Fraction(c) - margin) ** 2
            if dot > 0 and dot * dot >= hi * nq * nx:
                assert (i, j) in got, (i, j)
            if dot <= 0 or dot * dot <= lo * nq * nx:
                assert (i, j) not in got, (i, j)


# ----------------------------------------------------------------------------------------
# L1 / chi-square histogram distances
# ----------------------------------------------------------------------------------------

def exact_l1(q, x) -> Fraction:
    return sum((abs(Fraction(a) - Fraction(b)) for a, b in zip(q.tolist(), x.tolist())), Fraction(0))


def exact_chi2(q, x) -> Fraction:
    s = Fraction(0)
    for a, b in zip(q.tolist(), x.tolist()):
        fa, fb = Fraction(a), Fraction(b)
        if fa + fb > 0:
            s += (fa - fb) ** 2 / (fa + fb)
    return s


def _nonneg_rows(g, n, d):
    return np.abs(W.mixed_magnitude_rows(g, n, d)).astype(np.float32)


def pin_hist_dist_within_rounding_of_exact(orc):
    """|L1_64 - L1| <= (d+2) 2^-53 L1 and |chi2_64 - chi2| <= (d+6) 2^-53 chi2 (standard bounds)."""
    g = _g(31)
    for d in (1, 2, 5, 16, 33):
        for gen in (_nonneg_rows, lambda g, n, d: W.dirichlet_histograms(g, n, d)):
            X = gen(g, 5, d)
            for i in range(X.shape[0]):
                for j in range(X.shape[0]):
                    for metric, ex, slack in ((oracle.METRIC_L1, exact_l1, d + 2), (oracle.METRIC_CHI2, exact_chi2, d + 6)):
                        D = ex(X[i], X[j])
                        got = orc.hist_dist(X[i], X[j], metric)
                        if D == 0:
                            assert got == 0.0, (metric, d, i, j, got)
                        else:
                            assert abs(Fraction(got) - D) <= Fraction(slack, 2**53) * D, (metric, d, i, j, got, float(D))


def pin_dist_blocks_match_exact(orc):
    """The block forms equal the exact rational matrices, over any row range [r0, r1).

    oracle_dist_block and oracle_hist_dist_block fill an (r1 - r0) x |S| row-major matrix
    for rows r0 .. r1-1 of R. On 2^-3-grid rows every squared L2 and every L1 distance is
    exact in FP64, so each entry must equal the rational value itself; chi-square divides,
    so on histograms each entry lies within its standard bound (d+6) 2^-53 of the rational
    value. R and S differ in shape and content, so a transposed layout, a row offset
    dropped or doubled, the other operand, or the other metric each changes some entry.
    """
    g = _g(41)
    d = 6
    R = W.grid_points(g, 11, d)
    S = W.grid_points(g, 7, d)
    L2 = exact_matrix(R, S)
    L1 = [[exact_l1(R[i], S[j]) for j in range(7)] for i in range(11)]
    Hr = W.dirichlet_histograms(g, 9, d)
    Hs = W.dirichlet_histograms(g, 5, d)
    C2 = [[exact_chi2(Hr[i], Hs[j]) for j in range(5)] for i in range(9)]
    for r0, r1 in ((0, 11), (3, 8), (10, 11), (4, 4)):
        D = orc.dist_block(R, S, r0, r1)
        assert D.shape == (r1 - r0, 7), (r0, r1, D.shape)
        A = orc.hist_dist_block(R, S, oracle.METRIC_L1, r0, r1)
        assert A.shape == (r1 - r0, 7), (r0, r1, A.shape)
        for i in range(r0, r1):
            for j in range(7):
                assert Fraction(float(D[i - r0, j])) == L2[i][j], ("L2", r0, r1, i, j)
                assert Fraction(float(A[i - r0, j])) == L1[i][j], ("L1", r0, r1, i, j)
    for r0, r1 in ((0, 9), (2, 7), (8, 9)):
        X = orc.hist_dist_block(Hr, Hs, oracle.METRIC_CHI2, r0, r1)
        assert X.shape == (r1 - r0, 5), (r0, r1, X.shape)
        for i in range(r0, r1):
            for j in range(5):
                err = abs(Fraction(float(X[i - r0, j])) - C2[i][j])
                assert err <= Fraction(d + 6, 2**53) * C2[i][j], ("chi2", r0, r1, i, j)


def _thr_between(values, lo_rank: int):
    """A threshold strictly inside a wide gap of the exact values (no distance near it)."""
    vals = sorted(set(values))
    for r in range(max(0, lo_rank), len(vals) - 1):
        a, b = vals[r], vals[r + 1]
        if b - a > Fraction(1, 10**6) * max(b, Fraction(1, 10**30)):
            t = float((a + b) / 2)
            if a < Fraction(t) < b:
                return t, Fraction(t)
    raise AssertionError("no usable gap")


def pin_hist_join_matches_exact_rational(orc):
    """The L1 / chi-square joins (all modes) equal the exact-rational nested loop on tiny inputs."""
    g = _g(32)
    for metric, ex in ((oracle.METRIC_L1, exact_l1), (oracle.METRIC_CHI2, exact_chi2)):
        for d, nR, nS in ((1, 7, 9), (6, 13, 11), (12, 9, 14)):
            R = _nonneg_rows(g, nR, d) if d != 12 else W.dirichlet_histograms(g, nR, d)
            S = _nonneg_rows(g, nS, d) if d != 12 else W.dirichlet_histograms(g, nS, d)
            M = [[ex(R[i], S[j]) for j in range(nS)] for i in range(nR)]
            vals = [v for row in M for v in row]
            for rank in (0, len(vals) // 5, len(vals) // 2):
                t, ft = _thr_between(vals, rank)
                want = {(i, j) for i in range(nR) for j in range(nS) if M[i][j] <= ft}
                assert pair_set(orc.hist_join(R, S, t, metric, MODE_RXS)) == want, (metric, d, rank)
            MS = [[ex(R[i], R[j]) for j in range(nR)] for i in range(nR)]
            t, ft = _thr_between([MS[i][j] for i in range(nR) for j in range(nR) if i != j], nR)
            up = {(i, j) for i in range(nR) for j in range(i + 1, nR) if MS[i][j] <= ft}
            full = {(i, j) for i in range(nR) for j in range(nR) if MS[i][j] <= ft}
            assert pair_set(orc.hist_join(R, None, t, metric, MODE_SELF_UPPER)) == up, (metric, d)
            assert pair_set(orc.hist_join(R, None, t, metric, MODE_SELF_FULL)) == full, (metric, d)


def pin_hist_closed_forms(orc):
    """One-hot rows, histogram intersection, chi2(h, 0) = sum h, symmetry, chi2 <= L1."""
    d = 10
    E = np.eye(d, dtype=np.float32)
    for metric in (oracle.METRIC_L1, oracle.METRIC_CHI2):
        for i in range(d):
            for j in range(d):
                assert orc.hist_dist(E[i], E[j], metric) == (0.0 if i == j else 2.0), (metric, i, j)
        # distinct one-hot rows are exactly 2 apart: the inclusive threshold 2 keeps every pair
        assert len(orc.hist_join(E, None, 2.0, metric, MODE_SELF_UPPER)) == d * (d - 1) // 2
        assert len(orc.hist_join(E, None, float(np.nextafter(2.0, 0.0)), metric, MODE_SELF_UPPER)) == 0
    g = _g(33)
    # histograms on the 2^-10 grid summing to exactly 1: every FP64 step is exact
    for _ in range(40):
        a = g.multinomial(1024, g.dirichlet(np.full(d, 0.7))).astype(np.float32) / np.float32(1024)
        b = g.multinomial(1024, g.dirichlet(np.full(d, 0.7))).astype(np.float32) / np.float32(1024)
        inter = float(np.minimum(a, b).astype(np.float64).sum())
        assert orc.hist_dist(a, b, oracle.METRIC_L1) == 2.0 - 2.0 * inter
        assert orc.hist_dist(a, np.zeros(d, np.float32), oracle.METRIC_CHI2) == 1.0
        assert orc.hist_dist(np.zeros(d, np.float32), b, oracle.METRIC_CHI2) == 1.0
    X = np.concatenate([_nonneg_rows(g, 6, 9), W.dirichlet_histograms(g, 6, 9)])
    for i in range(X.shape[0]):
        for j in range(X.shape[0]):
            l1 = orc.hist_dist(X[i], X[j], oracle.METRIC_L1)
            c2 = orc.hist_dist(X[i], X[j], oracle.METRIC_CHI2)
            assert l1 == orc.hist_dist(X[j], X[i], oracle.METRIC_L1)
            assert c2 == orc.hist_dist(X[j], X[i], oracle.METRIC_CHI2)
            assert c2 <= l1 * (1 + 30 * 2.0**-53), (i, j, c2, l1)


def pin_hist_topk_order_ties_and_join(orc):
    """Histogram top-k: exact rational order where values are well separated, ties (duplicate
    rows) by the smaller store row, -1 past |S|, and the join's matches as a prefix."""
    g = _g(36)
    for metric, ex in ((oracle.METRIC_L1, exact_l1), (oracle.METRIC_CHI2, exact_chi2)):
        Q = W.dirichlet_histograms(g, 4, 7)
        S = W.dirichlet_histograms(g, 12, 7)
        S[9] = S[2]                      # a duplicate: equal distances, row 2 first
        k = 15
        idx, dist = orc.hist_topk(Q, S, k, metric)
        for i in range(Q.shape[0]):
            exact = [ex(Q[i], S[j]) for j in range(S.shape[0])]
            order = sorted(range(S.shape[0]), key=lambda j: (exact[j], j))
            assert idx[i, :12].tolist() == order, (metric, i)
            assert np.all(idx[i, 12:] == -1) and np.all(dist[i, 12:] == -1.0)
            assert np.all(np.diff(dist[i, :12]) >= 0)
            assert idx[i].tolist().index(2) < idx[i].tolist().index(9)
            t = float(dist[i, 5])
            m = orc.hist_join(Q[i:i + 1], S, t, metric, MODE_RXS)
            assert set(m[:, 1].tolist()) == set(idx[i, :len(m)].tolist())


def pin_inner_product_exact(orc):
    """The canonical dot product within (d+1) 2^-53 sum|q_k x_k| of the exact rational value
    (products exact in FP64); the inner-product join equal to the exact rational set in all
    three modes; on unit rows, consistent with the cosine join outside a small margin."""
    g = _g(37)
    for d in (1, 3, 16, 40):
        X = W.mixed_magnitude_rows(g, 6, d) * np.where(g.random((6, d)) < 0.5, -1, 1).astype(np.float32)
        for i in range(6):
            for j in range(6):
                ex = sum(Fraction(a) * Fraction(b) for a, b in zip(X[i].tolist(), X[j].tolist()))
                mag = sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(X[i].tolist(), X[j].tolist()))
                assert abs(Fraction(orc.dot(X[i], X[j])) - ex) <= Fraction(d + 1, 2**53) * mag, (d, i, j)
    R = W.dirichlet_histograms(g, 9, 6) - np.float32(1 / 6)
    S = W.dirichlet_histograms(g, 11, 6) - np.float32(1 / 6)
    M = [[sum(Fraction(a) * Fraction(b) for a, b in zip(R[i].tolist(), S[j].tolist())) for j in range(11)]
         for i in range(9)]
    vals = sorted(set(v for row in M for v in row))
    for r in (1, len(vals) // 3, len(vals) - 2):
        t = float((vals[r - 1] + vals[r]) / 2)
        want = {(i, j) for i in range(9) for j in range(11) if M[i][j] >= Fraction(t)}
        assert pair_set(orc.ip_join(R, S, t, MODE_RXS)) == want, r
    MS = [[sum(Fraction(a) * Fraction(b) for a, b in zip(R[i].tolist(), R[j].tolist())) for j in range(9)]
          for i in range(9)]
    t = float(np.median([float(MS[i][j]) for i in range(9) for j in range(9) if i != j]))
    assert pair_set(orc.ip_join(R, None, t, MODE_SELF_UPPER)) == \
        {(i, j) for i in range(9) for j in range(i + 1, 9) if MS[i][j] >= Fraction(t)}
    assert pair_set(orc.ip_join(R, None, t, MODE_SELF_FULL)) == \
        {(i, j) for i in range(9) for j in range(9) if MS[i][j] >= Fraction(t)}
    # inclusive threshold on an exact dyadic dot product: [0.5, 0.25] . [0.5, 0.5] = 0.375
    A = np.array([[0.5, 0.25]], dtype=np.float32)
    B = np.array([[0.5, 0.5]], dtype=np.float32)
    assert orc.dot(A[0], B[0]) == 0.375
    assert pair_set(orc.ip_join(A, B, 0.375, MODE_RXS)) == {(0, 0)}
    assert pair_set(orc.ip_join(A, B, float(np.nextafter(0.375, 1.0)), MODE_RXS)) == set()
    U = orc.normalize(W.dirichlet_histograms(g, 20, 8))
    c = 0.9
    ip = pair_set(orc.ip_join(U, None, c, MODE_SELF_UPPER))
    cs = pair_set(orc.cosine_join(U, None, c, MODE_SELF_UPPER))
    for i in range(20):
        for j in range(i + 1, 20):
            v = orc.dot(U[i], U[j])
            if abs(v - c) > 1e-5:
                assert ((i, j) in ip) == ((i, j) in cs) == (v >= c), (i, j)


# ----------------------------------------------------------------------------------------
# colour-histogram transformer
# ----------------------------------------------------------------------------------------

HIST_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "color_hist_small.txt")


def read_hist_golden(path=HIST_GOLDEN):
    frames = boxes = None
    cases, bins = [], None
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "frames":
            nF, H, Wd = map(int, tok[1:4])
            frames = np.zeros((nF, H, Wd, 3), dtype=np.uint8)
            boxes = []
        elif tok[0] == "pixels":
            f, y = int(tok[1]), int(tok[2])
            for x, px in enumerate(tok[4:]):
                frames[f, y, x] = [int(v) for v in px.split(",")]
        elif tok[0] == "box":
            boxes.append([int(v) for v in tok[1:6]])
        elif tok[0] == "bins":
            bins = tuple(int(v) for v in tok[1:4])
            cases.append((bins, {}))
        elif tok[0] == "counts":
            cases[-1][1][int(tok[1])] = [int(v) for v in tok[3:]]
    return frames, np.array(boxes, dtype=np.int32), cases


def pin_color_hist_golden_fixture(orc):
    """The hand-derived fixture: every box's histogram is its hand count over its area."""
    frames, boxes, cases = read_hist_golden()
    for bins, counts in cases:
        got = orc.color_hist(frames, boxes, bins)
        for b, cnt in counts.items():
            x0, y0, x1, y1 = boxes[b, 1:]
            area = np.float32((x1 - x0) * (y1 - y0))
            want = np.array(cnt, dtype=np.float32) / area
            assert np.array_equal(got[b], want), (bins, b, got[b], want)


def pin_color_hist_binning_definition(orc):
    """Each 8-bit value lands in the bin j with j*256/b <= v < (j+1)*256/b, channel by channel."""
    v = np.arange(256, dtype=np.uint8)
    for b in (1, 2, 3, 5, 7, 8, 16, 256):
        for ch, bins in ((0, (b, 1, 1)), (1, (1, b, 1)), (2, (1, 1, b))):
            frames = np.zeros((1, 1, 256, 3), dtype=np.uint8)
            frames[0, 0, :, ch] = v
            boxes = np.array([[0, x, 0, x + 1, 1] for x in range(256)], dtype=np.int32)
            got = orc.color_hist(frames, boxes, bins)
            for x in range(256):
                j = [jj for jj in range(b) if Fraction(jj * 256, b) <= x < Fraction((jj + 1) * 256, b)]
                assert len(j) == 1
                want = np.zeros(b, dtype=np.float32)
                want[j[0]] = 1.0
                assert np.array_equal(got[x], want), (b, ch, x)


def pin_color_hist_invariants(orc):
    """Counts sum to the area, adjacent boxes add up, pixel order inside a frame does not matter,
    a one-colour frame is one-hot at its colour's bin."""
    g = _g(34)
    nF, H, Wd = 3, 13, 21
    frames = g.integers(0, 256, size=(nF, H, Wd, 3), dtype=np.uint8)
    bins = (4, 3, 2)
    boxes = []
    for _ in range(30):
        f = int(g.integers(0, nF))
        x0, y0 = int(g.integers(0, Wd - 2)), int(g.integers(0, H - 1))
        x1, y1 = int(g.integers(x0 + 2, Wd + 1)), int(g.integers(y0 + 1, H + 1))
        xm = (x0 + x1) // 2
        boxes += [[f, x0, y0, x1, y1], [f, x0, y0, xm, y1], [f, xm, y0, x1, y1]]
    boxes = np.array(boxes, dtype=np.int32)
    h = orc.color_hist(frames, boxes, bins).astype(np.float64)
    area = ((boxes[:, 3] - boxes[:, 1]) * (boxes[:, 4] - boxes[:, 2])).astype(np.float64)
    cnt = np.rint(h * area[:, None])
    assert np.all(np.abs(h * area[:, None] - cnt) <= 1e-5 * area[:, None])
    assert np.array_equal(cnt.sum(axis=1), area)
    for t in range(0, len(boxes), 3):
        assert np.array_equal(cnt[t], cnt[t + 1] + cnt[t + 2]), t
    whole = np.array([[f, 0, 0, Wd, H] for f in range(nF)], dtype=np.int32)
    perm = frames.reshape(nF, H * Wd, 3)[:, g.permutation(H * Wd)].reshape(nF, H, Wd, 3)
    assert np.array_equal(orc.color_hist(frames, whole, bins), orc.color_hist(perm, whole, bins))
    one = np.zeros((1, H, Wd, 3), dtype=np.uint8)
    one[...] = (200, 90, 130)        # bins: 200 -> 3 of 4, 90 -> 1 of 3, 130 -> 1 of 2
    got = orc.color_hist(one, np.array([[0, 0, 0, Wd, H]], dtype=np.int32), bins)[0]
    want = np.zeros(24, dtype=np.float32)
    want[(3 * 3 + 1) * 2 + 1] = 1.0
    assert np.array_equal(got, want)
    for bad in ([1, 0, 0, 1, 1], [0, 0, 0, 0, 1], [0, 0, 0, Wd + 1, 1], [0, -1, 0, 1, 1], [0, 0, 2, 1, 2]):
        try:
            orc.color_hist(one, np.array([bad], dtype=np.int32), bins)
        except ValueError:
            continue
        raise AssertionError(f"invalid box accepted: {bad}")


# ----------------------------------------------------------------------------------------
# connected components and q4 deduplication
# ----------------------------------------------------------------------------------------

def _min_label_partition(n, pairs):
    """Components from scipy's graph routine, relabelled by the smallest member."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    A = sp.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    nc, lab = connected_components(A, directed=False)
    first = np.full(nc, n, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(n))
    return first[lab], nc


def pin_components_match_library(orc):
    """Random graphs (with self-loops and repeated edges) against scipy's connected components."""
    g = _g(35)
    for n, m in ((1, 0), (7, 0), (10, 4), (50, 30), (300, 250), (400, 900)):
        pairs = g.integers(0, n, size=(m, 2)) if m else np.empty((0, 2), np.int64)
        if m:
            pairs = np.concatenate([pairs, pairs[: m // 5], np.stack([pairs[:3, 0], pairs[:3, 0]], 1)])
        lab, c = orc.components(n, pairs)
        want, nc = _min_label_partition(n, pairs)
        assert c == nc and np.array_equal(lab, want), (n, m)
        assert np.all(lab <= np.arange(n)) and np.array_equal(lab[lab], lab)
        if len(pairs):
            assert np.array_equal(lab[pairs[:, 0]], lab[pairs[:, 1]])


def pin_components_closed_forms(orc):
    """A path listed back to front is one component labelled 0; no edges leave every row alone."""
    n = 64
    path = np.array([[i, i + 1] for i in range(n - 2, -1, -1)], dtype=np.int64)
    lab, c = orc.components(n, path)
    assert c == 1 and np.all(lab == 0)
    lab, c = orc.components(n, path[:, ::-1])
    assert c == 1 and np.all(lab == 0)
    lab, c = orc.components(n, np.empty((0, 2), np.int64))
    assert c == n and np.array_equal(lab, np.arange(n))
    # two interleaved paths: evens and odds
    ev = np.array([[i, i + 2] for i in range(n - 4, -1, -2)], dtype=np.int64)
    od = ev + 1
    lab, c = orc.components(n, np.concatenate([od, ev]))
    assert c == 2 and np.array_equal(lab, np.arange(n) % 2)
    try:
        orc.components(3, np.array([[0, 3]]))
    except ValueError:
        pass
    else:
        raise AssertionError("an edge outside [0, n) was accepted")


def pin_dedup_plans_hand_example(orc):
    """q4's two plan orders (Sec. 7.4.3) on a hand-built line of rows: 0-1 and 1-2 match, 0-2 do not."""
    X = np.array([[0.0], [1.0], [2.0], [10.0], [20.0], [21.0]], dtype=np.float32)
    P, C = 1, 2
    labels = np.array([P, C, P, P, C, C], dtype=np.int32)
    lab, c = orc.dedup(X, 1.0, plan=oracle.DEDUP_ALL)
    assert c == 3 and lab.tolist() == [0, 0, 0, 3, 4, 4]
    lab, c = orc.dedup(X, 1.0, labels, P, oracle.DEDUP_FILTER_MATCH)
    assert c == 3 and lab.tolist() == [0, -1, 2, 3, -1, -1]
    lab, c = orc.dedup(X, 1.0, labels, P, oracle.DEDUP_MATCH_FILTER)
    assert c == 2 and lab.tolist() == [0, 0, 0, 3, 4, 4]
    lab, c = orc.dedup(X, 1.0, labels, C, oracle.DEDUP_MATCH_FILTER)
    assert c == 2
    lab, c = orc.dedup(X, 1.0, labels, 7, oracle.DEDUP_FILTER_MATCH)
    assert c == 0 and np.all(lab == -1)


ALL_PINS = [
    pin_sqdist_within_rounding_of_exact,
    pin_join_matches_exact_rational,
    pin_golden_fixture,
    pin_boundary_closed_forms,
    pin_self_join_symmetry_and_diagonal,
    pin_monotone_in_eps,
    pin_permutation_and_union,
    pin_topk_matches_exact_order,
    pin_normalize_exact_properties,
    pin_cosine_join_matches_exact,
    pin_topk_small_store_and_join_consistency,
    pin_hist_dist_within_rounding_of_exact,
    pin_hist_join_matches_exact_rational,
    pin_hist_closed_forms,
    pin_dist_blocks_match_exact,
    pin_hist_topk_order_ties_and_join,
    pin_inner_product_exact,
    pin_color_hist_golden_fixture,
    pin_color_hist_binning_definition,
    pin_color_hist_invariants,
    pin_components_match_library,
    pin_components_closed_forms,
    pin_dedup_plans_hand_example,
]
