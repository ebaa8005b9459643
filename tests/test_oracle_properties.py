"""Randomised properties of the oracle's further functions (CPU only).

Each property follows from the definitions in the paper's terms, not from the oracle's code:
the histogram distances are metrics-like (zero on equal rows, symmetric, L1 obeys the
triangle inequality up to rounding), the colour histogram of a box is the sum of the
histograms of any split of it, and connected components are invariant under relabelling
the edge list (order, orientation, duplicates).
"""

import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

ORC = oracle.default()


def _rows(seed, n, d, kind):
    g = np.random.default_rng(seed)
    if kind == 0:
        return g.dirichlet(np.full(d, 0.5), size=n).astype(np.float32)
    return np.abs(g.standard_normal((n, d)) * np.exp2(g.integers(-8, 8, size=(n, 1)))).astype(np.float32)


@settings(max_examples=60, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), d=st.integers(1, 40), kind=st.integers(0, 1))
def test_hist_distances_metric_properties(seed, d, kind):
    X = _rows(seed, 3, d, kind)
    a, b, c = X
    for m in (oracle.METRIC_L1, oracle.METRIC_CHI2):
        assert ORC.hist_dist(a, a, m) == 0.0
        assert ORC.hist_dist(a, b, m) == ORC.hist_dist(b, a, m)
        assert ORC.hist_dist(a, b, m) >= 0.0
    ab, bc, ac = (ORC.hist_dist(x, y, oracle.METRIC_L1) for x, y in ((a, b), (b, c), (a, c)))
    assert ac <= (ab + bc) * (1 + 4 * (d + 2) * 2.0**-53)


@settings(max_examples=40, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), h=st.integers(1, 9), w=st.integers(1, 13),
       bins=st.sampled_from([(1, 1, 1), (2, 2, 2), (4, 3, 2), (8, 4, 4), (3, 5, 7)]))
def test_color_hist_split_additivity(seed, h, w, bins):
    g = np.random.default_rng(seed)
    frames = g.integers(0, 256, size=(1, h, w, 3), dtype=np.uint8)
    box = [0, 0, 0, w, h]
    parts = [box]
    if w > 1:
        xm = int(g.integers(1, w))
        parts += [[0, 0, 0, xm, h], [0, xm, 0, w, h]]
    hist = ORC.color_hist(frames, np.array(parts, dtype=np.int32), bins).astype(np.float64)
    area = np.array([(p[3] - p[1]) * (p[4] - p[2]) for p in parts], dtype=np.float64)
    counts = np.rint(hist * area[:, None])
    assert counts[0].sum() == area[0]
    if len(parts) == 3:
        assert np.array_equal(counts[0], counts[1] + counts[2])


@settings(max_examples=60, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(1, 60), m=st.integers(0, 120))
def test_components_invariant_under_edge_relabelling(seed, n, m):
    g = np.random.default_rng(seed)
    e = g.integers(0, n, size=(m, 2)).astype(np.int64)
    lab, c = ORC.components(n, e)
    shuffled = e[g.permutation(m)][:, ::-1] if m else e
    lab2, c2 = ORC.components(n, np.concatenate([shuffled, shuffled[: m // 3]]))
    assert c == c2 and np.array_equal(lab, lab2)
    # every label is the smallest row of its class, and edges join equal labels
    assert np.all(lab <= np.arange(n))
    if m:
        assert np.array_equal(lab[e[:, 0]], lab[e[:, 1]])
