"""The float-float stage of the exact decision: its error bound, checked on the host.

The GPU decides a band pair that the FP32 bound cannot place with a float-float sum of
sum_k (q_k - x_k)^2 built from FP32 error-free transformations (csrc/exact.cuh: TwoSum of
q_k and -x_k, the FMA error of th^2, the TwoSum chain of the squares with its errors
collected in FP32, the small parts summed in FP32, lanes k = l, l+32, ... merged by an xor
butterfly, the three parts added in FP64), and claims

    |S - D| <= (d+34)^2 2^-48 D + (d+1) 2^-146

for the exact D (the sum of squared differences in rational arithmetic). The thresholds
that accept or reject on S (eq. of the threshold predicate, Sec. 3.2) are sound only if
this holds, so this test emulates the kernel's arithmetic step for step in numpy float32
(round to nearest, like the _rn intrinsics; the FMA as one rounding of the exact float64
residual) and checks the bound against exact rationals on random, cancelling, wide-range
and underflowing rows. A mutant check shows the test can fail: dropping the cross term
2 th tl breaks the bound.
"""

from fractions import Fraction

import numpy as np
import pytest

F = np.float32


def two_sum(a, b):
    s = F(a + b)
    bv = F(s - a)
    av = F(s - bv)
    e = F(F(a - av) + F(b - bv))
    return s, e


def fma_residual(th, p):
    # fl32(th*th - p) with one rounding: th*th is exact in float64 (48 bits), and so is the
    # difference from its float32 rounding p
    return F(np.float64(th) * np.float64(th) - np.float64(p))


def ff_lane(q, x, lane, d, drop_cross=False):
    s, c, m = F(0), F(0), F(0)
    for k in range(lane, d, 32):
        th, tl = two_sum(q[k], F(-x[k]))
        p = F(th * th)
        pe = fma_residual(th, p)
        cross = F(F(th + th) * tl)
        m = F(m + (pe if drop_cross else F(pe + cross)))
        s, e = two_sum(s, p)
        c = F(c + e)
    return s, c, m


def ff_sq(q, x, drop_cross=False):
    """The kernel's float-float value S of sum (q - x)^2: 32 lanes, xor butterfly, FP64 end."""
    d = len(q)
    lanes = [list(ff_lane(q, x, l, d, drop_cross)) for l in range(32)]
    for o in (16, 8, 4, 2, 1):
        nxt = []
        for l in range(32):
            a, b = lanes[l], lanes[l ^ o]
            s, e = two_sum(a[0], b[0])
            nxt.append([s, F(F(a[1] + b[1]) + e), F(a[2] + b[2])])
        lanes = nxt
    assert all(ln == lanes[0] for ln in lanes), "butterfly lanes disagree"
    s, c, m = lanes[0]
    return (np.float64(s) + np.float64(c)) + np.float64(m)


def exact_d(q, x):
    return sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(q, x))


def bound(d, D):
    return Fraction((d + 34) ** 2, 2 ** 48) * D + Fraction(d + 1, 2 ** 146)


def rows(seed):
    g = np.random.default_rng(seed)
    out = []
    for d in (1, 3, 31, 64, 129, 256, 1000):
        # histogram-like rows and a near neighbour (the band's typical pair)
        q = g.dirichlet(np.ones(d)).astype(F)
        out.append((q, (q * (1 + 1e-3 * g.standard_normal(d))).astype(F)))
        # signed rows of unit scale
        out.append((g.standard_normal(d).astype(F), g.standard_normal(d).astype(F)))
        # heavy cancellation: x one ulp away from q in most coordinates
        q = (g.standard_normal(d) * 2.0 ** g.integers(-20, 20, d)).astype(F)
        out.append((q, np.nextafter(q, F(np.inf)).astype(F)))
        # wide dynamic range up to the domain limit 2^40
        q = (g.standard_normal(d) * 2.0 ** g.integers(-60, 40, d)).astype(F)
        x = (g.standard_normal(d) * 2.0 ** g.integers(-60, 40, d)).astype(F)
        out.append((q, x))
        # differences in the subnormal range of the squares
        q = (g.standard_normal(d) * 2.0 ** -70).astype(F)
        out.append((q, (q + F(2.0 ** -80) * g.standard_normal(d).astype(F)).astype(F)))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ff_sum_within_its_bound(seed):
    worst = 0.0
    for q, x in rows(seed):
        d = len(q)
        S = ff_sq(q, x)
        D = exact_d(q, x)
        err = abs(Fraction(float(S)) - D)
        b = bound(d, D)
        assert err <= b, (d, float(err), float(b))
        worst = max(worst, float(err / b))
    assert worst < 1.0


def test_ff_bound_is_far_tighter_than_fp32():
    # the point of the stage: at d = 256 the float-float zone is about 5e4 times narrower
    d = 256
    assert (d + 34) ** 2 * 2.0 ** -48 * 5e4 < (d + 8) * 2.0 ** -24


def test_mutant_without_cross_term_breaks_the_bound():
    g = np.random.default_rng(9)
    broke = 0
    for _ in range(20):
        d = 64
        # q - x inexact in FP32 (magnitudes far apart), so the TwoSum remainders are non-zero
        q = g.standard_normal(d).astype(F)
        x = (F(1e-3) * g.standard_normal(d)).astype(F)
        S = ff_sq(q, x, drop_cross=True)
        D = exact_d(q, x)
        if abs(Fraction(float(S)) - D) > bound(d, D):
            broke += 1
    assert broke > 0
