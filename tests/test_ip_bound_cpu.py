"""The inner-product join's FP32 recheck bound, checked on the host.

`k_finalize_ip` (csrc/exact.cuh: warp_band_decide_ip) settles a band pair of q.x >= t with an
FP32 dot product S32 and A32 = sum_k |q_k x_k|, both accumulated with fmaf over 16-byte slices by
an 8-lane group (lane l takes slices l, l+8, ...) and reduced by xor shuffles (4, 2, 1). It
accepts when RD(S32 - B) >= RU32(t) and rejects when RU(S32 + B) < RD32(t), with
B = RU(cf A32 + ca), cf = (2d+16) 2^-24 and ca = d 2^-146 + 2^-149. Both decisions agree with
the canonical FP64 dot C (the oracle's) only if

    |S32 - q.x| + g64 A <= cf A32 + ca,   g64 = (d+4) 2^-53 >= |C - q.x| / A,

for the exact dot q.x and A = sum |q_k x_k|. This test emulates the group's arithmetic step
for step with correctly rounded float32 operations (each fmaf and each addition rounded once,
to nearest even, subnormals included) and checks the inequality against exact rationals on
signed, cancelling, wide-range and underflowing rows. A mutant that trusts the FP32 dot as
exact (cf = 0) shows that the test can fail.
"""

from fractions import Fraction

import numpy as np
import pytest

EMIN, P = -126, 24   # float32: smallest normal exponent, significand bits


def f32(x: Fraction) -> Fraction:
    """x rounded to the nearest float32 (ties to even), subnormals included (no overflow here)."""
    if x == 0:
        return Fraction(0)
    sgn = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()   # 2^e <= a < 2^(e+2)
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    q = max(e, EMIN) - (P - 1)   # quantum: ulp of a's binade, or of the subnormal range
    m = a / Fraction(2) ** q
    n = m.numerator // m.denominator
    r = m - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sgn * n * Fraction(2) ** q


def fma(a, b, c):
    return f32(a * b + c)


def add(a, b):
    return f32(a + b)


def group_dot(q, x):
    """S32 and A32 of one 8-lane group, in the kernel's order."""
    d = len(q)
    Q = [Fraction(float(v)) for v in q]
    X = [Fraction(float(v)) for v in x]
    sd, sa = [Fraction(0)] * 8, [Fraction(0)] * 8
    if d % 4 == 0:
        for gl in range(8):
            for i in range(gl, d // 4, 8):
                for j in range(4):
                    k = 4 * i + j
                    sd[gl] = fma(Q[k], X[k], sd[gl])
                    sa[gl] = fma(abs(Q[k]), abs(X[k]), sa[gl])
    else:
        for gl in range(8):
            for k in range(gl, d, 8):
                sd[gl] = fma(Q[k], X[k], sd[gl])
                sa[gl] = fma(abs(Q[k]), abs(X[k]), sa[gl])
    for o in (4, 2, 1):
        sd = [add(sd[l], sd[l ^ o]) for l in range(8)]
        sa = [add(sa[l], sa[l ^ o]) for l in range(8)]
    assert len(set(sd)) == 1 and len(set(sa)) == 1
    return sd[0], sa[0], Q, X


def slack(d, cf=None):
    cf = Fraction(2 * d + 16, 2 ** 24) if cf is None else cf
    return cf, Fraction(d, 2 ** 146) + Fraction(1, 2 ** 149)


def rows(seed):
    g = np.random.default_rng(seed)
    out = []
    for d in (4, 13, 64, 128, 260):
        out.append((g.standard_normal(d), g.standard_normal(d)))                      # signed
        q = g.standard_normal(d)
        out.append((q, -q * (1 + 1e-7 * g.standard_normal(d))))                       # cancelling
        out.append((g.standard_normal(d) * 2.0 ** g.integers(-40, 40, d),
                    g.standard_normal(d) * 2.0 ** g.integers(-40, 40, d)))            # wide range
        out.append((g.standard_normal(d) * 2.0 ** -70, g.standard_normal(d) * 2.0 ** -70))   # underflow
    return [(np.asarray(q, np.float32), np.asarray(x, np.float32)) for q, x in out]


@pytest.mark.parametrize("seed", [1, 2])
def test_ip_fp32_bound_covers_the_canonical_dot(seed):
    worst = 0.0
    for q, x in rows(seed):
        d = len(q)
        sd, sa, Q, X = group_dot(q, x)
        exact = sum(a * b for a, b in zip(Q, X))
        A = sum(abs(a * b) for a, b in zip(Q, X))
        cf, ca = slack(d)
        need = abs(sd - exact) + Fraction(d + 4, 2 ** 53) * A
        have = cf * sa + ca
        assert need <= have, (d, float(need), float(have))
        if have > 0:
            worst = max(worst, float(need / have))
    assert worst < 1.0


def test_mutant_trusting_the_fp32_dot_fails():
    g = np.random.default_rng(5)
    broke = 0
    for _ in range(12):
        d = 256
        q = g.standard_normal(d).astype(np.float32)
        x = g.standard_normal(d).astype(np.float32)
        sd, sa, Q, X = group_dot(q, x)
        exact = sum(a * b for a, b in zip(Q, X))
        A = sum(abs(a * b) for a, b in zip(Q, X))
        cf, ca = slack(d, Fraction(0))
        if abs(sd - exact) + Fraction(d + 4, 2 ** 53) * A > cf * sa + ca:
            broke += 1
    assert broke > 0
