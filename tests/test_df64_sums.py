"""The double-float running sums and products of the Newton fit's edge pass
(csrc/newton.cuh), checked on the CPU with the same float32 operations
(fused multiply-adds rounded once, formed exactly in Decimal):

* Fast2Sum with the operands ordered (fmaxf / fminf for non-negative
  terms, a magnitude compare for any signs) gives TwoSum's sum and error
  bit for bit, and both are exact (Knuth's TwoSum; Dekker's Fast2Sum);
* the weighted terms as chained FMA-split products: M c = p1 + e1 exactly
  up to the rounding of the low part's product, and (p1 + e1) c = p2 + e2
  to double-float accuracy, for the centred integer weights c of a line;
* an unnormalised ratio chain r <- r x e (no renormalisation of the pair)
  keeps its low part within about one float ulp per step of its high part
  and the pair's value within the accuracy the fit needs (1e-11 n) over
  the longest line (24 cells).
No GPU code runs here."""
from decimal import Decimal, getcontext

import numpy as np
import pytest

from test_df64_exp import fadd, fma, fmul, fsub, ts

f32 = np.float32
getcontext().prec = 60


def fast2sum_nn(a, b):
    s = fadd(a, b)
    big, small = (a, b) if a >= b else (b, a)
    return s, fsub(small, fsub(s, big))


def fast2sum_mag(a, b):
    s = fadd(a, b)
    big, small = (a, b) if abs(a) >= abs(b) else (b, a)
    return s, fsub(small, fsub(s, big))


def D(x):
    return Decimal(float(x))


@pytest.mark.parametrize("signs", ["non_negative", "mixed"])
def test_ordered_fast2sum_is_two_sum(signs):
    rng = np.random.default_rng(7 if signs == "mixed" else 3)
    for _ in range(4000):
        # a running sum and a term over a wide range of exponents, as along a
        # Gaussian line walked from the box edge (the term may exceed the sum)
        a = f32(rng.uniform(0.5, 1.0) * 2.0 ** rng.integers(-40, 40))
        b = f32(rng.uniform(0.5, 1.0) * 2.0 ** (int(np.log2(a)) + rng.integers(-30, 30)))
        if signs == "mixed":
            a, b = f32(a * rng.choice([-1, 1])), f32(b * rng.choice([-1, 1]))
        s_ts, e_ts = ts(a, b)
        s_f, e_f = (fast2sum_nn if signs == "non_negative" else fast2sum_mag)(a, b)
        assert s_f == s_ts and e_f == e_ts, (a, b)
        assert D(s_f) + D(e_f) == D(a) + D(b)


def test_chained_products_split_exactly():
    rng = np.random.default_rng(11)
    for _ in range(3000):
        hi = f32(rng.uniform(0.5, 1.0) * 2.0 ** rng.integers(-60, 20))
        lo = f32(float(hi) * rng.uniform(-1, 1) * 2.0 ** -24)
        c = f32(rng.integers(-15, 16))
        p1 = fmul(hi, c)
        e1 = fma(hi, c, -p1)
        assert D(p1) + D(e1) == D(hi) * D(c)  # the product's rounding error, exactly
        e1 = fma(lo, c, e1)
        p2 = fmul(p1, c)
        e2 = fma(p1, c, -p2)
        assert D(p2) + D(e2) == D(p1) * D(c)
        e2 = fma(e1, c, e2)
        exact1 = (D(hi) + D(lo)) * D(c)
        exact2 = exact1 * D(c)
        scale = (D(hi) + D(lo)) * (abs(D(c)) + 1) ** 2
        assert abs(D(p1) + D(e1) - exact1) <= scale * Decimal(2) ** -47
        assert abs(D(p2) + D(e2) - exact2) <= scale * Decimal(2) ** -46
        assert p2 >= 0  # the S2 sum's terms are non-negative (ordered Fast2Sum by fmaxf / fminf)


def mul_raw(a, b):
    p = fmul(a[0], b[0])
    e = fma(a[0], b[0], -p)
    e = fma(a[0], b[1], e)
    e = fma(a[1], b[0], e)
    return p, e


def test_unnormalised_ratio_chain_stays_accurate():
    rng = np.random.default_rng(5)
    for _ in range(200):
        # one-cell ratio of a Gaussian line and its step factor exp(2 k_xx),
        # as double-float pairs (the nearest float and the remainder)
        r0 = Decimal(float(rng.uniform(0.05, 20.0)))
        ein = Decimal(float(rng.uniform(0.2, 0.999)))
        pair = lambda x: (f32(float(x)), f32(float(x - D(f32(float(x))))))  # noqa: E731
        r, e = pair(r0), pair(ein)
        exact = D(r[0]) + D(r[1])
        step = D(e[0]) + D(e[1])
        for k in range(1, 25):
            r = mul_raw(r, e)
            exact *= step
            assert abs(D(r[1])) <= k * Decimal(2) ** -23 * abs(D(r[0])), k
            assert abs(D(r[0]) + D(r[1]) - exact) <= 4 * Decimal(k * k) * Decimal(2) ** -48 * exact, k
            assert abs(D(r[0]) + D(r[1]) - exact) <= Decimal("1e-12") * exact
