"""The double-float exponential of the Newton fit (csrc/df64.cuh), checked on
the CPU: every entry of its 2^(j/256) table against 50-digit decimal values,
and the algorithm itself (the same float32 operations, with fused
multiply-adds formed exactly in float64 before rounding) against decimal exp
for arguments across the fit's range. No GPU code runs here."""
import math
import os
import re
from decimal import Decimal, getcontext

import numpy as np

HERE = os.path.dirname(__file__)
SRC = os.path.join(HERE, "..", "paper_2109_06743_gb300", "csrc", "df64.cuh")
f32 = np.float32


def table():
    src = open(SRC).read()
    body = src.split("kExp2Frac[257] = {")[1].split("};")[0]
    return [(f32(float(a)), f32(float(b))) for a, b in re.findall(r"\{([-0-9.e+]+)f, ([-0-9.e+]+)f\}", body)]


def constants():
    src = open(SRC).read()
    fn = src.split("df2 df2_exp(df2 x)")[1].split("\n}\n")[0]
    ln2 = re.search(r"ln2 = \{([-0-9.e+]+)f, ([-0-9.e+]+)f\}", fn).groups()
    ln2_256 = re.search(r"ln2_256 = \{([-0-9.e+]+)f, ([-0-9.e+]+)f\}", fn).groups()
    inv = re.search(r"k256InvLn2 = ([-0-9.e+]+)f", fn).group(1)
    return tuple(f32(float(v)) for v in ln2), tuple(f32(float(v)) for v in ln2_256), f32(float(inv))


def test_table_entries_are_the_double_float_pairs_of_two_to_j_over_256():
    getcontext().prec = 50
    ln2 = Decimal(2).ln()
    tab = table()
    assert len(tab) == 257
    for j, (hi, lo) in zip(range(-128, 129), tab):
        exact = (ln2 * j / 256).exp()
        assert abs(Decimal(float(hi)) - exact) <= Decimal(2) ** -24 * exact  # hi is the rounded value
        assert abs(Decimal(float(hi)) + Decimal(float(lo)) - exact) <= Decimal(2) ** -47 * exact, j


# float32 arithmetic with round-to-nearest; fma(a, b, c) rounds once (a * b is
# exact in float64 for float32 operands)
def fadd(a, b):
    return f32(f32(a) + f32(b))


def fsub(a, b):
    return f32(f32(a) - f32(b))


def fmul(a, b):
    return f32(f32(a) * f32(b))


def fma(a, b, c):
    return f32(float(Decimal(float(a)) * Decimal(float(b)) + Decimal(float(c))))


def qts(a, b):
    s = fadd(a, b)
    return s, fsub(b, fsub(s, a))


def ts(a, b):
    s = fadd(a, b)
    bb = fsub(s, a)
    return s, fadd(fsub(a, fsub(s, bb)), fsub(b, bb))


def dadd(a, b):
    s = ts(a[0], b[0])
    t = ts(a[1], b[1])
    s = qts(s[0], fadd(s[1], t[0]))
    return qts(s[0], fadd(s[1], t[1]))


def dmul(a, b):
    p = fmul(a[0], b[0])
    e = fma(a[0], b[0], -p)
    e = fma(a[0], b[1], e)
    e = fma(a[1], b[0], e)
    return qts(p, e)


def df2_exp(x):
    (l2h, l2l), (l8h, l8l), k256 = constants()
    k = f32(np.rint(fmul(x[0], f32(1.4426950408889634))))
    p = fmul(k, l2h)
    e = fma(k, l2h, -p)
    r = dadd(x, tuple(-v for v in qts(p, fma(k, l2l, e))))
    jf = f32(min(max(np.rint(fmul(r[0], k256)), -128), 128))
    p = fmul(jf, l8h)
    e = fma(jf, l8h, -p)
    r = dadd(r, tuple(-v for v in qts(p, fma(jf, l8l, e))))
    rh = r[0]
    t = fma(rh, f32(1.0 / 120.0), f32(1.0 / 24.0))
    t = fma(rh, t, f32(1.0 / 6.0))
    t = fmul(fmul(t, fmul(rh, rh)), rh)
    r2 = dmul(r, r)
    s = dadd(r, (fmul(f32(0.5), r2[0]), fmul(f32(0.5), r2[1])))
    s = qts(s[0], fadd(s[1], t))
    T = table()[int(jf) + 128]
    s = dadd(T, dmul(T, s))
    sc = f32(2.0 ** int(k))
    return fmul(s[0], sc), fmul(s[1], sc)


def test_exp_algorithm_accuracy():
    getcontext().prec = 50
    rng = np.random.default_rng(2109)
    worst_small = worst_mid = 0.0
    for x in list(rng.uniform(-5, 5, 300)) + list(rng.uniform(-60, 60, 300)):
        hi = f32(x)
        lo = f32(rng.uniform(-1, 1) * abs(float(hi)) * 2.0 ** -25)
        ref = (Decimal(float(hi)) + Decimal(float(lo))).exp()
        y = df2_exp((hi, lo))
        rel = float(abs(Decimal(float(y[0])) + Decimal(float(y[1])) - ref) / ref)
        if abs(x) < 5:
            worst_small = max(worst_small, rel)
        else:
            worst_mid = max(worst_mid, rel)
    assert worst_small < 1e-14 and worst_mid < 3e-13, (worst_small, worst_mid)
    assert math.isfinite(worst_small)
