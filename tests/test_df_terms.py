"""The error bound behind the root step's double-float strong terms,
checked on the host.

The lane-per-chunk kernel of the root solve evaluates alpha exp(-gamma
|x - s|^2) with pairs of floats (TwoSum / TwoProduct by FMA): u = x - s from
exact three-float forms of x and s, r2 and z = gamma r2 in double-float, and
exp(-z) = 2^(-k/1024) exp(-r) with a double-float table and a short
polynomial for |r| <= ln 2 / 2048.  The step accepts the result when
2^-42 sum |term| (1 + z) stays below its share of the Newton step's error
budget, so each term's relative error must stay below (1 + z) 2^-44 with
room.  This test restates that arithmetic operation by operation in numpy
float32 (FMA through exact rationals) and measures it against 150-bit
arithmetic on random points, vectors and gammas, including near-coincident
x and s (heavy cancellation in u)."""
import random
from fractions import Fraction

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mpmath.mp.prec = 150

f32 = np.float32

# ln 2 / 1024 = A + B + C, each the float nearest the remainder
LN2_A = f32(float.fromhex("0x1.62e43p-11"))
LN2_B = f32(float.fromhex("-0x1.05c61p-39"))
LN2_C = f32(float.fromhex("-0x1.950d88p-64"))


def fma(a, b, c):
    """a b + c rounded once to float32 (through an exact rational)."""
    v = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    return f32(float(v))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def two_prod(a, b):
    p = f32(a * b)
    return p, fma(a, b, -p)


def df_add(x, y):
    s = two_sum(x[0], y[0])
    return fast_two_sum(s[0], f32(s[1] + f32(x[1] + y[1])))


def df_mul(x, y):
    p = two_prod(x[0], y[0])
    return fast_two_sum(p[0], fma(x[0], y[1], fma(x[1], y[0], p[1])))


def split3(v):
    """v = h + m + l exactly (a double in three floats)."""
    h = f32(v)
    r = v - float(h)
    m = f32(r)
    return h, m, f32(r - float(m))


def _table():
    tab = []
    for t in range(1024):
        v = float(mpmath.power(2, -mpmath.mpf(t) / 1024))
        h = f32(v)
        tab.append((h, f32(v - float(h))))
    return tab


TAB = _table()


def df_term(x, s, alpha, gamma):
    """alpha exp(-gamma |x - s|^2) as the kernel computes it (hi, lo)."""
    r2 = (f32(0), f32(0))
    for xk, sk in zip(x, s):
        xa, xb, xc = split3(xk)
        s1, s2, s3 = split3(sk)
        a = two_sum(xa, -s1)
        b = two_sum(xb, -s2)
        m = two_sum(a[1], b[0])
        lo = f32(m[1] + f32(b[1] + f32(xc - s3)))
        h = two_sum(a[0], m[0])
        u = fast_two_sum(h[0], f32(h[1] + lo))
        p = two_prod(u[0], u[0])
        r2 = df_add(r2, fast_two_sum(p[0], fma(f32(2 * u[0]), u[1], p[1])))
    g1 = f32(gamma)
    z = df_mul((g1, f32(gamma - float(g1))), r2)
    kf = f32(np.rint(f32(z[0] * f32(1477.3197218702985))))
    ka = two_prod(kf, LN2_A)
    rr = two_sum(z[0], -ka[0])
    rr = fast_two_sum(rr[0], f32(f32(rr[1] + f32(z[1] - ka[1])) - fma(kf, LN2_B, f32(kf * LN2_C))))
    rh = rr[0]
    br = fma(rh, fma(rh, f32(1 / 24), f32(-1 / 6)), f32(0.5))
    one_r = two_sum(f32(1), -rh)
    er = fast_two_sum(one_r[0], f32(one_r[1] + fma(f32(rh * rh), br, -rr[1])))
    ki = int(kf)
    e = df_mul(TAB[ki & 1023], er)
    e = (f32(np.ldexp(e[0], -(ki >> 10))), f32(np.ldexp(e[1], -(ki >> 10))))
    a1 = f32(alpha)
    return df_mul((a1, f32(alpha - float(a1))), e), float(z[0])


def test_double_float_term_within_bound():
    random.seed(0)
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(1500):
        d = random.choice([3, 5, 7])
        gamma = random.choice([1.5, 4.0, 6.0, 0.7])
        x = [random.uniform(-3.2, 3.2) for _ in range(d)]
        rad = random.uniform(0, 2.5) / np.sqrt(gamma)
        dirv = rng.standard_normal(d)
        dirv /= np.linalg.norm(dirv)
        s = [x[k] + rad * dirv[k] * random.choice([1, 1, 1, 1e-3, 1e-6]) for k in range(d)]
        alpha = random.uniform(-3, 3)
        (hi, lo), z = df_term(x, s, alpha, gamma)
        r2 = sum((mpmath.mpf(a) - mpmath.mpf(b)) ** 2 for a, b in zip(x, s))
        exact = mpmath.mpf(alpha) * mpmath.exp(-mpmath.mpf(gamma) * r2)
        rel = float(abs(mpmath.mpf(float(hi)) + mpmath.mpf(float(lo)) - exact) / abs(exact))
        worst = max(worst, rel / ((1 + z) * 2 ** -44))
    # measured about 0.25 of the bound; the kernel's check doubles it again
    assert worst < 0.5
