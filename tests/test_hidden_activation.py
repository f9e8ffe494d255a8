"""The activation of the mixed form's fused hidden-layer epilogue (Eq. 1,
H = g(XW + b) with g the logistic function or tanh), re-derived in numpy
with IEEE float32 operations (CPU only; shares nothing with the kernel).

The epilogue evaluates g on a double-float argument u = h + l (about 2^-44
relative) without FP64 instructions: a table holds sigma and sigma' as
double-float pairs at z_k = -40 + k/64, and a fourth-order Taylor expansion
in d = u - z_k (|d| <= 2^-7) adds the rest, with the terms beyond the linear
one in float32; tanh u = 2 sigma(2u) - 1.  Checked here against float64
sigma and tanh: the absolute error stays below 2^-39.5 (sigma) and 2^-38.5
(tanh) over the whole argument range, including the table's ends, the
midpoints between grid points and arguments beyond +-40 (measured worst
2^-40.4 and 2^-39.4, near |u| = 1.4, where the float32 roundings of the
higher-order terms, which stay below 2^-18, add up)."""
import math
from fractions import Fraction

import numpy as np

f32 = np.float32
SIG_N = 5121


def rn32(q):
    f = f32(float(q))
    best = None
    for c in (np.nextafter(f, f32(-np.inf)), f, np.nextafter(f, f32(np.inf))):
        k = (abs(Fraction(float(c)) - q), int(np.frombuffer(f32(c).tobytes(), np.uint32)[0]) & 1)
        if best is None or k < best[0]:
            best = (k, c)
    return best[1]


def fmaf(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def df_add(x, y):
    s = two_sum(x[0], y[0])
    return fast_two_sum(s[0], f32(f32(s[1] + x[1]) + y[1]))


def df_mul(x, y):
    p = f32(x[0] * y[0])
    e = fmaf(x[0], y[0], -p)
    e = fmaf(x[0], y[1], fmaf(x[1], y[0], e))
    return fast_two_sum(p, e)


def table():
    z = -40.0 + np.arange(SIG_N) / 64.0
    s0 = 1.0 / (1.0 + np.exp(-z))
    s1 = s0 * (1.0 - s0)
    s0h, s1h = s0.astype(np.float32), s1.astype(np.float32)
    return np.stack([s0h, (s0 - s0h).astype(np.float32), s1h,
                     (s1 - s1h).astype(np.float32)], axis=1)


TAB = table()


def sigmoid_df(u):
    uh, ul = u
    if uh <= f32(-40):
        return f32(0), f32(0)
    if uh >= f32(40):
        return f32(1), f32(0)
    k = int(np.rint(f32(f32(uh + f32(40)) * f32(64))))
    k = min(max(k, 0), SIG_N - 1)
    z0 = f32(f32(k) * f32(0.015625) - f32(40))
    assert Fraction(float(z0)) == Fraction(k, 64) - 40
    assert float(uh) - float(z0) == float(f32(uh - z0))      # the difference is exact
    d = two_sum(f32(uh - z0), ul)
    t = TAB[k]
    lin = df_mul((t[2], t[3]), d)
    s, s1 = t[0], t[2]
    a2 = f32(s1 * fmaf(f32(-2), s, f32(1)))
    q6 = fmaf(f32(f32(6) * s), f32(s - f32(1)), f32(1))
    q12 = fmaf(f32(f32(12) * s), f32(s - f32(1)), f32(1))
    a3, a4 = f32(s1 * q6), f32(a2 * q12)
    dh = d[0]
    inner = fmaf(dh, f32(a4 * f32(1 / 24)), f32(a3 * f32(1 / 6)))
    hot = f32(f32(dh * dh) * fmaf(dh, inner, f32(f32(0.5) * a2)))
    h = df_add((t[0], t[1]), lin)
    return fast_two_sum(h[0], f32(h[1] + hot))


def tanh_df(u):
    sg = sigmoid_df((f32(2 * u[0]), f32(2 * u[1])))
    return df_add((f32(2 * sg[0]), f32(2 * sg[1])), (f32(-1), f32(0)))


def pair(v):
    h = f32(v)
    return h, f32(v - float(h))


def arguments(seed):
    rng = np.random.default_rng(seed)
    u = list(rng.uniform(-42.0, 42.0, 1500))
    u += list(rng.normal(0.0, 3.0, 1500))
    grid = -40.0 + rng.integers(0, SIG_N, 300) / 64.0
    u += list(grid) + list(grid + 2.0 ** -7) + list(grid - 2.0 ** -7)   # midpoints
    u += [-40.0, 40.0, -39.999, 39.999, -40.001, 40.001, 0.0, 1e-30, -1e-30, 50.0, -50.0]
    return u


def test_logistic_within_2_pow_minus_39_5():
    worst = 0.0
    for v in arguments(1):
        h, l = pair(v)
        x = float(h) + float(l)
        y = sigmoid_df((h, l))
        ref = 1.0 / (1.0 + math.exp(-x)) if x > -700 else 0.0
        worst = max(worst, abs(float(y[0]) + float(y[1]) - ref))
    assert worst <= 2.0 ** -39.5, worst


def test_tanh_within_2_pow_minus_38_5():
    worst = 0.0
    for v in arguments(2):
        h, l = pair(v / 2)
        x = float(h) + float(l)
        y = tanh_df((h, l))
        worst = max(worst, abs(float(y[0]) + float(y[1]) - math.tanh(x)))
    assert worst <= 2.0 ** -38.5, worst


def test_taylor_terms_beyond_the_linear_one_are_small():
    # a2 d^2/2 + a3 d^3/6 + a4 d^4/24 over the table with |d| <= 2^-7: the
    # float32 evaluation of these terms costs a few 2^-24 of this
    s = TAB[:, 0].astype(np.float64)
    s1 = s * (1 - s)
    a2, a3 = s1 * (1 - 2 * s), s1 * (1 - 6 * s + 6 * s * s)
    a4 = a2 * (1 - 12 * s + 12 * s * s)
    d = 2.0 ** -7
    hot = np.abs(a2) * d * d / 2 + np.abs(a3) * d ** 3 / 6 + np.abs(a4) * d ** 4 / 24
    assert hot.max() < 2.0 ** -18
