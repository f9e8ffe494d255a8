"""The double-float refinement residual of the mixed form (the correction
step's R = T - H beta, whose H^T R drives the refinement of Eq. 5's least-
squares solution), re-derived in numpy with IEEE float32 operations (CPU
only; shares nothing with the kernel).

Each of a warp's 32 lanes accumulates the products H[i, j] beta[j] of its
neurons j = lane, lane + 32, ... into an unnormalised pair (s_h, s_l) with
TwoProduct by FMA and TwoSum, renormalises it, and the lanes combine their
pairs by a butterfly of double-float adds; the residual is T[i] minus that
sum, in double-float.  Checked here against exact rational arithmetic: the
error stays below 2^-47 of sum_j |H[i, j] beta[j]| (measured 2^-50 to 2^-53
for 64 to 1000 neurons; T's own truncation to a pair is part of the target),
which is what lets the refinement converge to the least-squares solution of
the double-float H.  The product H^T R of the same step sums each split of
the samples into one unnormalised pair; its error grows with the split's
length, pinned below as measured."""
import struct
from fractions import Fraction

import numpy as np

f32 = np.float32


def rn32(q):
    f = f32(float(q))
    best = None
    for c in (np.nextafter(f, f32(-np.inf)), f, np.nextafter(f, f32(np.inf))):
        k = (abs(Fraction(float(c)) - q), int(np.frombuffer(f32(c).tobytes(), np.uint32)[0]) & 1)
        if best is None or k < best[0]:
            best = (k, c)
    return best[1]


def fmaf(a, b, c):
    # float32 FMA: the float64 product is exact (two 24-bit significands);
    # the sum is rounded once, exactly, through rationals
    return rn32(Fraction(float(a) * float(b)) + Fraction(float(c)))


def renorm(s, e):
    h = f32(s + e)
    return h, f32(e - f32(h - s))


def df_add(a, b):
    s = f32(a[0] + b[0])
    bb = f32(s - a[0])
    e = f32(f32(f32(a[0] - f32(s - bb)) + f32(b[0] - bb)) + f32(a[1] + b[1]))
    return renorm(s, e)


def acc_prod(sh, sl, a, b):
    p = f32(a[0] * b[0])
    e = fmaf(a[0], b[0], -p)
    e = fmaf(a[0], b[1], e)
    e = fmaf(a[1], b[0], e)
    s = f32(sh + p)
    bb = f32(s - sh)
    sl = f32(sl + f32(f32(f32(sh - f32(s - bb)) + f32(p - bb)) + e))
    return s, sl


def pair(v):
    h = f32(v)
    return h, f32(v - float(h))


def trunc_pair(v):
    """The kernel's conversion of an FP64 target: h = v cut to 24 significant
    bits, l = the rest cut to 24 bits (normal range)."""
    def cut(x):
        b = struct.unpack("<Q", struct.pack("<d", x))[0] & ~((1 << 29) - 1)
        return struct.unpack("<d", struct.pack("<Q", b))[0]
    h = cut(v)
    return f32(h), f32(cut(v - h))


def residual_row(h_row, beta, t):
    lanes = []
    for lane in range(32):
        sh = sl = f32(0)
        for j in range(lane, len(h_row), 32):
            sh, sl = acc_prod(sh, sl, h_row[j], beta[j])
        lanes.append(renorm(sh, sl))
    o = 16
    while o:
        lanes = [df_add(lanes[k], lanes[k ^ o]) for k in range(32)]
        o >>= 1
    v = lanes[0]
    return df_add(trunc_pair(t), (-v[0], -v[1]))


def test_residual_within_2_pow_minus_47_of_the_products():
    rng = np.random.default_rng(3)
    worst = 0.0
    for case in range(6):
        L = [1000, 777, 64][case % 3]
        x = rng.normal(size=L)
        h_row = [pair(1.0 / (1.0 + np.exp(-v))) for v in x]           # sigmoid values
        beta = [pair(v) for v in rng.normal(scale=10.0 ** rng.integers(-3, 4), size=L)]
        exact_dot = sum(Fraction(float(a[0])) * Fraction(float(b[0])) +
                        Fraction(float(a[0])) * Fraction(float(b[1])) +
                        Fraction(float(a[1])) * Fraction(float(b[0])) +
                        Fraction(float(a[1])) * Fraction(float(b[1]))
                        for a, b in zip(h_row, beta))
        # a target close to the fit, so that the residual cancels heavily
        t = float(exact_dot) * (1.0 + 1e-9)
        tp = trunc_pair(t)
        assert abs(t - float(tp[0]) - float(tp[1])) < abs(t) * 2.0 ** -47
        r = residual_row(h_row, beta, t)
        got = Fraction(float(r[0])) + Fraction(float(r[1]))
        want = Fraction(float(tp[0])) + Fraction(float(tp[1])) - exact_dot
        scale = sum(abs((Fraction(float(a[0])) + Fraction(float(a[1]))) *
                        (Fraction(float(b[0])) + Fraction(float(b[1]))))
                    for a, b in zip(h_row, beta))
        worst = max(worst, float(abs(got - want) / scale))
    assert worst <= 2.0 ** -47, worst


def htr_element(h_col, r_col, chunk):
    """G[j] = sum_i H[i, j] R[i]: one thread per neuron and split of the
    samples, an unnormalised pair over the split's samples, each split's pair
    added into one double, the splits summed in order in FP64."""
    g = 0.0
    for i0 in range(0, len(h_col), chunk):
        sh = sl = f32(0)
        for h, r in zip(h_col[i0:i0 + chunk], r_col[i0:i0 + chunk]):
            sh, sl = acc_prod(sh, sl, h, r)
        g += float(sh) + float(sl)
    return g


def test_normal_equations_residual_grows_with_the_split_length():
    """The split's pair is never renormalised, so the low word's own
    roundings grow with the split length k: measured up to about k 2^-51.4 of
    sum |H R| when every product has one sign (2^-45 to 2^-51 with mixed
    signs, as a least-squares residual has), checked here against k 2^-50.
    Splits of 448, 1984 and 13184 samples: what the split count gives for
    2000 neurons on 60000 samples, 6000 on 100000 and 8000 on 500000."""
    rng = np.random.default_rng(5)
    for chunk, N, same_sign in ((64, 64, True), (448, 1344, False), (448, 448, True),
                                (1984, 3968, False), (1984, 1984, True), (13184, 13184, True)):
        h_col = [pair(1.0 / (1.0 + np.exp(-v))) for v in rng.normal(size=N)]
        r = rng.normal(scale=1e-4, size=N)
        if same_sign:
            r = np.abs(r)
        r_col = [pair(v) for v in r]
        F = [(Fraction(float(a[0])) + Fraction(float(a[1])),
              Fraction(float(b[0])) + Fraction(float(b[1]))) for a, b in zip(h_col, r_col)]
        exact = sum(a * b for a, b in F)
        scale = sum(abs(a * b) for a, b in F)
        got = htr_element(h_col, r_col, chunk)
        rel = float(abs(Fraction(got) - exact) / scale)
        assert rel <= chunk * 2.0 ** -50, (chunk, same_sign, rel)
