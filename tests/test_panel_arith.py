"""The scalar arithmetic of the pivot panel (Eq. 6, diagonal pivoting of the
Gram matrix), re-derived in Python with exact rationals and IEEE float32 /
float64 operations (CPU only; shares nothing with the kernels).

The panel compares diagonals as unsigned integer keys, so that the search
for the largest remaining diagonal runs on the integer pipes, and it takes
1/sqrt of each pivot without an FP64 divide or square root:

* a double's key orders like its value (NaN below everything);
* a double-float pair's key (the keys of h and l side by side) orders like
  h + l, both for pairs whose h is the rounded sum (every pair the
  double-float operations produce) and for pairs that truncate a double
  (the conversion that loads the equilibrated Gram), the two kinds that
  meet in one comparison;
* the conversion of a double to a truncated pair keeps it to 2^-47;
* the warp-wide choice takes the largest key, then the lowest original
  index, and the index word holds every accepted size;
* the FP64 reciprocal square root (a float seed, then one third-order step)
  is accurate to the last bit or two for any seed within the documented
  2-ulp error of the hardware's float reciprocal square root, and its
  double-float counterpart to about 2^-44.
"""
import os
import re
import struct
from fractions import Fraction

import numpy as np

f32 = np.float32
M64 = (1 << 64) - 1


def dbits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def dfrom(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def fbits(x):
    return struct.unpack("<I", struct.pack("<f", float(x)))[0]


def ffrom(b):
    return f32(struct.unpack("<f", struct.pack("<I", b))[0])


def dkey(v):
    b = dbits(v)
    if (b & 0x7FFFFFFFFFFFFFFF) > 0x7FF0000000000000:
        return 0
    return (~b & M64) if b >> 63 else (b | (1 << 63))


def fkey(f):
    b = fbits(f)
    return (~b & 0xFFFFFFFF) if b >> 31 else (b | 0x80000000)


def dfkey(h, l):
    if h != h:
        return 0
    return (fkey(h) << 32) | fkey(l)


def rn32(q):
    """A rational rounded to the nearest float32 (ties to even)."""
    f = f32(float(q))
    best = None
    for c in (np.nextafter(f, f32(-np.inf)), f, np.nextafter(f, f32(np.inf))):
        k = (abs(Fraction(float(c)) - q), fbits(c) & 1)
        if best is None or k < best[0]:
            best = (k, c)
    return best[1]


def fmaf(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def fma(a, b, c):
    # int / int true division rounds correctly to the nearest double
    q = Fraction(a) * Fraction(b) + Fraction(c)
    return q.numerator / q.denominator


def renorm(s, e):
    h = f32(s + e)
    return h, f32(e - f32(h - s))


def df_add(a, b):
    s = f32(a[0] + b[0])
    bb = f32(s - a[0])
    e = f32(f32(f32(a[0] - f32(s - bb)) + f32(b[0] - bb)) + f32(a[1] + b[1]))
    return renorm(s, e)


def df_mul(a, b):
    p = f32(a[0] * b[0])
    e = fmaf(a[0], b[0], -p)
    e = fmaf(a[0], b[1], e)
    e = fmaf(a[1], b[0], e)
    return renorm(p, e)


def d2df(v):
    """Truncated pair: h = v cut to 24 significant bits, l = the rest cut to
    24 bits (normal range)."""
    b = dbits(v)
    sgn = (b >> 63) << 31
    e = ((b >> 52) & 0x7FF) - 1023
    if e < -126:
        return f32(0), f32(0)
    h = ffrom(sgn | ((e + 127) << 23) | ((b >> 29) & 0x7FFFFF))
    m = b & 0x1FFFFFFF
    if m == 0:
        return h, f32(0)
    top = m.bit_length() - 1
    el = e - 52 + top
    if el < -126:
        return h, f32(0)
    mant = (m >> (top - 23)) & 0x7FFFFF if top >= 23 else (m << (23 - top)) & 0x7FFFFF
    return h, ffrom(sgn | ((el + 127) << 23) | mant)


def rn_pair(v):
    """Pair whose h is the rounded value (what TwoSum renormalisation gives)."""
    h = f32(v)
    return h, f32(v - float(h))


def rsqrtf_seeds(x):
    """Every float within 2 ulp of 1/sqrt(x): the documented error bound of
    the hardware's float reciprocal square root."""
    y = f32(1.0 / np.sqrt(float(x)))
    out = [y]
    lo = hi = y
    for _ in range(2):
        lo = np.nextafter(lo, f32(0))
        hi = np.nextafter(hi, f32(np.inf))
        out += [lo, hi]
    return out


def rsqrt64(v, seed_pick):
    """FP64 1/sqrt(v): float seed of v's leading 24 bits, then one third-order
    step y0 + y0 r (1/2 + 3/8 r) with r = 1 - v y0^2."""
    b = dbits(v)
    e = (b >> 52) - 1023
    vf = ffrom(((e + 127) << 23) | ((b >> 29) & 0x7FFFFF))
    y0f = seed_pick(rsqrtf_seeds(vf))
    yb = fbits(y0f)
    y0 = dfrom(((((yb >> 23) & 0xFF) - 127 + 1023) << 52) | ((yb & 0x7FFFFF) << 29))
    assert y0 == float(y0f)
    r = fma(-v, y0 * y0, 1.0)
    return fma(y0 * r, fma(0.375, r, 0.5), y0)


def df_rsqrt(v, y0):
    q = f32(y0 * y0)
    qe = fmaf(y0, y0, -q)
    r = df_add((f32(1), f32(0)), tuple(-x for x in df_mul(v, (q, qe))))
    rr = f32(r[0] + r[1])
    return renorm(y0, f32(f32(y0 * rr) * fmaf(f32(0.375), rr, f32(0.5))))


def sample_doubles(rng, n, emin, emax):
    e = rng.integers(emin, emax + 1, n)
    m = rng.uniform(1.0, 2.0, n)
    s = rng.choice([-1.0, 1.0], n)
    return s * np.ldexp(m, e)


def test_double_key_orders_like_the_value():
    rng = np.random.default_rng(1)
    v = list(sample_doubles(rng, 600, -1074, 1023))
    tiny = np.nextafter(0.0, 1.0)
    v += [0.0, -0.0, np.inf, -np.inf, tiny, -tiny, 2.2250738585072014e-308,
          np.finfo(np.float64).max, -np.finfo(np.float64).max, 1.0, np.nextafter(1.0, 2.0)]
    v = np.array(v)
    keys = np.array([dkey(x) for x in v], dtype=np.uint64)
    less = v[:, None] < v[None, :]
    k1 = np.broadcast_to(keys[:, None], less.shape)
    k2 = np.broadcast_to(keys[None, :], less.shape)
    assert np.all(k1[less] < k2[less])
    eq = v[:, None] == v[None, :]
    kd = k1.astype(np.float64) - k2.astype(np.float64)
    assert np.all(np.abs(kd[eq]) <= 1)            # -0 and +0 sit side by side
    assert dkey(np.nan) == 0 and dkey(-np.nan) == 0 and min(keys) > 0


def _pair_order(pairs):
    val = np.array([float(h) + float(l) for h, l in pairs])   # exact in float64
    keys = [dfkey(h, l) for h, l in pairs]
    for i in range(len(pairs)):
        for j in range(len(pairs)):
            if val[i] < val[j]:
                assert keys[i] < keys[j], (pairs[i], pairs[j])
            elif val[i] == val[j] and val[i] != 0:
                assert keys[i] == keys[j], (pairs[i], pairs[j])


def test_pair_key_orders_rounded_pairs_like_their_sum():
    rng = np.random.default_rng(2)
    base = sample_doubles(rng, 60, -100, 100)
    v = list(base)
    for x in base[:20]:                           # neighbours within one float ulp
        u = float(np.spacing(f32(x)))
        v += [x + k * u / 4 for k in (-3, -2, -1, 1, 2, 3)]
        v += [float(f32(x)) + u / 2, float(f32(x)) - u / 2]   # ties of the rounding
    for k in range(-3, 4):                        # around powers of two
        p = 2.0 ** k
        v += [p, p - p * 2.0 ** -25, p + p * 2.0 ** -24, p - p * 2.0 ** -26]
    pairs = [rn_pair(x) for x in v]
    for h, l in pairs:
        assert h == f32(float(h) + float(l))      # h is the rounded sum
    _pair_order(pairs)
    # the double-float operations hand back pairs of that kind
    ops = [rn_pair(x) for x in sample_doubles(rng, 80, -40, 40)]
    for a, b in zip(ops[:40], ops[40:]):
        for h, l in (df_add(a, b), df_mul(a, b)):
            assert h == f32(float(h) + float(l))


def test_pair_key_orders_truncated_pairs_like_their_sum():
    rng = np.random.default_rng(3)
    base = sample_doubles(rng, 60, -100, 100)
    v = list(base)
    for x in base[:20]:
        u = float(np.spacing(f32(x)))
        v += [x + k * u / 4 for k in (-3, -2, -1, 1, 2, 3)]
    _pair_order([d2df(x) for x in v])


def test_truncated_pair_keeps_the_double_to_2_47():
    rng = np.random.default_rng(4)
    for x in sample_doubles(rng, 3000, -70, 120):
        h, l = d2df(x)
        err = Fraction(x) - Fraction(float(h)) - Fraction(float(l))
        assert abs(err) < abs(Fraction(x)) * Fraction(1, 2 ** 47)
        # both parts truncate: same sign as x (or zero), |l| < ulp(h)
        assert h * x > 0 and l * x >= 0
        assert abs(float(l)) < float(np.spacing(abs(h)))


def test_fp64_reciprocal_square_root_from_any_seed_within_2_ulp():
    rng = np.random.default_rng(5)
    v = np.abs(sample_doubles(rng, 800, -125, 126))
    v = np.concatenate([v, [1.0, 2.0, 0.5, 4.0 - 2.0 ** -50, 2.0 ** -126, 2.0 ** 127 * 1.999]])
    worst = 0.0
    for x in v:
        for pick in range(5):
            y = rsqrt64(float(x), lambda s, p=pick: s[p])
            # |y^2 x - 1| is twice the relative error of y
            rel = abs(Fraction(y) ** 2 * Fraction(float(x)) - 1) / 2
            worst = max(worst, float(rel))
    assert worst <= 2.0 ** -52, worst


def test_double_float_reciprocal_square_root():
    rng = np.random.default_rng(6)
    v = np.abs(sample_doubles(rng, 400, -60, 60))
    worst = 0.0
    for x in v:
        pair = rn_pair(float(x))
        for y0 in rsqrtf_seeds(pair[0]):
            h, l = df_rsqrt(pair, y0)
            assert abs(l) <= float(np.spacing(abs(h))) / 2
            y = Fraction(float(h)) + Fraction(float(l))
            vv = Fraction(float(pair[0])) + Fraction(float(pair[1]))
            worst = max(worst, float(abs(y * y * vv - 1) / 2))
    # with |r| <= 2^-21 (a 2-ulp seed), four float roundings of size about
    # 2^-24 |y0 r / 2| and the double-float r (about 2^-46) bound the error
    # by 2^-43.8
    assert worst <= 2.0 ** -43.5, worst


def warp_best(keys, ords):
    """The panel's warp-wide choice: the largest 64-bit key by two 32-bit
    maximum reductions (high words, then low words among the lanes holding
    the largest high word), then the smallest ord among the lanes holding
    that key."""
    kh = [k >> 32 for k in keys]
    mh = max(kh)
    ml = max((k & 0xFFFFFFFF) if h == mh else 0 for k, h in zip(keys, kh))
    mk = (mh << 32) | ml
    return mk, min(o if k == mk else 0xFFFFFFFF for k, o in zip(keys, ords))


def test_warp_choice_takes_the_largest_diagonal_then_the_lowest_index():
    rng = np.random.default_rng(7)
    for trial in range(300):
        # few distinct diagonals, so that ties are common; keys of double-float pairs
        pool = [rn_pair(x) for x in np.abs(sample_doubles(rng, 4, -30, 5))]
        picks = rng.integers(0, len(pool), 32)
        keys = [dfkey(*pool[p]) for p in picks]
        orig = rng.permutation(16384)[:32]
        ords = [(int(g) << 14) | int(x) for g, x in zip(orig, rng.integers(0, 16384, 32))]
        mk, mo = warp_best(keys, ords)
        best = max(range(32), key=lambda i: (float(pool[picks[i]][0]) + float(pool[picks[i]][1]),
                                             -int(orig[i])))
        assert mk == keys[best] and mo == ords[best]


def test_candidate_order_word_holds_every_index():
    # ord = orig << 14 | x in 32 bits: both indices below 2^14 for every
    # accepted size, so the packing loses nothing and compares orig first
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "include", "elm.h")
    max_l = int(re.search(r"#define ELM_MAX_L (\d+)", open(hdr).read()).group(1))
    assert max_l <= 1 << 14
    hi = ((max_l - 1) << 14) | (max_l - 1)
    assert hi < 1 << 32
