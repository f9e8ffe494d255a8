"""The numerical scheme behind the tensor-core products, re-derived in numpy
(CPU only; it shares nothing with the kernels): signed 7-bit digits of
power-of-two-scaled rows, exact integer pair products grouped by diagonal
t = p + q, pairs with t > TMAX dropped.  Checks the properties the kernels
rely on: every digit is an integer of magnitude <= 64 (exact in bf16), the
P-digit expansion reconstructs a row to half a unit of the grid
2^-(6 + 7 (P - 1)), the dropped pairs move a dot product by no more than
their bound, and over a chunk of 1024 products a diagonal of at most four
pairs stays below 2^24 (exact in the FP32 accumulator)."""
import numpy as np

B = 7


def pow2_ceil(v):
    v = abs(float(v))
    if v == 0.0:
        return 1.0
    m, e = np.frexp(v)
    return float(np.ldexp(1.0, e - 1 if m == 0.5 else e))


def digits(row, P):
    """Balanced digits of row / pow2_ceil(max |row|), most significant first."""
    sc = pow2_ceil(np.max(np.abs(row)))
    r = np.asarray(row, dtype=np.float64) / sc * 2.0 ** (B - 1)   # exact (powers of two)
    out = []
    for _ in range(P):
        d = np.rint(r)
        out.append(d)
        r = (r - d) * 2.0 ** B
    return np.array(out), sc


def weight(p):
    """Value of one unit of digit p (1-based) on the scaled row."""
    return 2.0 ** -(B - 1 + B * (p - 1))


def test_digits_are_small_integers_and_reconstruct_to_the_grid():
    rng = np.random.default_rng(7)
    for P in (5, 6):
        for row in (rng.uniform(0, 1, 784).astype(np.float32).astype(np.float64),
                    rng.standard_normal(300),
                    rng.uniform(-1, 1, 1000) * 1e-3):
            d, sc = digits(row, P)
            assert np.all(d == np.rint(d)) and np.max(np.abs(d)) <= 2 ** (B - 1)
            rec = sum(d[p] * weight(p + 1) for p in range(P)) * sc
            grid = weight(P) * sc
            assert np.max(np.abs(rec - row)) <= 0.5 * grid * (1 + 1e-12)


def test_dropped_pairs_stay_within_their_bound():
    rng = np.random.default_rng(11)
    n, P, TMAX = 784, 6, 7
    x = np.where(rng.uniform(size=n) < 0.8, 0.0, rng.uniform(size=n)).astype(np.float32)
    w = rng.uniform(-1, 1, n)
    dx, sx = digits(x.astype(np.float64), P)
    dw, sw = digits(w, P)
    # exact integer products per diagonal t = p + q (p, q 1-based), as Python ints
    kept = 0
    for p in range(1, P + 1):
        for q in range(1, P + 1):
            if p + q > TMAX:
                continue
            s = int(np.dot(dx[p - 1].astype(np.int64), dw[q - 1].astype(np.int64)))
            kept += s * 2 ** (B * (2 * P - p - q))              # common denominator
    approx = kept / 2.0 ** (B * (2 * P - 2) + 2 * (B - 1)) * sx * sw
    exact_digits = np.dot(sum(dx[p] * weight(p + 1) for p in range(P)),
                          sum(dw[q] * weight(q + 1) for q in range(P))) * sx * sw
    # the dropped pairs: |d| <= 64 each, n products, weight 2^-(2(B-1) + B(t-2))
    bound = sum(n * 2 ** (2 * (B - 1)) * 2.0 ** -(2 * (B - 1) + B * (p + q - 2))
                for p in range(1, P + 1) for q in range(1, P + 1) if p + q > TMAX) * sx * sw
    assert abs(approx - exact_digits) <= bound
    # and the digits' own truncation: both rows on their grids
    grid_err = n * (0.5 * weight(P) * sx * np.max(np.abs(w)) + 0.5 * weight(P) * sw * sx)
    assert abs(approx - np.dot(x.astype(np.float64), w)) <= bound + grid_err
    # per product the dropped pairs weigh less than 6 units of 2^-42 (five pairs on
    # the first dropped diagonal, then a geometric tail): about 1e-12 of |x_k w_k|'s scale
    assert bound / (sx * sw) < n * 6 * 2.0 ** -42


def test_four_pair_diagonals_are_exact_in_fp32_over_a_chunk():
    # worst case: every digit at its largest magnitude, 1024 products, 4 pairs
    worst = 4 * 1024 * (2 ** (B - 1)) ** 2
    assert worst <= 2 ** 24
    # a diagonal of five pairs may exceed 2^24; the scheme accepts one FP32
    # rounding there because its weight is at most 2^-(4B) of the leading one
    assert 5 * 1024 * (2 ** (B - 1)) ** 2 > 2 ** 24
    rng = np.random.default_rng(3)
    a = rng.integers(-64, 65, size=(4, 1024)).astype(np.float32)
    b = rng.integers(-64, 65, size=(4, 1024)).astype(np.float32)
    acc = np.float32(0.0)
    for k in range(1024):
        for p in range(4):
            acc = np.float32(acc + np.float32(a[p, k] * b[p, k]))
    assert int(acc) == int(np.sum(a.astype(np.int64) * b.astype(np.int64)))


# ---------------------------------------------------------------------------
# The FP64-accurate Gram (ELM_PREC_FP64_TC): eight digits, every pair of
# weight above 2^-68 (p + q <= 9), split into the bands of diagonals 2..5
# and 6..9 that the two tensor-core launches sum.
EX_P, EX_TMAX = 8, 9
BANDS = ((2, 5, 4, 1024), (6, 9, 8, 512))      # (first, last diagonal, planes, K chunk)


def test_exact_gram_bands_cover_every_kept_pair_once():
    kept = {(p, q) for p in range(1, EX_P + 1) for q in range(1, EX_P + 1) if p + q <= EX_TMAX}
    seen = []
    for t0, t1, planes, _ in BANDS:
        for p in range(1, planes + 1):
            for q in range(1, planes + 1):
                if t0 <= p + q <= t1:
                    seen.append((p, q))
    assert sorted(seen) == sorted(kept) and len(seen) == 36


def test_exact_gram_band_partial_sums_fit_fp32():
    """The largest partial sum of one diagonal over one K chunk: at most
    (pairs on the diagonal) x 2^12 x chunk, which must stay within 2^24."""
    for t0, t1, planes, chunk in BANDS:
        for t in range(t0, t1 + 1):
            pairs = sum(1 for p in range(1, planes + 1) if 1 <= t - p <= planes)
            assert pairs * 2 ** 12 * chunk <= 2 ** 24, (t, pairs, chunk)


def test_exact_gram_is_fp64_accurate():
    """Band sums in exact integers, one FP64 conversion per band, against the
    exact Gram in rational arithmetic.  The digits hold each element to
    2^-56 of its row's scale sc (the FP64 value rounded once on that grid),
    the dropped pairs (p + q >= 10) weigh at most 7.1 2^-56 sc_j sc_k per
    product, and each band is rounded once to FP64 (two roundings of u):
        |G' - G|_jk <= 2u sum|h_ij h_ik| + 2^-56 (sc_j sum|h_ik| + sc_k sum|h_ij|)
                       + (7.1 + 2^-56) n 2^-56 sc_j sc_k.
    For rows of similar magnitude this is the FP64 dot-product level, without
    its factor n on the first term; rows spanning many binades are held
    relative to their largest element.  Rows of sigmoid and tanh values, of
    values spread over twenty binades and of values near 1e-7."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    n = 300
    cols = [1.0 / (1.0 + np.exp(-rng.normal(0, 3, n))),
            np.tanh(rng.normal(0, 4, n)),
            rng.normal(0, 1, n) * np.exp(rng.uniform(-20, 0, n)),
            rng.uniform(-1, 1, n) * 1e-7]
    Hc = np.stack(cols)                    # rows of the matrix the kernel slices
    D, S = [], []
    for row in Hc:
        d, sc = digits(row, EX_P)
        D.append(d.astype(np.int64))
        S.append(sc)
    u = 2.0 ** -53
    for j in range(len(cols)):
        for k in range(len(cols)):
            total = 0.0
            for t0, t1, planes, _ in BANDS:
                acc = 0                    # int64 running sum of the band, as the drains keep it
                for t in range(t0, t1 + 1):
                    s_t = sum(int(np.dot(D[j][p - 1], D[k][t - p - 1]))
                              for p in range(1, planes + 1) if 1 <= t - p <= planes)
                    acc += s_t * 2 ** (B * (t1 - t))
                unit = 2.0 ** (-2 * (B - 1)) * 2.0 ** (-B * (t1 - 2))
                total += float(acc) * unit * S[j] * S[k]
            exact = sum(Fraction(a) * Fraction(b) for a, b in zip(Hc[j], Hc[k]))
            g = 2.0 ** -56
            bound = (2 * u * float(np.sum(np.abs(Hc[j] * Hc[k])))
                     + g * (S[j] * float(np.sum(np.abs(Hc[k]))) + S[k] * float(np.sum(np.abs(Hc[j]))))
                     + (7.1 + g) * n * g * S[j] * S[k])
            err = abs(Fraction(total) - exact)
            assert err <= Fraction(bound), (j, k)
            # and in practice far inside it: below the FP64 dot-product level
            # of the row scales
            assert float(err) <= 4 * u * np.sqrt(n) * S[j] * S[k], (j, k)
