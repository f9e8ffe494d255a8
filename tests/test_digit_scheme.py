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
