"""The digit scheme of the mixed form's tensor-core trailing update (Eq. 6,
the Schur-complement update A - P^T P after each panel), re-derived in numpy
with IEEE float32 operations (CPU only; shares nothing with the kernel).

Each column's 32 panel entries, double-float pairs v = h + l, are scaled by
the smallest power of two s >= max |h| and split into six signed 8-bit
digits of weights 2^(-7-8j).  Checked here: the digits are integers of
magnitude <= 128 (exact in bf16) and reconstruct v / s to 2^-48; a diagonal
d = i + j of the pair products over 32 rows stays an integer below 2^22
(exact in an FP32 accumulator, in any order); the dropped pairs (i + j > 6)
move an entry by less than their bound; and the float32 fold of the seven
exact diagonal sums, scaled and subtracted from a double-float entry, meets
the double-float accuracy of the update it replaces.  The FP64 variant
(seven digits from an exact integer split, eight diagonals folded into two
47-bit integers and two FMAs) meets FP64 accuracy."""
from fractions import Fraction

import numpy as np

f32 = np.float32
NDIG, K = 6, 32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def rint_small(x):
    return f32(f32(x + f32(12582912.0)) - f32(12582912.0))


def df_pairs(v):
    """Double-float pairs of FP64 values: h = fl32(v), l = fl32(v - h)."""
    h = v.astype(np.float32)
    l = (v - h.astype(np.float64)).astype(np.float32)
    return h, l


def column_digits(h, l):
    """Scale (power of two) and the six digits of a column's entries, with the
    same float32 operations, in the same order, as the digit kernel."""
    m = np.max(np.abs(h))
    s = f32(1.0) if m == 0 else f32(2.0 ** int(np.ceil(np.log2(float(m)))))
    inv = f32(1.0) / s
    dig = np.zeros((NDIG, len(h)), dtype=np.float32)
    for k in range(len(h)):
        rh, rl = f32(f32(h[k] * inv) * f32(128.0)), f32(f32(l[k] * inv) * f32(128.0))
        for j in range(NDIG):
            a = rint_small(rh)
            rh, rl = two_sum(f32(rh - a), rl)
            rh, rl = f32(rh * f32(256.0)), f32(rl * f32(256.0))
            dig[j, k] = a
    return s, dig


def columns(seed, n, scale_spread=True):
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        v = rng.standard_normal(K) * (2.0 ** rng.integers(-30, 1) if scale_spread else 1.0)
        if c % 5 == 0:
            v[rng.integers(0, K, 8)] = 0.0       # pivots a panel did not take
        out.append(df_pairs(v))
    return out


def test_digits_are_bf16_integers_and_reconstruct_to_2_pow_minus_48():
    for h, l in columns(1, 40):
        s, d = column_digits(h, l)
        assert np.all(d == np.rint(d)) and np.max(np.abs(d)) <= 128
        w = 2.0 ** -(7 + 8 * np.arange(NDIG))
        rec = (d.astype(np.float64) * w[:, None]).sum(0)
        x = (h.astype(np.float64) + l.astype(np.float64)) / float(s)
        assert np.max(np.abs(rec - x)) <= 2.0 ** -48


def test_diagonal_sums_stay_below_2_pow_22():
    # worst case: every digit at its largest magnitude
    for dgl in range(NDIG + 1):
        pairs = sum(1 for i in range(NDIG) for j in range(NDIG) if i + j == dgl)
        assert pairs * K * 128 * 128 < 2 ** 22
    # and on data: the float32 sum in a shuffled order equals the integer sum
    rng = np.random.default_rng(3)
    cols = columns(4, 6)
    dig = [column_digits(h, l)[1] for h, l in cols]
    for x in range(len(dig)):
        for y in range(len(dig)):
            for dgl in range(NDIG + 1):
                terms = [dig[x][i, k] * dig[y][dgl - i, k] for i in range(NDIG)
                         if 0 <= dgl - i < NDIG for k in range(K)]
                exact = sum(int(t) for t in terms)
                acc = f32(0.0)
                for t in rng.permutation(np.array(terms, dtype=np.float32)):
                    acc = f32(acc + t)
                assert int(acc) == exact and abs(exact) < 2 ** 22


def fold_and_subtract(D, c, ah, al):
    """The drain's fold of the seven diagonal sums, scale c, A - result."""
    w = [f32(2.0 ** -(14 + 8 * d)) for d in range(NDIG + 1)]
    h1, l1 = two_sum(f32(D[0] * w[0]), f32(D[1] * w[1]))
    h2, l2 = two_sum(f32(D[2] * w[2]), f32(D[3] * w[3]))
    tail = f32(f32(D[4] * w[4]) + f32(f32(D[5] * w[5]) + f32(D[6] * w[6])))
    h, e = two_sum(h1, h2)
    l = f32(f32(f32(l1 + l2) + e) + tail)
    h, l = f32(h * c), f32(l * c)
    sh, se = two_sum(ah, f32(-h))
    se = f32(se + f32(al - l))
    rh = f32(sh + se)
    return rh, f32(se - f32(rh - sh))


def test_update_meets_double_float_accuracy():
    cols = columns(9, 12)
    dig = [column_digits(h, l) for h, l in cols]
    rng = np.random.default_rng(10)
    worst = 0.0
    for x in range(len(cols)):
        for y in range(len(cols)):
            sx, dx = dig[x]
            sy, dy = dig[y]
            D = []
            for dgl in range(NDIG + 1):
                D.append(f32(sum(int(dx[i, k]) * int(dy[dgl - i, k]) for i in range(NDIG)
                                 if 0 <= dgl - i < NDIG for k in range(K))))
            hx, lx = cols[x]
            hy, ly = cols[y]
            px = [Fraction(float(a)) + Fraction(float(b)) for a, b in zip(hx, lx)]
            py = [Fraction(float(a)) + Fraction(float(b)) for a, b in zip(hy, ly)]
            prod = sum(a * b for a, b in zip(px, py))
            a0 = rng.standard_normal() * float(sx) * float(sy) * 4
            ah, al = df_pairs(np.array([a0]))
            rh, rl = fold_and_subtract(D, f32(sx * sy), ah[0], al[0])
            exact = Fraction(float(ah[0])) + Fraction(float(al[0])) - prod
            got = Fraction(float(rh)) + Fraction(float(rl))
            err = abs(float(got - exact)) / (float(sx) * float(sy))
            worst = max(worst, err)
    # the digits' truncation (2^-48 per operand over 32 products), the dropped
    # pairs (below 2^-48 each) and the float32 fold: within 2^-43 of s_x s_y
    # (2^-44.9 measured here), against about 2^-19 for a single-float update
    assert worst <= 2.0 ** -43


def test_dropped_pairs_weigh_below_their_bound():
    # pairs (i, j), i + j >= 7, i, j < 6: |a_i b_j| <= 2^14 at weight
    # 2^(-14-8(i+j)), summed over 32 rows
    bound = sum(K * 2.0 ** 14 * 2.0 ** -(14 + 8 * (i + j))
                for i in range(NDIG) for j in range(NDIG) if i + j > NDIG)
    assert bound < 2.0 ** -46


# --------------------------------------------------------------- FP64 scheme
NDIG64 = 7


def column_digits64(v):
    """Scale 2^(E+1) (E: the largest exponent of the column) and the seven
    balanced base-256 digits of rint(v / s 2^55), with integer operations in
    the kernel's order (least significant digit first)."""
    m = np.max(np.abs(v))
    e = 0 if m == 0 else int(np.frexp(m)[1])      # m < 2^e
    e = max(-126, min(127, e))
    dig = np.zeros((NDIG64, len(v)), dtype=np.int64)
    for k, x in enumerate(v):
        X = int(np.rint(np.ldexp(x, 55 - e)))        # |X| < 2^55
        for j in range(NDIG64 - 1, 0, -1):
            r = ((X + 128) & 255) - 128
            dig[j, k] = r
            X = (X - r) >> 8
        dig[0, k] = X
    return 2.0 ** e, dig


def test_fp64_digits_are_bf16_integers_and_exact_to_2_pow_minus_56():
    rng = np.random.default_rng(21)
    for _ in range(30):
        v = rng.standard_normal(K) * 2.0 ** rng.integers(-40, 3)
        v[rng.integers(0, K, 5)] = 0.0
        s, d = column_digits64(v)
        assert np.max(np.abs(d)) <= 128
        for k in range(K):
            rec = sum(Fraction(int(d[j, k])) * Fraction(2) ** (-7 - 8 * j) for j in range(NDIG64))
            assert abs(rec * Fraction(s) - Fraction(float(v[k]))) <= Fraction(2) ** -56 * Fraction(s)


def test_fp64_fold_meets_fp64_accuracy():
    rng = np.random.default_rng(22)
    worst = 0.0
    for _ in range(40):
        x = rng.standard_normal(K) * 2.0 ** rng.integers(-20, 2)
        y = rng.standard_normal(K) * 2.0 ** rng.integers(-20, 2)
        sx, dx = column_digits64(x)
        sy, dy = column_digits64(y)
        # diagonals d = 0..7 of the digit pairs, exact integers below 2^22
        D = [sum(int(dx[i, k]) * int(dy[dgl - i, k]) for i in range(NDIG64)
                 if 0 <= dgl - i < NDIG64 for k in range(K)) for dgl in range(NDIG64 + 1)]
        assert all(abs(v) < 2 ** 22 for v in D)
        hi = ((D[0] * 256 + D[1]) * 256 + D[2]) * 256 + D[3]
        lo = ((D[4] * 256 + D[5]) * 256 + D[6]) * 256 + D[7]
        assert abs(hi) < 2 ** 47 and abs(lo) < 2 ** 47
        a = float(rng.standard_normal()) * sx * sy * 8
        total = float(lo) * 2.0 ** -70 + float(hi) * 2.0 ** -38   # one rounding (the FMA)
        got = a - total * (sx * sy)
        exact = Fraction(a) - sum(Fraction(float(p)) * Fraction(float(q)) for p, q in zip(x, y))
        err = abs(Fraction(got) - exact) / Fraction(sx * sy)
        worst = max(worst, float(err))
    # truncation of the operands (2^-56 each, 32 products) and two FP64
    # roundings, on the scale s_x s_y of the products (up to 32 in size)
    assert worst <= 2.0 ** -47


# --------------------------------------------- K = R11^-1 R12 by 32-row blocks
def digits_of_rows(M):
    """Six balanced 8-bit digits of each row of M (float64) on its own
    power-of-two scale, as in the digit kernels (scale >= the row's largest
    magnitude); returns (scales, digits[j, row, col])."""
    nrow, ncol = M.shape
    sc = np.ones(nrow)
    dig = np.zeros((NDIG, nrow, ncol))
    for i in range(nrow):
        m = np.max(np.abs(M[i]))
        if m > 0:
            sc[i] = 2.0 ** int(np.ceil(np.log2(m)))
        r = M[i] / sc[i] * 128.0
        for j in range(NDIG):
            a = np.rint(r)
            dig[j, i] = a
            r = (r - a) * 256.0
    return sc, dig


def digit_product(A, B):
    """A (p x 32) times B (32 x q) from digit slices: per-row scales of A,
    per-column scales of B, pairs i + j <= 6 summed as exact integers per
    diagonal, weights 2^(-14-8d)."""
    sa, da = digits_of_rows(A)
    sb, db = digits_of_rows(B.T)
    out = np.zeros((A.shape[0], B.shape[1]))
    for dgl in range(NDIG + 1):
        D = sum(da[i] @ db[dgl - i].T for i in range(NDIG) if 0 <= dgl - i < NDIG)
        assert np.max(np.abs(D)) < 2 ** 22 and np.all(D == np.rint(D))
        out += D * 2.0 ** (-14 - 8 * dgl)
    return out * sa[:, None] * sb[None, :]


def test_blocked_k_solve_with_digit_updates():
    """The K solve's algorithm: backward substitution in 32-row blocks (the
    last one ragged), X_k = U_k^{-1} B_k, and the rows above updated with the
    digit-slice product; agrees with the direct solve to about 2^-44 kappa."""
    rng = np.random.default_rng(31)
    r, q = 150, 37
    R = np.triu(rng.standard_normal((r, r)) * 0.3) + np.diag(2.0 + rng.uniform(size=r))
    B0 = rng.standard_normal((r, q))
    B = B0.copy()
    nblk = (r + 31) // 32
    for k in range(nblk - 1, -1, -1):
        lo, hi = 32 * k, min(32 * k + 32, r)
        U = R[lo:hi, lo:hi]
        B[lo:hi] = np.linalg.solve(U, B[lo:hi])          # X_k (inverse diagonal block)
        if lo:
            A = np.zeros((lo, 32))
            A[:, :hi - lo] = R[:lo, lo:hi]
            X = np.zeros((32, q))
            X[:hi - lo] = B[lo:hi]
            B[:lo] -= digit_product(A, X)
    ref = np.linalg.solve(R, B0)
    err = np.linalg.norm(B - ref) / np.linalg.norm(ref)
    assert err <= np.linalg.cond(R) * 2.0 ** -44
