"""Index arithmetic of the tensor-core trailing update and of the blocked K
solve (Eq. 6 and the K = R11^-1 R12 solve), re-derived on the CPU from the
kernels' launch shapes: every access stays inside its buffer and every
output entry is written exactly once, for ragged sizes.  Shares nothing
with the kernels; the arithmetic itself is checked in
test_trailing_digit_scheme.py.

Trailing update: a launch covers Lcap rows (a multiple of 128) and is sized
for the Lup columns known when it is enqueued (the factorisation replays a
captured graph); at run time Ln <= Lup columns remain.  Block b of the
2 nrb (nrb + 1) blocks takes row block rb (from a float square root and two
correction loops) and column block cb < 4 (rb + 1): 128 x 32 tiles of the
lower triangle.  Each thread holds one row x and 16 columns y = yb + k of
its tile, k < kv, writes A'[y, x] (y <= x) directly and stages A'[x, y];
the staged tile's strictly lower entries are written row-wise afterwards.
"""
import numpy as np
import pytest

TR, TC = 128, 32


def row_block(b, sqrt=lambda v: np.sqrt(np.float32(v))):
    rb = int((float(sqrt(np.float32(2.0) * np.float32(b) + np.float32(1.0))) - 1.0) * 0.5)
    while rb > 0 and 2 * rb * (rb + 1) > b:
        rb -= 1
    while 2 * (rb + 1) * (rb + 2) <= b:
        rb += 1
    return rb, b - 2 * rb * (rb + 1)


@pytest.mark.parametrize("skew", [0, -2, 2])
def test_blocks_cover_each_lower_tile_once(skew):
    # a square root a few ulp off still lands on the right row block
    def sq(v):
        r = np.sqrt(v)
        for _ in range(abs(skew)):
            r = np.nextafter(r, np.float32(np.inf) if skew > 0 else np.float32(0))
        return r

    for nrb in list(range(1, 40)) + [63, 100, 200]:
        seen = set()
        for b in range(2 * nrb * (nrb + 1)):
            rb, cb = row_block(b, sq)
            assert 0 <= rb < nrb and 0 <= cb < 4 * (rb + 1), (nrb, b, rb, cb)
            seen.add((rb, cb))
        assert len(seen) == 2 * nrb * (nrb + 1)


def trailing_writes(Lcap, Lup, Ln, lda):
    """Counts of the entries of A' written by one launch, and checks of every
    read and write index against the buffers."""
    assert Lcap % TR == 0 and Ln <= Lup <= Lcap <= lda
    rows = -(-Lup // TR) * TR                     # rows the digit kernel fills
    assert rows <= Lcap
    nrb = rows // TR
    count = np.zeros((Ln, Ln), dtype=np.int64)
    rem = np.arange(Ln)                           # compaction map: entries < lda
    x_loc = np.arange(TR)[:, None, None]
    half = np.arange(2)[None, :, None]
    k = np.arange(16)[None, None, :]
    for b in range(2 * nrb * (nrb + 1)):
        rb, cb = row_block(b)
        r0, c0 = rb * TR, cb * TC
        if r0 >= Ln or c0 >= Ln:
            continue
        # tensor-map boxes: 128 rows of A planes, 32 rows of B planes
        assert r0 + TR <= Lcap and c0 + TC <= Lcap
        x = r0 + x_loc
        yb = c0 + half * 16
        kv = np.minimum(Ln - yb, x - yb + 1)
        kv = np.where(x < Ln, np.minimum(kv, 16), 0)
        valid = k < kv
        y = yb + k
        xs, ys = np.broadcast_to(x, valid.shape)[valid], np.broadcast_to(y, valid.shape)[valid]
        # the prefix k < kv is exactly the set y < Ln, y <= x, x < Ln
        full = (np.broadcast_to(x, valid.shape) < Ln) & (np.broadcast_to(y, valid.shape) < Ln) \
            & (np.broadcast_to(y, valid.shape) <= np.broadcast_to(x, valid.shape))
        assert np.array_equal(valid, full)
        assert np.all(rem[ys] * lda + rem[xs] < lda * lda)      # reads of A
        np.add.at(count, (ys, xs), 1)                          # upper entries A'[y, x]
        staged = np.zeros((TR, TC), dtype=bool)
        staged[(xs - r0), (ys - c0)] = True
        # strictly lower entries from the staged tile, one row segment per warp
        for i in range(TR):
            xr = r0 + i
            if xr >= Ln:
                continue
            yl = c0 + np.arange(TC)
            sel = yl < xr
            assert np.all(staged[i, sel]), (b, i)             # staged before written
            np.add.at(count, (np.full(sel.sum(), xr), yl[sel]), 1)
    return count


@pytest.mark.parametrize("Lcap,Lup,Ln", [
    (384, 300, 300), (384, 300, 257), (384, 384, 384), (512, 460, 401),
    (1152, 1100, 1100), (1152, 1100, 1033), (2048, 2000, 1968), (2048, 1700, 1699),
])
def test_trailing_update_writes_each_entry_once(Lcap, Lup, Ln):
    count = trailing_writes(Lcap, Lup, Ln, lda=Lcap)
    assert count.min() == 1 and count.max() == 1


def test_trailing_update_with_nothing_left():
    assert trailing_writes(384, 300, 0, lda=384).size == 0


def ksolve_writes(r, q):
    """One pass of the blocked backward substitution's launches: per step k
    the digit rows and columns written, then the tiles of B updated."""
    Rcap, Qcap = -(-r // TR) * TR, -(-q // TC) * TC
    nblk, nnt, nxb = -(-r // 32), -(-q // TC), -(-q // 8)
    solved = np.zeros(r, dtype=np.int64)            # X_k rows written into B
    for k in range(nblk - 1, -1, -1):
        rows, c0 = 32 * k, 32 * k
        nrb = -(-rows // 8)
        nbk = min(r - c0, 32)
        assert 0 < nbk <= 32
        # prep: warps of the first nrb blocks take rows i < rows (digits of
        # R[i, c0 ..] into GR row i); the rest take columns c < q
        i = np.arange(nrb * 8)
        assert np.all(i[i < rows] < Rcap)
        c = np.arange(nxb * 8)
        assert np.all(c[c < q] < Qcap)
        solved[c0:c0 + nbk] += 1                     # B[c0 + lane, c], lane < nbk
        assert c0 + nbk <= r
        if rows == 0:
            continue
        nmt = -(-rows // TR)
        upd = np.zeros((rows, q), dtype=np.int64)
        for blk in range(nmt * nnt):
            r0, t0 = (blk // nnt) * TR, (blk % nnt) * TC
            assert r0 + TR <= Rcap and t0 + TC <= Qcap   # tensor-map boxes
            ri = r0 + np.arange(TR)[:, None]
            ci = t0 + np.arange(TC)[None, :]
            m = (ri < rows) & (ci < q)
            np.add.at(upd, (np.broadcast_to(ri, m.shape)[m], np.broadcast_to(ci, m.shape)[m]), 1)
        assert upd.min() == 1 and upd.max() == 1       # every row above, every column
    assert np.all(solved == 1)


@pytest.mark.parametrize("r,q", [(32, 1), (33, 5), (150, 37), (257, 64), (900, 200), (2100, 333)])
def test_k_solve_launches_cover_b_once_per_step(r, q):
    ksolve_writes(r, q)
