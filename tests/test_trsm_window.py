"""The slab window of the cluster triangular solve (the solves with R11 of
Eq. 7), re-derived on the CPU: CTA cr of a cluster of CS owns the 32-row
blocks k2 = kl CS + cr, and keeps the tiles of R coupling the step's block
with nsl of its own blocks in shared memory.  A block takes part in every
step before it in the forward solve R^T x = b and in every step after it in
the backward solve R x = b, so the window holds the last own blocks, or the
first.  Checked here: the window indexes stay inside the slab buffer, the
copies stay inside R's rows and columns, and no other contiguous window of
nsl own blocks serves more (step, block) updates from shared memory."""
import itertools

import pytest

TB = 32


def window(nblk, CS, cr, nsl, rev):
    nmine = (nblk - cr + CS - 1) // CS
    wlo = 0 if rev else (nmine - nsl if nmine > nsl else 0)
    return nmine, wlo


def later(k2, k, nblk, rev):
    return k2 < nblk and (k2 < k if rev else k2 > k)


def served(nblk, CS, cr, lo, nsl, rev):
    """(step, own block) updates whose tile of R sits in the window."""
    n = 0
    for s in range(nblk):
        k = nblk - 1 - s if rev else s
        for kl in range(lo, lo + nsl):
            if later(kl * CS + cr, k, nblk, rev):
                n += 1
    return n


@pytest.mark.parametrize("rev", [False, True])
def test_window_is_in_bounds_and_serves_the_most_updates(rev):
    for r, CS in itertools.product([1, 31, 32, 33, 300, 1000, 2000, 5100], [8, 16]):
        nblk = (r + TB - 1) // TB
        nown = (nblk + CS - 1) // CS
        for nsl in sorted({0, 1, 2, nown // 2, max(nown - 1, 0), nown}):
            for cr in range(CS):
                nmine, wlo = window(nblk, CS, cr, nsl, rev)
                assert 0 <= nmine <= nown and 0 <= wlo
                for kl in range(wlo, wlo + nsl):           # slab slots used
                    assert 0 <= kl - wlo < nsl
                    k2 = kl * CS + cr
                    if k2 < nblk:                          # a copy is issued
                        assert kl < nmine and k2 * TB < r + TB
                        assert (k2 * TB * 8) % 16 == 0     # tensor-map x alignment
                best = max(served(nblk, CS, cr, lo, nsl, rev)
                           for lo in range(max(nmine - nsl, 0) + 1))
                assert served(nblk, CS, cr, wlo, nsl, rev) == best


def test_whole_window_when_everything_fits():
    for nblk, CS in [(5, 8), (40, 8), (160, 16)]:
        nown = (nblk + CS - 1) // CS
        for cr in range(CS):
            for rev in (False, True):
                nmine, wlo = window(nblk, CS, cr, nown, rev)
                assert wlo == 0 and nmine <= nown   # every own block in shared memory
