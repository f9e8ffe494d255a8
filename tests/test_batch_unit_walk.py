"""The unit walk of the batched tensor-core launch (the hidden layers, Eq. 1,
and the Grams, Eqs. 9-13, of every problem of a call in one launch),
re-derived on the CPU: the host writes first[p], the prefix sums of the
problems' tile counts; CTA b of G takes units b, b + G, ... and finds each
unit's problem by a binary search for the last p with first[p] <= u.
Checked here: every tile of every problem is taken exactly once, each CTA
takes its units in ascending order, and problems without tiles are skipped."""
import numpy as np


def unit_owner(first, nprob, u):
    lo, hi = 0, nprob - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if first[mid] <= u:
            lo = mid
        else:
            hi = mid - 1
    return lo, u - first[lo]


def walk(tiles, G):
    first = np.concatenate([[0], np.cumsum(tiles)]).astype(np.int64)
    nprob = len(tiles)
    taken = [np.zeros(t, dtype=np.int64) for t in tiles]
    for b in range(G):
        u, last = b, -1
        while u < first[nprob]:
            p, t = unit_owner(first, nprob, u)
            assert 0 <= t < tiles[p], (u, p, t)
            assert u > last
            taken[p][t] += 1
            last, u = u, u + G
    return taken


def test_every_tile_once_with_uneven_and_empty_problems():
    rng = np.random.default_rng(7)
    cases = [[1], [5], [0, 3], [3, 0], [0, 0, 4, 0], [2, 0, 0, 7, 1]]
    cases += [list(rng.integers(0, 400, n)) for n in (3, 17, 128)]
    cases += [list(rng.integers(1, 3000, 128))]     # the batched workload's scale
    for tiles in cases:
        for G in (1, 7, 152):
            for t in walk(tiles, G):
                assert np.all(t == 1)


def test_hidden_and_gram_tile_counts_of_a_batch():
    # tile counts as the host forms them: hidden (Lp / 128) (Np / 64), Gram
    # nJ (nJ + 1) with nJ = Lp / 128 over L + m rows
    rng = np.random.default_rng(8)
    N = rng.integers(5000, 50001, 128)
    L = rng.integers(100, 3001, 128)
    m = rng.integers(2, 27, 128)
    pad = lambda v, b: -(-v // b) * b
    hid = [(pad(l + k, 128) // 128) * (pad(n, 64) // 64) for n, l, k in zip(N, L, m)]
    gram = [(pad(l + k, 128) // 128) * (pad(l + k, 128) // 128 + 1) for l, k in zip(L, m)]
    for tiles in (hid, gram):
        for t in walk(tiles, 152):
            assert np.all(t == 1)
