"""The seeded input generator (synth/) against the published definition of
SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; the reference sequence of the
generator started from state 0, also Java's SplittableRandom with seed 0),
and the properties the workloads rely on: counter form (any window of a
stream equals the same window of a longer draw), uniforms in [0, 1) on a
2^-53 grid, and Gaussians with the right moments."""
import numpy as np

import synth


def test_splitmix64_reference_outputs():
    # the first outputs of the generator whose state starts at 0
    got = [int(x) for x in synth.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # SplittableRandom(0).nextLong(), read as a signed 64-bit integer
    assert got[0] - (1 << 64) == -2152535657050944081


def test_counter_form_windows_agree():
    full = synth.splitmix64(12345, 1000)
    for off, cnt in ((0, 1), (1, 7), (500, 500), (999, 1)):
        assert np.array_equal(synth.splitmix64(12345, cnt, off), full[off:off + cnt])


def test_uniform_grid_and_range():
    u = synth.uniform01(7, (100000,))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))   # on the 2^-53 grid
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002


def test_normal_moments():
    z = synth.normal(9, (200000,), std=2.0)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 2.0) < 0.02
    assert abs(np.mean(z ** 4) / 16.0 - 3.0) < 0.1          # Gaussian kurtosis


def test_integers_and_permutation():
    k = synth.integers(3, 50000, 5, 9)
    assert k.min() == 5 and k.max() == 9
    assert np.all(np.bincount(k - 5) > 9000)
    p = synth.permutation(4, 1000)
    assert np.array_equal(np.sort(p), np.arange(1000))
