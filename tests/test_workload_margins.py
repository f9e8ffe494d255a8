"""Rank-decision margins of the workloads the parity tests use, from the
oracle: the smallest accepted pivot (unit-diagonal scale) must clear both
rank thresholds -- L 2^-52 (FP64 Gram) and 2^-32 (mixed Gram) -- by a wide
factor, so that the GPU's rank can be compared bit-exactly."""
import os

import numpy as np
import pytest

import oracle
import synth

CASES = {
    "small_fp64": lambda: synth.workload_small_fp64(),
    "sparse_pixels": lambda: synth.workload_sparse_pixels(N=3000, L_unique=333),
    "rank_deficient": lambda: synth.workload_rank_deficient(N=4000, L_unique=250, n_dup=25,
                                                           n_scaled=13),
    "tanh_wide_m": lambda: synth.make_problem(2500, 54, 301, 26, act=synth.ACT_TANH),
    "scaled": lambda: synth.make_problem(1500, 20, 140, 5, n_dup=10, n_scaled=30,
                                         x_kind="uniform11"),
    "wide": lambda: synth.make_problem(50, 8, 80, 3, x_dtype=np.float64, x_kind="normal"),
    "gina_shaped_500": lambda: synth.workload_gina_shaped(L=500),
    "gina_shaped_2000": lambda: synth.workload_gina_shaped(L=2000),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_rank_margins_cover_mixed_threshold(name):
    p = CASES[name]()
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"], p["act"])
    S, _ = oracle.gram(H)
    r, perm, R = oracle.pivchol(S)
    assert r == min(p["rank"], p["N"])
    piv = np.diag(R)[:r] ** 2 / np.diag(S)[perm[:r]]
    assert piv.min() > 1000 * 2.0 ** -32
    assert piv.min() > 1e6 * oracle.default_tau(S.shape[0])


FULL = ("rank_deficient", "batched", "large")
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", FULL)
def test_full_size_margins_from_the_oracle(name):
    """The same margins at every workload's full size, as the oracle recorded
    them (tests/golden/make_full_goldens.py).  Every planted dependence is
    found (remaining diagonals far below tau = L 2^-52).  The smallest
    genuine pivot clears tau by at least a factor of two everywhere; the
    single-problem workloads clear it by six orders of magnitude.  In the
    batched workload tanh neurons on 54 or 128 inputs saturate, and some
    problems have kappa(H) of 10^6 to 5*10^7: their smallest pivots lie
    within 1000x of the mixed threshold 2^-32 (the mixed form hands those it
    cannot settle to the FP64 form), and the tightest lies 2.4x above tau,
    so its rank is compared bit-exactly with no more margin than that."""
    path = os.path.join(GOLD, "full_%s.npz" % name)
    if not os.path.exists(path):
        pytest.skip("golden file not written yet")
    g = np.load(path)
    tau = g["tau"]
    assert np.all(g["rejected_max"] < 1e-2 * tau)
    assert np.all(g["piv_min"] > 2 * tau)
    if name != "batched":
        assert np.all(g["piv_min"] > 1e6 * tau)
        assert np.all(g["piv_min"] > 1e3 * 2.0 ** -32)
    else:
        tight64 = int(np.sum(g["piv_min"] < 1e3 * tau))
        tight_mixed = int(np.sum(g["piv_min"] < 1e3 * 2.0 ** -32))
        below_mixed = int(np.sum(g["piv_min"] < 2.0 ** -32))
        assert (tight64, tight_mixed, below_mixed) == (13, 52, 11)
