"""Rank-decision margins of the workloads the parity tests use, from the
oracle: the smallest accepted pivot (unit-diagonal scale) must clear both
rank thresholds -- L 2^-52 (FP64 Gram) and 2^-32 (mixed Gram) -- by a wide
factor, so that the GPU's rank can be compared bit-exactly."""
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
