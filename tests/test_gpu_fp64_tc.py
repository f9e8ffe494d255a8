"""The FP64 form with its products on the tensor cores (ELM_PREC_FP64_TC):
every element of X, W^T and [H^T; T^T] split into eight 7-bit digits on a
2^-55 grid of its row's power-of-two scale and every digit pair of weight
above 2^-68 summed exactly in two tensor-core launches, so the
pre-activations and the Gram are as accurate as FP64 products.  The FP64 bar applies: rank bit-exact and beta within 1e-9 of the
oracle, on the shapes the FP64 form is tested on, and beta within 1e-10 of
the plain FP64 form on the better-conditioned problems (two Grams rounded
differently at 2^-53 move beta by about kappa(S) u, kappa(S) up to 5e6)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import problem, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def elm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_02436_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(elm):
    import torch
    c = elm.elm_create(0, torch.cuda.current_stream())
    yield c
    c.close()


CASES = {
    "small_fp64": lambda: synth.workload_small_fp64(),
    "sparse_pixels": lambda: synth.workload_sparse_pixels(N=3001, L_unique=333),
    "rank_deficient": lambda: synth.workload_rank_deficient(N=4000, L_unique=250, n_dup=25,
                                                           n_scaled=13),
    "tanh_wide_m": lambda: synth.make_problem(2500, 54, 301, 26, act=synth.ACT_TANH),
    "ragged": lambda: synth.make_problem(1037, 13, 121, 3, x_kind="normal", x_dtype=np.float64),
    "tiny": lambda: synth.make_problem(65, 5, 7, 1, act=synth.ACT_TANH),
    # more than 256 columns stay active for 40 panels: the trailing updates
    # run on the tensor cores from seven-digit slices with the exact fold
    "trailing_on_tensor_cores": lambda: synth.make_problem(6000, 64, 1200, 5, n_dup=30,
                                                           n_scaled=10),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_tc_matches_oracle(elm, ctx, case):
    p = CASES[case]()
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64_TC, check=False)[0]
    assert res["form"] == elm.FORM_FP64_TC and res["status"] in (0, 5)
    assert res["rank"] == r == min(p["rank"], p["N"])
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-9
    if case in ("small_fp64", "sparse_pixels", "ragged", "trailing_on_tensor_cores"):
        p64 = problem(p)
        elm.elm_train(ctx, p64, precision=elm.PREC_FP64)
        assert rel(prob["beta"].cpu().numpy(), p64["beta"].cpu().numpy()) <= 1e-10


def test_fp64_tc_host_buffers(elm, ctx):
    p = synth.make_problem(700, 9, 60, 4, n_dup=5)
    prob = dict(X=p["X"], W=p["W"], b=p["b"], a=p["a"], act=0, T=p["T"])
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64_TC)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"])
    assert res["rank"] == r and rel(prob["beta"], ref) <= 1e-9


@pytest.mark.parametrize("N,n,L,xdt,act,kind,n_scaled", [
    (1037, 13, 120, np.float32, 0, "normal", 0),
    (300, 784, 333, np.float32, 0, "uniform01", 0),     # two exact K chunks
    (65, 5, 7, np.float64, 1, "uniform11", 0),
    (777, 21, 90, np.float64, 1, "normal", 9),          # power-of-two output scales a_j
    (2049, 1100, 129, np.float32, 0, "uniform01", 0),   # ragged tiles, three K chunks
])
def test_fp64_tc_hidden_matches_oracle(elm, ctx, N, n, L, xdt, act, kind, n_scaled):
    """Pre-activations at FP64 level: every operand element is rounded once
    at 2^-56 of its row's power-of-two scale (xs_i for X, ws_j for W), every
    kept digit pair is summed exactly and the pairs left out weigh below
    2^-68, so |dz_ij| <= 2^-55 (xs_i |W_j|_1 + ws_j |X_i|_1) plus the FP64
    roundings of the sum and of the oracle's own product (2^-52 sum_k
    |x_k w_k| + |b|); |dH| <= |a_j| |dz| (g' <= 1) plus the rounding of g.
    Checked against the oracle element by element."""
    p = synth.make_problem(N, n, L, 3, n_dup=min(7, L // 3), n_scaled=n_scaled, x_dtype=xdt,
                           act=act, x_kind=kind,
                           x_sparsity=0.8 if kind == "uniform01" else 0.0)
    t = problem(p)
    L = p["L"]                                  # with the planted copies
    Ht = elm.elm_hidden(ctx, t["X"], t["W"], t["b"], t["a"], act,
                        precision=elm.PREC_FP64_TC).cpu().numpy()
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"], act)
    X, W = np.abs(p["X"].astype(np.float64)), np.abs(p["W"])
    p2 = lambda v: 2.0 ** np.ceil(np.log2(np.maximum(v, 1e-300)))   # power-of-two scales
    xs, ws = p2(X.max(axis=1)), p2(W.max(axis=0))
    dz = (2.0 ** -55 * (xs[:, None] * W.sum(axis=0)[None, :] + ws[None, :] * X.sum(axis=1)[:, None])
          + 2.0 ** -52 * (X @ W + np.abs(p["b"])[None, :]))
    a = np.ones(L) if p["a"] is None else np.abs(p["a"])
    bound = 2 * a[None, :] * dz + 4 * 2.0 ** -53 * np.abs(H)
    assert Ht.shape == (L, N)
    assert np.all(np.abs(Ht.T - H) <= bound)
