"""The FP64 form with its Gram on the tensor cores (ELM_PREC_FP64_TC): every
element of [H^T; T^T] split into eight 7-bit digits on a 2^-55 grid of its
row's power-of-two scale and every digit pair of weight above 2^-68 summed
exactly in two tensor-core launches, so the Gram is as accurate as an FP64
one.  The FP64 bar applies: rank bit-exact and beta within 1e-9 of the
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
    if case in ("small_fp64", "sparse_pixels", "ragged"):
        p64 = problem(p)
        elm.elm_train(ctx, p64, precision=elm.PREC_FP64)
        assert rel(prob["beta"].cpu().numpy(), p64["beta"].cpu().numpy()) <= 1e-10


def test_fp64_tc_host_buffers(elm, ctx):
    p = synth.make_problem(700, 9, 60, 4, n_dup=5)
    prob = dict(X=p["X"], W=p["W"], b=p["b"], a=p["a"], act=0, T=p["T"])
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64_TC)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"])
    assert res["rank"] == r and rel(prob["beta"], ref) <= 1e-9
