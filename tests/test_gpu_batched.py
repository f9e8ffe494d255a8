"""Several problems in one elm_train call (mixed form): their hidden layers
and Grams run as one tensor-core launch each, walking the tiles of every
problem, before each problem's factorisation, solves and refinement.  The
batched launch does the same integer arithmetic per tile as a launch per
problem, so every beta equals, bit for bit, the beta of training that
problem alone; and each matches the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import problem, rel

pytestmark = pytest.mark.gpu

TIMEOUT = 6


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


def cases():
    return [synth.make_problem(3001, 16, 333, 5, act=synth.ACT_SIGMOID),
            synth.make_problem(1500, 54, 140, 2, n_dup=10, n_scaled=6, act=synth.ACT_TANH,
                               x_kind="uniform11"),
            synth.make_problem(700, 128, 90, 26, x_dtype=np.float64),
            synth.make_problem(40, 8, 120, 3),                     # wide: trained on its own
            synth.workload_sparse_pixels(N=2500, L_unique=300),
            synth.make_problem(65, 5, 7, 1, act=synth.ACT_TANH)]


def test_batched_call_equals_one_call_per_problem(elm, ctx):
    ps = cases()
    probs = [problem(p) for p in ps]
    probs[2] = dict(probs[2], X=ps[2]["X"], T=ps[2]["T"])     # host buffers in the batch
    res = elm.elm_train(ctx, probs, precision=elm.PREC_MIXED)
    for p, pr, r in zip(ps, probs, res):
        one = problem(p)
        r1 = elm.elm_train(ctx, one, precision=elm.PREC_MIXED)[0]
        assert (r["rank"], r["form"], r["refine_iters"]) == (r1["rank"], r1["form"],
                                                             r1["refine_iters"])
        b = pr["beta"] if isinstance(pr["beta"], np.ndarray) else pr["beta"].cpu().numpy()
        assert np.array_equal(b, one["beta"].cpu().numpy())
        ref, rr, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
        assert r["rank"] == rr == min(p["rank"], p["N"])
        assert rel(b, ref) <= 1e-6
    assert res[3]["form"] == elm.FORM_WIDE


def test_batched_wait_bound_expires_then_trains(elm, ctx):
    ps = cases()[:3]
    res = elm.elm_train(ctx, [problem(p) for p in ps], precision=elm.PREC_MIXED,
                        wait_limit_ns=1, check=False)
    assert all(r["status"] == TIMEOUT for r in res)
    probs = [problem(p) for p in ps]
    res = elm.elm_train(ctx, probs, precision=elm.PREC_MIXED)
    for p, pr, r in zip(ps, probs, res):
        ref, rr, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
        assert r["status"] == 0 and r["rank"] == rr
        assert rel(pr["beta"].cpu().numpy(), ref) <= 1e-6
