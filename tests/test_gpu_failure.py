"""Failure detection on the GPU in forms that fault, trap and hang nothing:
a bound on the tensor kernels' pipeline waits that runs out (the kernels
stop issuing work, let their own copies and MMAs finish, free their tensor
memory and return; the host reports a timeout and the context stays
usable), and refinement that ends before reaching its tolerance."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import problem, rel

pytestmark = pytest.mark.gpu

TIMEOUT, NOT_CONVERGED = 6, 5


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


def test_wait_bound_expires_then_the_context_trains_normally(elm, ctx):
    p = synth.workload_sparse_pixels(N=3000, L_unique=333)
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    # a 1 ns bound: the first pipeline wait that is not already satisfied
    # gives up, in every tensor-core launch of the training
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED, wait_limit_ns=1, check=False)[0]
    assert res["status"] == TIMEOUT
    with pytest.raises(elm.ElmError) as e:
        elm.elm_train(ctx, problem(p), precision=elm.PREC_MIXED, wait_limit_ns=1)
    assert e.value.status == TIMEOUT
    # the same context, default bound: oracle parity
    for _ in range(2):
        prob = problem(p)
        res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
        assert res["status"] == 0 and res["rank"] == r == p["rank"]
        assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-6


def test_refinement_cut_short_is_reported_and_beta_still_written(elm, ctx):
    p = synth.workload_small_fp64()
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64, max_refine=1, refine_tol=1e-300,
                        check=False)[0]
    assert res["status"] == NOT_CONVERGED
    assert res["refine_iters"] == 1 and res["rel_update"] > 1e-300
    assert res["rank"] == r == 180
    # one step leaves beta within the FP64 bar all the same
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-9
    # elm_train's own return value reports it
    with pytest.raises(elm.ElmError) as e:
        elm.elm_train(ctx, problem(p), precision=elm.PREC_FP64, max_refine=1, refine_tol=1e-300)
    assert e.value.status == NOT_CONVERGED
    # with the default tolerance the same problem converges
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64)[0]
    assert res["status"] == 0 and res["rel_update"] <= 1e-12
    assert np.isfinite(prob["beta"].cpu().numpy()).all()
