"""The wide branch (N < L): H^+ = H^T (H H^T)^+, the case the paper states
beside Eq. 8, through the N x N Gram of the rows of H and the full-rank
factorisation of the rows.  Parity with the oracle (which forms the same
Moore-Penrose solution through the L x L Gram): rank bit-exact, beta within
1e-9; both precisions take this FP64 branch."""
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


@pytest.mark.parametrize("N,n,L,m,act,xdt", [
    (50, 8, 80, 3, 0, np.float64),
    (500, 40, 2000, 5, 0, np.float32),
    (333, 17, 401, 1, 1, np.float32),      # ragged tiles, tanh, one target
    (1, 4, 30, 2, 0, np.float64),          # a single sample
])
def test_wide_matches_oracle(elm, ctx, N, n, L, m, act, xdt):
    p = synth.make_problem(N, n, L, m, act=act, x_dtype=xdt, x_kind="normal")
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert r == N
    for prec in (elm.PREC_FP64, elm.PREC_MIXED):
        prob = problem(p)
        res = elm.elm_train(ctx, prob, precision=prec)[0]
        assert res["form"] == elm.FORM_WIDE and res["status"] == 0
        assert res["rank"] == r
        beta = prob["beta"].cpu().numpy()
        assert rel(beta, ref) <= 1e-9
        # minimum norm: beta lies in the row space of H (beta = H^T z)
        H = oracle.hidden(p["X"], p["W"], p["b"], p["a"], p["act"])
        z = np.linalg.lstsq(H.T, beta, rcond=None)[0]
        assert np.linalg.norm(H.T @ z - beta) <= 1e-9 * np.linalg.norm(beta)


def test_wide_with_repeated_samples(elm, ctx):
    """Rows of H repeated (the same sample drawn twice, different targets):
    rank N - repeats, and beta the minimum-norm least-squares solution."""
    p = synth.make_problem(120, 10, 300, 4, x_dtype=np.float64, x_kind="uniform11")
    X, T = p["X"].copy(), p["T"].copy()
    rep = [(7, 3), (50, 11), (99, 60), (101, 60)]      # row a takes row b's sample
    for a_, b_ in rep:
        X[a_] = X[b_]
    q = dict(p, X=X, T=T)
    ref, r, _ = oracle.train(X, p["W"], p["b"], p["a"], p["act"], T)
    assert r == 120 - len(rep)
    prob = problem(q)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64)[0]
    assert res["form"] == elm.FORM_WIDE and res["rank"] == r
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-9
