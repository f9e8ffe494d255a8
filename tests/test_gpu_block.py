"""The paper's own route as a GPU variant: the block formulae of Eqs. 19-23
(transposition of Eq. 19 fixed; the N x N matrix C of Eq. 22 entering only
through the Schur complement D = S11 - S12 A^{-1} S21) for a full-rank split
H = [H1 H2], on the shape of the paper's Table 1 experiment.  Parity with
the oracle's literal evaluation of the same formulae (orc_block_rbp, which
forms C), and with the oracle's training once refined; a split that is
singular because H is rank deficient is reported, as the oracle reports it."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import problem, rel

pytestmark = pytest.mark.gpu

NUMERIC = 4


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


@pytest.mark.parametrize("L,r1", [(500, 250), (1000, 137)])
def test_block_formulae_match_the_oracle_on_the_table1_shape(elm, ctx, L, r1):
    p = synth.workload_gina_shaped(L=L)
    H = oracle.hidden(p["X"], p["W"], p["b"], None, 0)
    ref_block = oracle.block_rbp(H, r1, p["T"])
    # unrefined: the formulae alone, both sides in FP64 normal-equation form
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64, block_split=r1, max_refine=0)[0]
    assert res["form"] == elm.FORM_BLOCK and res["status"] == 0 and res["rank"] == L
    assert rel(prob["beta"].cpu().numpy(), ref_block) <= 1e-9
    # refined: the minimum-norm least-squares solution of the training
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], None, 0, p["T"])
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED, block_split=r1)[0]
    assert res["form"] == elm.FORM_BLOCK and res["status"] == 0
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-9


def test_block_split_singular_when_rank_deficient(elm, ctx):
    p = synth.make_problem(900, 12, 80, 3, n_dup=6, x_dtype=np.float64)
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"], p["act"])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.block_rbp(H, 40, p["T"])
    res = elm.elm_train(ctx, problem(p), precision=elm.PREC_FP64, block_split=40,
                        check=False)[0]
    assert res["status"] == NUMERIC and res["rank"] < 86


def test_block_split_arguments_are_checked(elm, ctx):
    p = synth.make_problem(300, 5, 40, 2)
    for bad in (40, 41):
        with pytest.raises(elm.ElmError) as e:
            elm.elm_train(ctx, problem(p), block_split=bad)
        assert e.value.status == 1
