"""The row-sharded route on the GPU (elm_rows_*, elm_factor_*), its ranks
emulated by row blocks in one process (no kernel waits on another): the
blocks' Gram blocks summed in order, one factorisation, refinement residuals
summed the same way.  Parity with the oracle's training of the whole
problem: rank bit-exact, beta within 1e-9 (FP64) or 1e-6 (mixed)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel, to_dev

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
    "sparse_pixels": lambda: synth.workload_sparse_pixels(N=7001, L_unique=450),
    "rank_deficient": lambda: synth.workload_rank_deficient(N=6000, L_unique=300, n_dup=30,
                                                            n_scaled=15),
    "tanh": lambda: synth.make_problem(5000, 54, 333, 7, act=synth.ACT_TANH),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("nblocks", [1, 3])
def test_row_blocks_match_oracle(elm, ctx, case, nblocks):
    from paper_2011_02436_gb300.sharded import LibraryOps, train_row_blocks
    p = CASES[case]()
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    t = to_dev(p)
    rows = np.array_split(np.arange(p["N"]), nblocks)
    blocks = [(t["X"][int(q[0]):int(q[-1]) + 1], t["W"], t["b"], t["a"], p["act"],
               t["T"][int(q[0]):int(q[-1]) + 1]) for q in rows]
    for prec, bar in ((elm.PREC_FP64, 1e-9), (elm.PREC_MIXED, 1e-6)):
        beta, rank, info = train_row_blocks(LibraryOps(ctx, prec), blocks, precision=prec)
        assert rank == r == p["rank"]
        # two FP64 steps may stop just short of 1e-12 on the tanh case
        # (kappa(H) near 1e4): elm_train reports that as not converged too
        assert info["converged"] or (prec == elm.PREC_FP64 and info["rel_update"] <= 1e-9)
        # one block: the mixed form hands over to the FP64 form exactly where
        # elm_train does (the same Gram, the same refinement)
        if prec == elm.PREC_MIXED and nblocks == 1:
            import torch
            pr = dict(X=t["X"], W=t["W"], b=t["b"], a=t["a"], act=p["act"], T=t["T"],
                      beta=torch.empty_like(beta))
            res = elm.elm_train(ctx, pr, precision=prec)[0]
            assert info["handed_over"] == (res["form"] == elm.FORM_MIXED_TO_FP64)
        assert rel(beta.cpu().numpy(), ref) <= bar


def test_row_block_gram_is_the_sum_over_its_rows(elm, ctx):
    p = synth.make_problem(3000, 20, 150, 4, n_dup=5)
    t = to_dev(p)
    whole = elm.RowBlock(ctx, t["X"], t["W"], t["b"], t["a"], 0, t["T"], elm.PREC_FP64)
    a = elm.RowBlock(ctx, t["X"][:1234], t["W"], t["b"], t["a"], 0, t["T"][:1234], elm.PREC_FP64)
    b = elm.RowBlock(ctx, t["X"][1234:], t["W"], t["b"], t["a"], 0, t["T"][1234:], elm.PREC_FP64)
    (S, Z), (Sa, Za), (Sb, Zb) = whole.gram(), a.gram(), b.gram()
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"], 0)
    S0, Z0 = oracle.gram(H, p["T"])
    for got in (S, Sa + Sb):
        assert rel(got.cpu().numpy(), S0) <= 1e-14
    for got in (Z, Za + Zb):
        assert rel(got.cpu().numpy(), Z0) <= 1e-14
    f = elm.GramFactor(ctx, S, 4, elm.PREC_FP64)
    assert f.rank == p["rank"] == 150
    beta = f.solve(Z)
    r0, perm0, R0 = oracle.pivchol(S0)
    beta0 = oracle.frsolve(R0, r0, perm0, Z0)
    # both solve the normal equations once, unrefined: they agree to about
    # cond(S1) u, S1 the Gram of the independent columns
    S1 = S0[np.ix_(perm0[:r0], perm0[:r0])]
    assert rel(beta.cpu().numpy(), beta0) <= 100 * np.linalg.cond(S1) * 2.0 ** -53
    for h in (whole, a, b, f):
        h.close()
