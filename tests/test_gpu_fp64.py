"""GPU parity of the FP64 path through the C ABI against the CPU oracle.

Bars: rank bit-exact; beta within 1e-9 relative Frobenius error; H within
a few ulps (the GPU fuses multiply-adds, the oracle does not); duplicate
neurons give bitwise-equal columns of H.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import problem, rel, to_dev

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


@pytest.mark.parametrize("xdt,act", [(np.float32, 0), (np.float64, 1), (np.float32, 1)])
def test_hidden_matches_oracle(elm, ctx, xdt, act):
    p = synth.make_problem(1037, 13, 120, 3, n_dup=7, n_scaled=3, x_dtype=xdt, act=act,
                           x_kind="normal")
    t = to_dev(p)
    Ht = elm.elm_hidden(ctx, t["X"], t["W"], t["b"], t["a"], act).cpu().numpy()
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"], act)
    assert Ht.shape == (130, 1037)
    assert np.max(np.abs(Ht.T - H)) < 1e-14 * max(1.0, np.abs(H).max())
    src, sc = p["src"], p["scale"]
    for j in range(130):                                    # bitwise duplicates
        k = int(np.nonzero((src == src[j]) & (sc == 1.0))[0][0])
        assert np.array_equal(Ht[j], sc[j] * Ht[k])


def test_hidden_host_buffers(elm, ctx):
    p = synth.make_problem(300, 7, 50, 2, x_dtype=np.float64)
    Ht = elm.elm_hidden(ctx, p["X"], p["W"], p["b"], None, 0)      # numpy in, numpy out
    assert isinstance(Ht, np.ndarray)
    assert np.max(np.abs(Ht.T - oracle.hidden(p["X"], p["W"], p["b"]))) < 1e-14


@pytest.mark.parametrize("n_dup,n_scaled", [(0, 0), (12, 0), (8, 6)])
def test_pinv_rank_and_penrose(elm, ctx, n_dup, n_scaled):
    p = synth.make_problem(90, 6, 40, 2, n_dup=n_dup, n_scaled=n_scaled, x_dtype=np.float64)
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"])
    import torch
    Ht = torch.from_numpy(np.ascontiguousarray(H.T)).cuda()
    r, perm, Xp = elm.elm_pinv_rank(ctx, Ht, want_pinv=True)
    Xo, ro = oracle.pinv(H)
    assert r == ro == 40
    Xp = Xp.cpu().numpy()
    # Both sides form H^+ through the Gram matrix (Eq. 5, Eq. 7) without
    # refinement, so each carries a forward error of order kappa(H1)^2 u
    # (u = 2^-53) and so does their difference; about 2.6e-8 here.
    s = np.linalg.svd(H[:, perm[:r]], compute_uv=False)
    kappa = s[0] / s[-1]
    assert rel(Xp, Xo) < 8.0 * kappa * kappa * 2.0 ** -53
    assert sorted(perm.tolist()) == list(range(H.shape[1]))
    assert list(perm[r:]) == sorted(perm[r:])
    assert np.linalg.matrix_rank(H[:, perm[:r]]) == r       # H1 columns independent


def test_train_small_fp64_workload(elm, ctx):
    """2000x16, L=200 with 20 duplicated neurons: rank 180."""
    p = synth.workload_small_fp64()
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r == 180
    assert res["form"] == elm.FORM_FP64
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("case", ["sparse_pixels", "rank_deficient", "tanh_wide_m"])
def test_train_reduced_workloads(elm, ctx, case):
    if case == "sparse_pixels":
        p = synth.workload_sparse_pixels(N=3000, L_unique=333)
    elif case == "rank_deficient":
        p = synth.workload_rank_deficient(N=4000, L_unique=250, n_dup=25, n_scaled=13)
    else:
        p = synth.make_problem(2500, 54, 301, 26, act=synth.ACT_TANH)
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r == p["rank"]
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("N,n,L,m", [(50, 8, 80, 3), (1, 3, 5, 1), (7, 1, 1, 1), (129, 65, 64, 17)])
def test_train_edge_shapes(elm, ctx, N, n, L, m):
    """Wide H (N < L, rank N), a single sample, L = 1, ragged tiles."""
    p = synth.make_problem(N, n, L, m, x_dtype=np.float64, x_kind="normal")
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-9


def test_train_host_buffers(elm, ctx):
    p = synth.make_problem(700, 9, 60, 4, n_dup=5)
    prob = dict(X=p["X"], W=p["W"], b=p["b"], a=p["a"], act=0, T=p["T"])
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"])
    assert isinstance(prob["beta"], np.ndarray)
    assert res["rank"] == r
    assert rel(prob["beta"], ref) <= 1e-9


def test_predict_matches_oracle(elm, ctx):
    p = synth.make_problem(1111, 21, 150, 19, act=1, x_kind="normal")
    beta = synth.normal(99, (150, 19))
    t = to_dev(p)
    import torch
    Y = elm.elm_predict(ctx, t["X"], t["W"], t["b"], t["a"], 1,
                        torch.from_numpy(beta).cuda()).cpu().numpy()
    ref = oracle.predict(p["X"], p["W"], p["b"], p["a"], 1, beta)
    assert rel(Y, ref) < 1e-13


def test_nonfinite_input_is_reported(elm, ctx):
    p = synth.make_problem(200, 5, 20, 2)
    p["X"][3, 2] = np.nan
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64, check=False)[0]
    assert res["status"] == 4                                # ELM_ERR_NUMERIC


def test_bad_arguments_are_rejected_before_launch(elm, ctx):
    import torch
    p = synth.make_problem(100, 5, 20, 2)
    t = to_dev(p)
    empty_beta = torch.zeros((20, 0), dtype=torch.float64, device="cuda")   # m = 0
    with pytest.raises(elm.ElmError) as e:
        elm.elm_predict(ctx, t["X"], t["W"], t["b"], None, 0, empty_beta)
    assert e.value.status == 1
    with pytest.raises(elm.ElmError) as e:                   # unknown activation
        elm.elm_hidden(ctx, t["X"], t["W"], t["b"], None, 7)
    assert e.value.status == 1


def test_train_many_targets_rank_deficient(elm, ctx):
    # m = 40 targets: column passes in the residual kernels and the skinny
    # K products of the rank-deficient solve
    p = synth.make_problem(3000, 11, 150, 40, n_dup=20, n_scaled=10, x_kind="normal",
                           target="regression")
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r == 150
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-9
