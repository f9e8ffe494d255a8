"""Parity at the full sizes of the workload configurations, in the launch
configuration bench.py times (device-resident inputs, default options),
element by element against the FP64 CPU oracle's beta (Eq. 5, beta = H^+ T):

  * sparse pixels (60000 x 784, L = 2000): the oracle trains it here (about
    15 s on 16 cores); both forms against it;
  * rank-deficient (100000 x 64, L = 6000, rank 5100), large (500000 x 128,
    L = 8000) and the 128 batched problems: against the oracle's results
    stored in tests/golden/full_*.npz by tests/golden/make_full_goldens.py,
    which calls only the oracle and the input generators; the inputs'
    fingerprints are checked first, so both sides saw the same bytes;
  * the rank equal to the oracle's (bit-exact) and to the planted rank;
  * beta within 1e-6 (mixed form) or 1e-9 (FP64 form) relative Frobenius
    error of the oracle's.  Where FP64 arithmetic itself cannot fix beta
    that closely, the bar widens to the problem's least-squares forward
    error scale (below), which the golden file records per problem.

Forward error scale of a least-squares solution computed in FP64 through
the normal equations with k refinement steps (both sides take k = 2):
    u (kappa + kappa^2 eta) + (kappa^2 u)^(k+1),
    eta = ||T - H beta|| / (||H||_2 ||beta||),
with kappa the condition number of H after column equilibration (both the
oracle and the library equilibrate) and u = 2^-53.  The first term is
Wedin's perturbation bound, the level a converged refinement reaches; the
second is what k steps leave of the first solve's error kappa(S) u, each
step contracting it by kappa(S) u = kappa^2 u (Higham, Accuracy and
Stability of Numerical Algorithms, ch. 20).  Two FP64 solvers may each be
that far from the exact beta, so the widened bar is 8 times the scale.  It
is used only for problems whose recorded scale exceeds 1/100 of the bar.
"""
import hashlib
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U = 2.0 ** -53
WIDEN = 8.0


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


def to_problem(p):
    import torch
    dev = torch.device("cuda", 0)
    L, m = p["W"].shape[1], p["T"].shape[1]
    return dict(X=torch.from_numpy(p["X"]).to(dev), W=torch.from_numpy(p["W"]).to(dev),
                b=torch.from_numpy(p["b"]).to(dev),
                a=None if p.get("a") is None else torch.from_numpy(p["a"]).to(dev),
                act=int(p.get("act", 0)), T=torch.from_numpy(p["T"]).to(dev),
                beta=torch.empty((L, m), dtype=torch.float64, device=dev))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def digest(a):
    return "" if a is None else hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def golden(name, probs):
    """The stored oracle results, after checking the inputs' fingerprints."""
    path = os.path.join(GOLD, "full_%s.npz" % name)
    if not os.path.exists(path):
        pytest.skip("oracle results not written: tests/golden/make_full_goldens.py %s" % name)
    g = np.load(path)
    assert int(g["count"]) == len(probs)
    for i, p in enumerate(probs):
        assert digest(p["X"]) == str(g["fp_X"][i]), "X differs from the golden inputs"
        assert digest(p["W"]) == str(g["fp_W"][i])
        assert digest(p["b"]) == str(g["fp_b"][i])
        assert digest(p.get("a")) == str(g["fp_a"][i])
        assert np.isclose(np.linalg.norm(p["T"]), float(g["fp_T_norm"][i]), rtol=1e-12, atol=0)
    return g


def error_scale(g, i, steps=2):
    """u (kappa + kappa^2 eta) + (kappa^2 u)^(steps+1) of problem i
    (equilibrated H)."""
    kappa = float(g["kappa"][i])
    L = g["beta_%03d" % i].shape[0]
    h2 = np.sqrt(float(g["ev_max"][i])) * float(g["h_fro"][i]) / np.sqrt(L)   # ~ ||H||_2
    eta = float(g["res_norm"][i]) / (h2 * float(g["beta_norm"][i]))
    return U * (kappa + kappa * kappa * eta) + (kappa * kappa * U) ** (steps + 1)


def bar_for(g, i, bar):
    sc = error_scale(g, i)
    return bar if sc <= bar / 100.0 else max(bar, WIDEN * sc)


def check_against_golden(elm, ctx, name, probs, precision, bar):
    g = golden(name, probs)
    dev_probs = [to_problem(p) for p in probs]
    res = elm.elm_train(ctx, dev_probs, precision=precision, check=False)
    worst = []
    for i, (p, pr, r) in enumerate(zip(probs, dev_probs, res)):
        ref = g["beta_%03d" % i]
        assert r["status"] in (0, 5), (i, r)             # 5: beta written, not converged
        assert r["rank"] == int(g["rank"][i]) == int(p["rank"]), (i, r["rank"])
        err = rel(pr["beta"].cpu().numpy(), ref)
        tol = bar_for(g, i, bar)
        assert err <= tol, (i, err, tol, float(g["kappa"][i]))
        worst.append(err)
    return res, worst, [pr["beta"].cpu().numpy() for pr in dev_probs]


def test_sparse_pixels_full_against_oracle(elm, ctx):
    p = synth.workload_sparse_pixels()
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], None, 0, p["T"])
    assert r == 2000
    for prec, bar in ((elm.PREC_MIXED, 1e-6), (elm.PREC_FP64, 1e-9)):
        pr = to_problem(p)
        res = elm.elm_train(ctx, pr, precision=prec)[0]
        assert res["status"] == 0 and res["rank"] == r
        assert res["form"] == (elm.FORM_MIXED if prec == elm.PREC_MIXED else elm.FORM_FP64)
        assert rel(pr["beta"].cpu().numpy(), ref) <= bar


def test_rank_deficient_full_against_golden(elm, ctx):
    p = synth.workload_rank_deficient()
    res, worst, betas = check_against_golden(elm, ctx, "rank_deficient", [p], elm.PREC_MIXED,
                                             1e-6)
    assert res[0]["status"] == 0 and res[0]["form"] == elm.FORM_MIXED
    # the minimum-norm split over planted copies (Moore-Penrose, Eq. 5):
    # duplicates share equally, a copy scaled by s gets s times the weight
    beta = betas[0]
    src, sc = p["src"], p["scale"]
    for j in range(len(src)):
        k = int(np.nonzero((src == src[j]) & (sc == 1.0))[0][0])
        if k != j:
            assert np.allclose(beta[j], sc[j] * beta[k], rtol=1e-9, atol=1e-12 * np.abs(beta).max())


def test_batched_full_against_golden(elm, ctx):
    ps = synth.workload_batched()
    res, worst, _ = check_against_golden(elm, ctx, "batched", ps, elm.PREC_MIXED, 1e-6)
    assert all(r["form"] in (elm.FORM_MIXED, elm.FORM_MIXED_TO_FP64) for r in res)
    # every problem whose scale allows the strict bar meets it
    g = np.load(os.path.join(GOLD, "full_batched.npz"))
    strict = [i for i in range(len(ps)) if error_scale(g, i) <= 1e-8]
    assert len(strict) >= 100
    assert max(worst[i] for i in strict) <= 1e-6


@pytest.mark.slow
def test_large_full_against_golden(elm, ctx):
    p = synth.workload_large()
    res, worst, _ = check_against_golden(elm, ctx, "large", [p], elm.PREC_MIXED, 1e-6)
    assert res[0]["status"] == 0 and res[0]["form"] == elm.FORM_MIXED


@pytest.mark.parametrize("L", [500, 2000])
def test_gina_shaped_matches_oracle(elm, ctx, L):
    """The shape of the paper's Table 1 experiment (3468 x 971, L = 500 and
    2000): the oracle end to end, both forms."""
    p = synth.workload_gina_shaped(L=L)
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], None, int(p["act"]), p["T"])
    assert r == L
    for prec, tol in ((elm.PREC_MIXED, 1e-6), (elm.PREC_FP64, 1e-9)):
        pr = to_problem(p)
        res = elm.elm_train(ctx, pr, precision=prec)[0]
        assert res["status"] == 0 and res["rank"] == r
        assert rel(pr["beta"].cpu().numpy(), ref) < tol
