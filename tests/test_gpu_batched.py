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
            synth.make_problem(65, 5, 7, 1, act=synth.ACT_TANH),
            # more than 65536 samples: the Gram digit planes in two blocks
            synth.make_problem(70001, 16, 150, 3, act=synth.ACT_SIGMOID)]


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


LANE_CASES = [12, 108, 74, 5, 36, 91]   # kappa(H) 4.7e7 .. 1e4, L 194 .. 2687


def test_lanes_do_not_change_results(elm, ctx):
    """The back halves (factorisation, solves, refinement, hand-over to the
    FP64 form) of a batched call run on several lanes at once, each with its
    own stream, workspaces and host thread: every result is bit for bit the
    one of a single lane, and each beta meets its bar against the oracle's
    stored result for that problem of the batched workload."""
    import os
    from test_gpu_full_configs import GOLD, bar_for, digest
    path = os.path.join(GOLD, "full_batched.npz")
    if not os.path.exists(path):
        pytest.skip("oracle results not written")
    g = np.load(path)
    ps = synth.workload_batched(only=LANE_CASES)
    for i, p in zip(LANE_CASES, ps):
        assert digest(p["X"]) == str(g["fp_X"][i])
    out = {}
    for lanes in (1, 3, 8):
        probs = [problem(p) for p in ps]
        res = elm.elm_train(ctx, probs, precision=elm.PREC_MIXED, lanes=lanes, check=False)
        out[lanes] = (res, [pr["beta"].cpu().numpy() for pr in probs])
    keys = ("status", "rank", "form", "refine_iters", "rel_update")
    for lanes in (3, 8):
        for r1, b1, r, b in zip(*out[1], *out[lanes]):
            assert [r[k] for k in keys] == [r1[k] for k in keys]
            assert np.array_equal(b, b1)
    res, betas = out[1]
    assert any(r["form"] == elm.FORM_MIXED_TO_FP64 for r in res)
    for i, r, b in zip(LANE_CASES, res, betas):
        assert r["status"] in (0, 5) and r["rank"] == int(g["rank"][i])
        assert rel(b, g["beta_%03d" % i]) <= bar_for(g, i, 1e-6)


def test_lanes_rank_deficient_k_on_tensor_cores(elm, ctx):
    """Rank-deficient problems whose K = R11^-1 R12 is formed on the tensor
    cores (r >= 256, q >= 64) and whose trailing updates run on the tensor
    cores, trained in one batched call on several lanes at once (each lane
    its own workspaces for the digit planes): bit for bit the results of one
    lane, ranks and betas as the oracle's."""
    shapes = [(3000, 30, 400, 3, 80, 20), (2500, 20, 330, 5, 60, 40), (3500, 40, 520, 2, 100, 0),
              (2800, 25, 300, 4, 70, 10)]
    ps = [synth.make_problem(N, n, L, m, n_dup=d, n_scaled=sc, x_kind="normal",
                             seed=synth.SEED_BASE + 7000 + 13 * i)
          for i, (N, n, L, m, d, sc) in enumerate(shapes)]
    out = {}
    for lanes in (1, 4):
        probs = [problem(p) for p in ps]
        res = elm.elm_train(ctx, probs, precision=elm.PREC_MIXED, lanes=lanes, check=False)
        out[lanes] = (res, [pr["beta"].cpu().numpy() for pr in probs])
    for r1, b1, r4, b4 in zip(*out[1], *out[4]):
        assert r1["rank"] == r4["rank"] and np.array_equal(b1, b4)
    for p, r, b in zip(ps, *out[1]):
        ref, rank, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
        assert r["status"] == 0 and r["form"] == elm.FORM_MIXED   # settled in the mixed form
        assert r["rank"] == rank == p["rank"]
        assert rel(b, ref) <= 1e-6
