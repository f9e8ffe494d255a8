"""The autotuner: elm_autotune times launch choices (pivot-panel cluster
size and width, tensor-kernel pipeline depth, lanes of a batched call) on
the caller's problems, keeps the fastest per shape bucket in the context and
in a cache file, and elm_train uses it (also in a fresh context that loads
the file).  The choices change launches only: beta stays within the form's
bar against the oracle."""
import math

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


def bucket(prec, p):
    lg = lambda v: int(math.floor(math.log2(v)))
    return "p%d_L%d_N%d_n%d" % (prec, lg(p["L"]), lg(p["N"]), lg(p["X"].shape[1]))


def test_one_problem_mixed_choice_file_and_reuse(elm, ctx, tmp_path):
    import torch
    p = synth.workload_sparse_pixels(N=3000, L_unique=333)
    path = tmp_path / "tune.txt"
    ch = elm.elm_autotune(ctx, problem(p), precision=elm.PREC_MIXED, path=str(path))
    assert ch["panel_cluster"] in (8, 16) and ch["panel_width"] in (16, 24, 32)
    assert ch["hidden_stages"] in (2, 3) and ch["gram_stages"] in (2, 3)
    assert ch["best_ms"] > 0
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    assert lines[0] == "%s cs=%d nb=%d hs=%d gs=%d lanes=0" % (
        bucket(elm.PREC_MIXED, p), ch["panel_cluster"], ch["panel_width"],
        ch["hidden_stages"], ch["gram_stages"])
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    c2 = elm.elm_create(0, torch.cuda.current_stream())
    try:
        elm.elm_autotune_load(c2, str(path))
        prob = problem(p)
        res = elm.elm_train(c2, prob, precision=elm.PREC_MIXED)[0]
        assert res["rank"] == r
        assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-6
    finally:
        c2.close()


def test_fp64_choice_and_a_second_bucket_in_the_same_file(elm, ctx, tmp_path):
    path = tmp_path / "tune.txt"
    p1 = synth.make_problem(2000, 16, 200, 3, n_dup=10)
    p2 = synth.make_problem(900, 9, 60, 2, act=synth.ACT_TANH, x_dtype=np.float64)
    elm.elm_autotune(ctx, problem(p1), precision=elm.PREC_MIXED, path=str(path))
    ch = elm.elm_autotune(ctx, problem(p2), precision=elm.PREC_FP64, path=str(path))
    assert ch["panel_width"] in (16, 24) and ch["hidden_stages"] == 0 and ch["gram_stages"] == 0
    keys = sorted(l.split()[0] for l in path.read_text().splitlines())
    assert keys == sorted([bucket(elm.PREC_MIXED, p1), bucket(elm.PREC_FP64, p2)])
    prob = problem(p2)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_FP64)[0]
    ref, r, _ = oracle.train(p2["X"], p2["W"], p2["b"], p2["a"], p2["act"], p2["T"])
    assert res["rank"] == r and rel(prob["beta"].cpu().numpy(), ref) <= 1e-9


def test_batched_call_lanes(elm, ctx, tmp_path):
    path = tmp_path / "tune.txt"
    ps = [synth.make_problem(1500 + 300 * i, 16, 100 + 40 * i, 3) for i in range(6)]
    probs = [problem(p) for p in ps]
    ch = elm.elm_autotune(ctx, probs, precision=elm.PREC_MIXED, path=str(path))
    assert ch["lanes"] in (1, 2, 4, 8)
    assert path.read_text().split()[0] == "p1_batch2"
    res = elm.elm_train(ctx, probs, precision=elm.PREC_MIXED)
    for p, pr, r in zip(ps, probs, res):
        ref, rr, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
        assert r["rank"] == rr and rel(pr["beta"].cpu().numpy(), ref) <= 1e-6


def test_load_skips_bad_lines_and_rejects_a_missing_file(elm, ctx, tmp_path):
    path = tmp_path / "tune.txt"
    path.write_text("p1_L9_N12_n4 cs=8 nb=24 hs=3 gs=2 lanes=0\n"
                    "garbage\n"
                    "p1_L9_N12_n5 cs=12 nb=24 hs=3 gs=2 lanes=0\n")     # cs outside {8, 16}
    elm.elm_autotune_load(ctx, str(path))
    with pytest.raises(elm.ElmError):
        elm.elm_autotune_load(ctx, str(tmp_path / "missing.txt"))
