"""GPU parity of the mixed path (tensor-core digit products, FP64 rank
decision, factorisation and refinement) against the CPU oracle.

Bars: rank bit-exact; beta within 1e-6 relative Frobenius error; the
tensor-core hidden layer within 1e-9 absolute of the FP64 definition.
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


@pytest.mark.parametrize("N,n,L,xdt,act,kind,n_scaled", [
    (1037, 13, 120, np.float32, 0, "normal", 0),
    (300, 784, 333, np.float32, 0, "uniform01", 0),
    (65, 5, 7, np.float64, 1, "uniform11", 0),
    (777, 21, 90, np.float32, 1, "normal", 9),      # power-of-two output scales a_j
])
def test_hidden_tensor_core_matches_oracle(elm, ctx, N, n, L, xdt, act, kind, n_scaled):
    p = synth.make_problem(N, n, L, 3, n_dup=min(7, L // 3), n_scaled=n_scaled, x_dtype=xdt,
                           act=act, x_kind=kind, x_sparsity=0.8 if n == 784 else 0.0)
    t = to_dev(p)
    Lt = p["L"]
    Ht = elm.elm_hidden(ctx, t["X"], t["W"], t["b"], t["a"], act,
                        precision=elm.PREC_MIXED).cpu().numpy()
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"], act)
    assert Ht.shape == (Lt, N)
    assert np.max(np.abs(Ht.T - H)) < 1e-9
    src, sc = p["src"], p["scale"]
    for j in range(Lt):                                    # bitwise duplicates
        k = int(np.nonzero((src == src[j]) & (sc == 1.0))[0][0])
        assert np.array_equal(Ht[j], sc[j] * Ht[k])


def test_train_small_fp64_workload_mixed(elm, ctx):
    p = synth.workload_small_fp64()
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r == 180
    assert res["form"] == elm.FORM_MIXED                   # no hand-over to FP64
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-6


@pytest.mark.parametrize("case", ["sparse_pixels", "rank_deficient", "tanh_wide_m", "scaled"])
def test_train_reduced_workloads_mixed(elm, ctx, case):
    if case == "sparse_pixels":
        p = synth.workload_sparse_pixels(N=3000, L_unique=333)
    elif case == "rank_deficient":
        p = synth.workload_rank_deficient(N=4000, L_unique=250, n_dup=25, n_scaled=13)
    elif case == "tanh_wide_m":
        p = synth.make_problem(2500, 54, 301, 26, act=synth.ACT_TANH)
    else:
        p = synth.make_problem(1500, 20, 140, 5, n_dup=10, n_scaled=30, x_kind="uniform11")
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r == p["rank"]
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-6


@pytest.mark.parametrize("N,n,L,m", [(50, 8, 80, 3), (1, 3, 5, 1), (7, 1, 1, 1), (129, 65, 64, 17),
                                     (700, 33, 257, 2)])
def test_train_edge_shapes_mixed(elm, ctx, N, n, L, m):
    p = synth.make_problem(N, n, L, m, x_dtype=np.float64, x_kind="normal")
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-6


def test_train_host_buffers_mixed(elm, ctx):
    p = synth.make_problem(700, 9, 60, 4, n_dup=5)
    prob = dict(X=p["X"], W=p["W"], b=p["b"], a=p["a"], act=0, T=p["T"])
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"])
    assert res["rank"] == r
    assert rel(prob["beta"], ref) <= 1e-6


@pytest.mark.parametrize("xdt,bad", [(np.float32, np.nan), (np.float64, np.inf),
                                     (np.float32, -np.inf)])
def test_nonfinite_input_is_reported_mixed(elm, ctx, xdt, bad):
    # the digit slicer of X records the non-finite entry (no separate pass)
    p = synth.make_problem(300, 9, 40, 2, x_dtype=xdt)
    p["X"][117, 4] = bad
    res = elm.elm_train(ctx, problem(p), precision=elm.PREC_MIXED, check=False)[0]
    assert res["status"] == 4                                # ELM_ERR_NUMERIC


def test_train_many_targets_rank_deficient_mixed(elm, ctx):
    # m = 40 targets run the column passes of 32 + 8 in the residual and the
    # skinny K products; duplicates and scaled copies make r < L
    p = synth.make_problem(3000, 11, 150, 40, n_dup=20, n_scaled=10, x_kind="normal",
                           target="regression")
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r == 150
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-6


@pytest.mark.parametrize("n", [1100, 2100])
def test_deep_inputs_span_several_exact_chunks(elm, ctx, n):
    # n > 1024 inputs: the hidden layer's K range spans several exact chunks
    # (the drain's int64 running sums, then the double-float pre-activation)
    p = synth.make_problem(400, n, 70, 3, x_kind="uniform01", x_sparsity=0.5)
    t = to_dev(p)
    Ht = elm.elm_hidden(ctx, t["X"], t["W"], t["b"], t["a"], 0,
                        precision=elm.PREC_MIXED).cpu().numpy()
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"], 0)
    assert np.max(np.abs(Ht.T - H)) < 1e-9
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"])
    assert res["rank"] == r
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-6


@pytest.mark.parametrize("xdt", [np.float32, np.float64])
def test_train_pinned_host_inputs_mixed(elm, ctx, xdt):
    # page-locked host inputs (the e2e path of bench.py), staged by the library
    import torch
    p = synth.make_problem(1500, 37, 90, 3, n_dup=6, x_dtype=xdt, x_sparsity=0.3)
    prob = dict(X=torch.from_numpy(p["X"]).pin_memory(), W=torch.from_numpy(p["W"]).pin_memory(),
                b=torch.from_numpy(p["b"]).pin_memory(), a=None, act=0,
                T=torch.from_numpy(p["T"]).pin_memory(),
                beta=torch.empty((p["L"], 3), dtype=torch.float64).pin_memory())
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], None, 0, p["T"])
    assert res["rank"] == r == 90
    assert rel(prob["beta"].numpy(), ref) <= 1e-6
    bad = torch.from_numpy(p["X"]).pin_memory()
    bad[100, 5] = float("nan")
    res = elm.elm_train(ctx, dict(prob, X=bad), precision=elm.PREC_MIXED, check=False)[0]
    assert res["status"] == 4


@pytest.mark.parametrize("prec", [0, 1])
def test_repeated_trainings_replay_the_factorisation_graph(elm, ctx, prec):
    """The factorisation's launches are captured into a CUDA graph on the
    first training of a shape and replayed on the next ones (same
    workspaces): beta is bitwise the same every time, and the launch counter
    counts the replayed kernels like launched ones."""
    p = synth.make_problem(2500, 20, 260, 4, n_dup=12, n_scaled=5)
    prob = problem(p)
    betas, counts = [], []
    for _ in range(3):
        c0 = elm.elm_launch_counter()
        res = elm.elm_train(ctx, prob, precision=prec)[0]
        counts.append(elm.elm_launch_counter() - c0)
        betas.append(prob["beta"].cpu().numpy().copy())
    assert np.array_equal(betas[0], betas[1]) and np.array_equal(betas[1], betas[2])
    assert counts[1] == counts[2] and counts[0] >= counts[1] > 0
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["rank"] == r
    assert rel(betas[2], ref) <= (1e-9 if prec == 0 else 1e-6)


@pytest.mark.parametrize("near_dup", [0.0, 1e-3])
def test_mixed_factorisation_alone_is_double_float_accurate(elm, ctx, near_dup):
    """The mixed factorisation by itself (double-float pivot panels, trailing
    updates on the tensor cores from 8-bit digit slices while more than 256
    columns remain), with no refinement to hide its error: the full-rank
    solve of a Gram of L = 1100 columns agrees with the oracle's FP64 solve to
    L kappa 2^-44 (kappa of the Gram), where a single-float trailing update
    would be off by about kappa 2^-24.  near_dup > 0 pairs half the columns
    with near copies of the other half (kappa about 10^7), so the later panels
    work on small remaining diagonals and small per-column digit scales."""
    import torch
    rng = np.random.default_rng(5)
    N, L, m = 4000, 1100, 3
    H = rng.uniform(-1, 1, (N, L))
    if near_dup:
        H[:, L // 2:] = H[:, :L // 2] + near_dup * rng.uniform(-1, 1, (N, L // 2))
    T = rng.standard_normal((N, m))
    S0, Z0 = oracle.gram(H, T)
    r0, perm0, R0 = oracle.pivchol(S0)
    assert r0 == L
    ref = oracle.frsolve(R0, r0, perm0, Z0)
    kappa = np.linalg.cond(S0)
    S = torch.from_numpy(S0).cuda()
    f = elm.GramFactor(ctx, S, m, elm.PREC_MIXED)
    assert f.rank == L
    beta = f.solve(torch.from_numpy(Z0).cuda()).cpu().numpy()
    f.close()
    assert rel(beta, ref) <= L * kappa * 2.0 ** -44


def test_train_rank_deficient_k_on_tensor_cores(elm, ctx):
    """r = 700 independent neurons and q = 150 duplicates or power-of-two
    scaled copies: the mixed form forms K = R11^-1 R12 by 32-row blocks whose
    updates run on the tensor cores (ragged last block, q not a multiple of
    the 32-column tiles); rank exact, beta within the mixed bar."""
    p = synth.make_problem(4000, 40, 700, 5, n_dup=100, n_scaled=50, x_kind="normal")
    prob = problem(p)
    res = elm.elm_train(ctx, prob, precision=elm.PREC_MIXED)[0]
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert res["form"] == elm.FORM_MIXED   # settled in the mixed form, K on the tensor cores
    assert res["rank"] == r == 700
    assert rel(prob["beta"].cpu().numpy(), ref) <= 1e-6


def test_mixed_full_rank_route_of_a_rank_deficient_gram(elm, ctx):
    """The mixed factorisation and the full-rank route without refinement on
    a Gram of rank r = 900 with q = 197 exact duplicate columns (K = R11^-1
    R12 on the tensor cores): rank as the oracle's, and the solve within
    L kappa 2^-44 of the oracle's FP64 route (kappa of the independent
    columns' Gram), where a K of single-float accuracy would miss by about
    kappa 2^-24."""
    import torch
    rng = np.random.default_rng(8)
    N, r, q, m = 4000, 900, 197, 3
    H0 = rng.uniform(-1, 1, (N, r))
    H = np.concatenate([H0, H0[:, rng.integers(0, r, q)]], axis=1)
    H = H[:, rng.permutation(r + q)]
    T = rng.standard_normal((N, m))
    S0, Z0 = oracle.gram(H, T)
    tau = 1e-9
    r0, perm0, R0 = oracle.pivchol(S0, tau)
    assert r0 == r
    ref = oracle.frsolve(R0, r0, perm0, Z0)
    f = elm.GramFactor(ctx, torch.from_numpy(S0).cuda(), m, elm.PREC_MIXED, tol_rank=tau)
    assert f.rank == r
    beta = f.solve(torch.from_numpy(Z0).cuda()).cpu().numpy()
    f.close()
    S1 = S0[np.ix_(perm0[:r0], perm0[:r0])]
    assert rel(beta, ref) <= (r + q) * np.linalg.cond(S1) * 2.0 ** -44
