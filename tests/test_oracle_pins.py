"""Pins for the FP64 CPU oracle: each check ties it to something other than
itself (hand-worked values, closed forms, LAPACK/SVD library routines,
invariants), chosen so that a dropped term, a sign or index error or a
transposed operand in any oracle routine fails at least one of them.
"""
import json
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def closed(expr):
    return eval(expr, {"sqrt": math.sqrt})


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def small(N=60, n=5, L_unique=10, m=3, n_dup=0, n_scaled=0, **kw):
    return synth.make_problem(N, n, L_unique, m, n_dup=n_dup, n_scaled=n_scaled,
                              x_dtype=np.float64, **kw)


# ---------------------------------------------------------------- hidden layer
def test_hidden_worked_example():
    g = load("hidden_worked.json")
    X, W, b = np.array(g["X"]), np.array(g["W"]), np.array(g["b"])
    assert oracle.hidden(X, W, b, act=0)[0, 0] == pytest.approx(float(Decimal(g["sigmoid"])), rel=4 * U)
    assert oracle.hidden(X, W, b, act=1)[0, 0] == pytest.approx(float(Decimal(g["tanh"])), rel=4 * U)


def test_hidden_special_values_and_symmetry():
    p = small(N=50, n=7, L_unique=9)
    X, W, b = p["X"], p["W"], p["b"]
    H0 = oracle.hidden(np.zeros_like(X), W, np.zeros_like(b))
    assert np.all(H0 == 0.5)                                  # g(0) = 1/2
    assert np.all(oracle.hidden(np.zeros_like(X), W, np.zeros_like(b), act=1) == 0.0)
    H = oracle.hidden(X, W, b)
    Hn = oracle.hidden(X, -W, -b)
    assert np.max(np.abs(H + Hn - 1.0)) < 4 * U               # g(z) + g(-z) = 1
    Ht = oracle.hidden(X, W, b, act=1)
    assert np.max(np.abs(Ht + oracle.hidden(X, -W, -b, act=1))) < 4 * U   # odd
    a = np.ldexp(1.0, np.arange(9) % 3 - 1) * np.where(np.arange(9) % 2, -1, 1)
    assert np.array_equal(oracle.hidden(X, W, b, a), H * a)   # output scale
    # bias enters once per neuron: shifting b by c equals a constant input column
    Xa = np.hstack([X, np.ones((X.shape[0], 1))])
    Wa = np.vstack([W, np.full((1, 9), 0.25)])
    assert np.max(np.abs(oracle.hidden(Xa, Wa, b) - oracle.hidden(X, W, b + 0.25))) < 8 * U


def test_hidden_matches_numpy_matmul():
    p = small(N=80, n=13, L_unique=21)
    H = oracle.hidden(p["X"], p["W"], p["b"])
    Z = p["X"] @ p["W"] + p["b"]
    assert np.max(np.abs(H - 1.0 / (1.0 + np.exp(-Z)))) < 1e-14


# ---------------------------------------------------------------- Gram
def test_gram_matches_blas_and_is_symmetric_psd():
    p = small(N=300, n=6, L_unique=17, m=4)
    H = oracle.hidden(p["X"], p["W"], p["b"])
    S, Z = oracle.gram(H, p["T"])
    assert rel(S, H.T @ H) < 1e-14
    assert rel(Z, H.T @ p["T"]) < 1e-14
    assert np.array_equal(S, S.T)
    assert np.linalg.eigvalsh(S).min() > -1e-12 * np.trace(S)
    S2, Z2 = oracle.gram(np.asfortranarray(H[:, ::-1]), p["T"])
    assert rel(S2, S[::-1, ::-1]) < 1e-14                     # orientation check


# ---------------------------------------------------------------- pivoted Cholesky
def test_pivchol_worked_full_rank():
    g = load("pivchol_spd3.json")
    r, perm, R = oracle.pivchol(np.array(g["S"], dtype=float))
    assert r == g["rank"]
    assert list(perm) == g["perm"]
    Rx = np.array([[closed(e) for e in row] for row in g["R_closed_form"]])
    assert np.max(np.abs(R[:r] - Rx)) < 1e-14


def test_pivchol_worked_rank_deficient():
    g = load("pivchol_rank2.json")
    r, perm, R = oracle.pivchol(np.array(g["S"], dtype=float))
    assert r == g["rank"]
    assert list(perm) == g["perm"]
    Rx = np.array([[closed(e) for e in row] for row in g["R_closed_form"]])
    assert np.max(np.abs(R[:r] - Rx)) < 1e-14
    K = np.linalg.solve(R[:r, :r], R[:r, r:])
    assert np.max(np.abs(K - np.array(g["K"]))) < 1e-14


def test_pivchol_reconstructs_permuted_gram():
    p = small(N=400, n=8, L_unique=30, n_dup=5, n_scaled=4)
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"])
    S, _ = oracle.gram(H)
    r, perm, R = oracle.pivchol(S)
    assert r == 30
    SP = S[np.ix_(perm, perm)]
    R1 = R[:r]
    assert rel(R1.T @ R1, SP) < 1e-12                         # P^T S P = R^T R
    assert sorted(perm) == list(range(S.shape[0]))
    assert list(perm[r:]) == sorted(perm[r:])
    # pivots are non-increasing on the equilibrated scale
    dg = np.diag(R1) ** 2 / np.diag(S)[perm[:r]]
    assert np.all(np.diff(dg) <= 1e-12)


# ---------------------------------------------------------------- pseudoinverse (Eq. 5)
@pytest.mark.parametrize("n_dup,n_scaled", [(0, 0), (3, 0), (2, 3)])
def test_penrose_conditions(n_dup, n_scaled):
    p = small(N=40, n=4, L_unique=9, n_dup=n_dup, n_scaled=n_scaled)
    H = oracle.hidden(p["X"], p["W"], p["b"], p["a"])
    X, r = oracle.pinv(H)
    assert r == 9
    sv = np.linalg.svd(H, compute_uv=False)
    kappa = sv[0] / sv[r - 1]
    tol = 100 * kappa ** 2 * U
    nH, nX = np.linalg.norm(H, 2), np.linalg.norm(X, 2)
    assert np.linalg.norm(H @ X @ H - H, 2) <= tol * nH
    assert np.linalg.norm(X @ H @ X - X, 2) <= tol * nX
    assert np.linalg.norm((H @ X).T - H @ X, 2) <= tol
    assert np.linalg.norm((X @ H).T - X @ H, 2) <= tol


def test_closed_form_eq8_full_rank():
    p = small(N=500, n=10, L_unique=40, m=5)
    H = oracle.hidden(p["X"], p["W"], p["b"])
    beta, r, _ = oracle.train(p["X"], p["W"], p["b"], None, 0, p["T"], nrefine=0)
    assert r == 40
    ref = np.linalg.solve(H.T @ H, H.T @ p["T"])              # Eq. 8 via LAPACK
    k = np.linalg.cond(H)
    assert rel(beta, ref) < 50 * k * k * U


@pytest.mark.parametrize("n_dup,n_scaled", [(4, 0), (3, 5)])
def test_matches_svd_pseudoinverse(n_dup, n_scaled):
    p = small(N=300, n=6, L_unique=25, m=4, n_dup=n_dup, n_scaled=n_scaled)
    beta, r, _, H = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"], return_h=True)
    assert r == 25
    ref = np.linalg.pinv(H, rcond=1e-10) @ p["T"]             # SVD route
    assert rel(beta, ref) < 1e-10
    ls = np.linalg.lstsq(H, p["T"], rcond=1e-10)[0]           # min-norm LS
    assert rel(beta, ls) < 1e-10


def test_duplicate_neuron_closed_form():
    """beta_j = a_j beta_u[g] / sum_{i in g} a_i^2 (min-norm share of a group)."""
    p = small(N=400, n=7, L_unique=20, m=3, n_dup=6, n_scaled=5)
    beta, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"])
    src, scale = p["src"], p["scale"]
    uniq = [int(np.nonzero((src == g) & (scale == 1.0))[0][0]) for g in range(20)]
    Hu = oracle.hidden(p["X"], p["W"][:, uniq], p["b"][uniq])
    bu = np.linalg.lstsq(Hu, p["T"], rcond=None)[0]
    expect = np.empty_like(beta)
    for j in range(beta.shape[0]):
        g = src[j]
        expect[j] = scale[j] * bu[g] / np.sum(scale[src == g] ** 2)
    assert rel(beta, expect) < 1e-10
    # duplicated neurons share equally
    for g in range(20):
        cols = np.nonzero((src == g) & (scale == 1.0))[0]
        for c in cols[1:]:
            assert np.max(np.abs(beta[c] - beta[cols[0]])) < 1e-11 * np.abs(beta).max()


# ---------------------------------------------------------------- invariants
def test_invariants_permutation_scale_residual():
    p = small(N=500, n=9, L_unique=30, m=4, n_dup=3)
    X, W, b, T = p["X"], p["W"], p["b"], p["T"]
    beta, r, _, H = oracle.train(X, W, b, None, 0, T, return_h=True)
    pi = synth.permutation(7, W.shape[1])
    bp, rp, _ = oracle.train(X, W[:, pi], b[pi], None, 0, T)
    assert rp == r and rel(bp, beta[pi]) < 1e-11                # column perm -> row perm
    b2, _, _ = oracle.train(X, W, b, np.full(W.shape[1], 2.0), 0, T)
    assert rel(b2, beta / 2) < 1e-11                          # H*2 -> beta/2
    G = H.T @ (T - H @ beta)                                  # normal equations
    assert np.linalg.norm(G) < 1e-10 * np.linalg.norm(H) ** 2 * np.linalg.norm(beta)


def test_refinement_reduces_error():
    """kappa(H) ~ 2e4: the normal equations alone lose ~kappa^2 u; two
    corrections with the exact residual recover ~kappa u."""
    p = small(N=800, n=4, L_unique=20, m=2)
    H = oracle.hidden(p["X"], p["W"], p["b"])
    ref = np.linalg.lstsq(H, p["T"], rcond=None)[0]
    e0 = rel(oracle.train(p["X"], p["W"], p["b"], None, 0, p["T"], nrefine=0)[0], ref)
    e2 = rel(oracle.train(p["X"], p["W"], p["b"], None, 0, p["T"], nrefine=2)[0], ref)
    assert e0 > 1e-10 and e2 < 1e-3 * e0 and e2 < 1e-11


# ---------------------------------------------------------------- Eqs. 19-23
@pytest.mark.parametrize("r1", [1, 6, 11])
def test_block_formula_full_rank_split(r1):
    p = small(N=120, n=5, L_unique=12, m=3)
    H = oracle.hidden(p["X"], p["W"], p["b"])
    beta = oracle.block_rbp(H, r1, p["T"])
    ref = np.linalg.solve(H.T @ H, H.T @ p["T"])
    assert rel(beta, ref) < 1e-8
    assert rel(oracle.train(p["X"], p["W"], p["b"], None, 0, p["T"])[0], beta) < 1e-8


def test_block_formula_singular_when_rank_deficient():
    """With r < L and H2 = H1 K, D = H1^T C H1 is singular: the reason the
    oracle reads the method through the full-rank factorisation."""
    p = small(N=120, n=5, L_unique=8, m=2, n_dup=3)
    H = oracle.hidden(p["X"], p["W"], p["b"])
    S, _ = oracle.gram(H)
    r, perm, _ = oracle.pivchol(S)
    assert r == 8
    with pytest.raises(np.linalg.LinAlgError):
        oracle.block_rbp(H[:, perm], r, p["T"])


# ---------------------------------------------------------------- ranks of the workloads
def test_rank_small_fp64_workload_and_margin():
    p = synth.workload_small_fp64()
    beta, r, perm, H = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"], return_h=True)
    assert r == 180
    S, _ = oracle.gram(H)
    tau = oracle.default_tau(200)
    rr, perm2, R = oracle.pivchol(S, tau=0.0)                 # run past the rank
    piv = np.diag(R) ** 2 / np.diag(S)[perm2]                 # unit-diagonal pivots
    assert piv[179] > 1e6 * tau                               # accepted margin
    assert np.all(np.abs(piv[180:rr]) < 1e-2 * tau)           # rejected margin
    ref = np.linalg.pinv(H, rcond=1e-10) @ p["T"]
    assert rel(beta, ref) < 1e-9


def test_rank_deficient_recipe_small():
    p = synth.workload_rank_deficient(N=3000, L_unique=200, n_dup=20, n_scaled=10,
                                      x_dtype=np.float64)
    beta, r, _, H = oracle.train(p["X"], p["W"], p["b"], p["a"], 0, p["T"], return_h=True)
    assert r == 200
    ref = np.linalg.pinv(H, rcond=1e-10) @ p["T"]
    assert rel(beta, ref) < 1e-9


def test_predict_is_h_beta():
    p = small(N=70, n=6, L_unique=11, m=3)
    beta, _, _, H = oracle.train(p["X"], p["W"], p["b"], None, 0, p["T"], return_h=True)
    Y = oracle.predict(p["X"], p["W"], p["b"], None, 0, beta)
    assert rel(Y, H @ beta) < 1e-14
