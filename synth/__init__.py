"""Seeded synthetic ELM workloads.

This module only draws inputs: random numbers, the hidden-neuron layout
(unique neurons, exact duplicates, power-of-two scaled copies) and targets.
It holds none of the training arithmetic (no hidden layer, no Gram, no
factorisation).  Both the CPU oracle's tests and the GPU path's tests and
benchmark take their inputs from here, so both sides see identical bytes.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated in counter form:
output i of the stream with seed s is mix(s + (i+1)*0x9E3779B97F4A7C15).
Uniform doubles use the top 53 bits; Gaussians use Box-Muller.

The paper's datasets (OCRHD, 3823x65, and GINA, 3468x971; Section 4) are not
available, so the workloads below are synthetic stand-ins with the shapes the
experiments call for: random input weights and biases (Algorithm 1, step 1),
a sigmoid hidden layer (Section 4), one-hot class targets.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
SEED_BASE = 0x201102436

ACT_SIGMOID = 0
ACT_TANH = 1


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 stream `seed`."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    x = splitmix64(seed, n)
    return ((x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)).reshape(shape)


def uniform(seed: int, shape, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, shape)


def normal(seed: int, shape, std: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape))
    u = uniform01(seed, (2 * n,))
    u1 = 1.0 - u[:n]          # (0, 1]
    u2 = u[n:]
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return (std * z).reshape(shape)


def permutation(seed: int, n: int) -> np.ndarray:
    """Seeded permutation of range(n): stable argsort of uniform keys."""
    return np.argsort(uniform01(seed, (n,)), kind="stable")


def integers(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on [lo, hi] (inclusive)."""
    u = uniform01(seed, (count,))
    return lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)


def one_hot(labels: np.ndarray, m: int) -> np.ndarray:
    T = np.zeros((labels.shape[0], m), dtype=np.float64)
    T[np.arange(labels.shape[0]), labels] = 1.0
    return T


def neuron_layout(seed: int, L_unique: int, n_dup: int, n_scaled: int):
    """Columns of the hidden layer as (source unique neuron, output scale).

    The first L_unique columns are unique neurons.  n_dup further columns
    copy a distinct unique neuron exactly; n_scaled copy a distinct unique
    neuron with output scale +-2^k, k in {-1, 1, 2}, so that the copy is an
    exact multiple of its source in every binary format.  All columns are
    then shuffled by a seeded permutation.  Returns (src, scale, expected
    rank).
    """
    L = L_unique + n_dup + n_scaled
    if n_dup + n_scaled > L_unique:
        raise ValueError("more copies than unique neurons")
    src = np.arange(L, dtype=np.int64)
    scale = np.ones(L)
    picks = permutation(seed + 1, L_unique)[: n_dup + n_scaled]
    src[L_unique:L_unique + n_dup] = picks[:n_dup]
    src[L_unique + n_dup:] = picks[n_dup:]
    if n_scaled:
        k = np.array([-1, 1, 2])[integers(seed + 2, n_scaled, 0, 2)]
        sgn = np.where(uniform01(seed + 3, (n_scaled,)) < 0.5, -1.0, 1.0)
        scale[L_unique + n_dup:] = sgn * np.ldexp(1.0, k)
    order = permutation(seed + 4, L)
    return src[order], scale[order], L_unique


def make_problem(N: int, n: int, L_unique: int, m: int, *, n_dup: int = 0,
                 n_scaled: int = 0, x_kind: str = "uniform01",
                 x_dtype=np.float32, act: int = ACT_SIGMOID,
                 target: str = "classes", seed: int = SEED_BASE,
                 x_sparsity: float = 0.0) -> dict:
    """One synthetic ELM training problem.

    x_kind: 'uniform01' (U[0,1]), 'uniform11' (U[-1,1]) or 'normal' (N(0,1)).
    x_sparsity: probability that an entry of X is zero (sparse-pixel-like).
    target: 'classes' -> one-hot {0,1} labels from argmax of a fixed random
    linear map of X; 'regression' -> sin of random projections + N(0, 0.01^2).
    W (n x L) and b (L) are U[-1,1]; a (L) is the per-neuron output scale
    (None when every column is unscaled).
    """
    if x_kind == "uniform01":
        X = uniform01(seed + 10, (N, n))
    elif x_kind == "uniform11":
        X = uniform(seed + 10, (N, n), -1.0, 1.0)
    elif x_kind == "normal":
        X = normal(seed + 10, (N, n))
    else:
        raise ValueError(x_kind)
    if x_sparsity > 0.0:
        X[uniform01(seed + 11, (N, n)) < x_sparsity] = 0.0
    X = X.astype(x_dtype)
    src, scale, rank = neuron_layout(seed + 20, L_unique, n_dup, n_scaled)
    Wu = uniform(seed + 30, (n, L_unique), -1.0, 1.0)
    bu = uniform(seed + 31, (L_unique,), -1.0, 1.0)
    W = np.ascontiguousarray(Wu[:, src])
    b = np.ascontiguousarray(bu[src])
    a = None if np.all(scale == 1.0) else scale
    Xd = X.astype(np.float64)
    if target == "classes":
        V = uniform(seed + 40, (n, m), -1.0, 1.0)
        labels = np.argmax(Xd @ V, axis=1)
        T = one_hot(labels, m)
    elif target == "regression":
        P = normal(seed + 40, (n, m), std=1.0 / np.sqrt(n))
        T = np.sin(Xd @ P) + normal(seed + 41, (N, m), std=0.01)
        labels = None
    else:
        raise ValueError(target)
    return dict(X=np.ascontiguousarray(X), W=W, b=b, a=a, act=act,
                T=np.ascontiguousarray(T), labels=labels, rank=rank,
                src=src, scale=scale, N=N, n=n, L=W.shape[1], m=m)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes are the full ones; every function takes keyword
# overrides so tests can draw the same recipe at smaller sizes.
# ---------------------------------------------------------------------------

def workload_small_fp64(**kw):
    """2000x16 U[0,1] FP64 inputs, L=200 sigmoid (180 unique + 20 exact
    duplicates -> rank 180), 4 one-hot classes."""
    args = dict(N=2000, n=16, L_unique=180, m=4, n_dup=20,
                x_kind="uniform01", x_dtype=np.float64,
                seed=SEED_BASE + 1000 * 1)
    args.update(kw)
    return make_problem(**args)


def workload_sparse_pixels(**kw):
    """60000x784, entries 0 w.p. 0.8 else U[0,1] (FP32), L=2000 sigmoid,
    10 one-hot classes, full column rank (MNIST/GINA-like shapes)."""
    args = dict(N=60000, n=784, L_unique=2000, m=10, x_kind="uniform01",
                x_sparsity=0.8, x_dtype=np.float32, seed=SEED_BASE + 1000 * 2)
    args.update(kw)
    return make_problem(**args)


def workload_rank_deficient(**kw):
    """100000x64 N(0,1) FP32, L=6000 sigmoid = 5100 unique + 600 exact
    duplicates + 300 power-of-two scaled copies (rank 5100), 3 regression
    targets sin(X p_k) + N(0, 0.01^2) with p_k ~ N(0, 1/64)."""
    args = dict(N=100000, n=64, L_unique=5100, m=3, n_dup=600, n_scaled=300,
                x_kind="normal", x_dtype=np.float32, target="regression",
                seed=SEED_BASE + 1000 * 3)
    args.update(kw)
    return make_problem(**args)


def workload_batched(count: int = 128, N_range=(5000, 50000),
                     L_range=(100, 3000), d_choices=(16, 54, 128),
                     m_range=(2, 26), seed: int = SEED_BASE + 1000 * 4, only=None):
    """`count` independent uneven problems: N uniform in N_range, d in
    d_choices, L uniform in L_range, sigmoid/tanh 50/50, m one-hot classes
    uniform in m_range, X U[0,1] FP32.  only: indices of the problems to
    generate (the same bytes as in the full list)."""
    Ns = integers(seed + 1, count, *N_range)
    ds = np.array(d_choices)[integers(seed + 2, count, 0, len(d_choices) - 1)]
    Ls = integers(seed + 3, count, *L_range)
    acts = (uniform01(seed + 4, (count,)) >= 0.5).astype(int)
    ms = integers(seed + 5, count, *m_range)
    return [make_problem(int(Ns[i]), int(ds[i]), int(Ls[i]), int(ms[i]),
                         act=int(acts[i]), x_dtype=np.float32,
                         seed=seed + 100 * (i + 1))
            for i in (range(count) if only is None else only)]


def workload_gina_shaped(L: int = 2000, **kw):
    """The shape of the paper's Table 1 experiment (3468 samples x 971
    features, L in {500, 1000, 1500, 2000}, sigmoid, two classes) on
    synthetic inputs: entries 0 w.p. 0.8 else U[0,1] (FP32)."""
    args = dict(N=3468, n=971, L_unique=L, m=2, x_kind="uniform01", x_sparsity=0.8,
                x_dtype=np.float32, seed=SEED_BASE + 1000 * 6 + L)
    args.update(kw)
    return make_problem(**args)


def workload_large(**kw):
    """500000x128 U[-1,1] FP32, L=8000 sigmoid, 20 one-hot classes."""
    args = dict(N=500000, n=128, L_unique=8000, m=20, x_kind="uniform11",
                x_dtype=np.float32, seed=SEED_BASE + 1000 * 5)
    args.update(kw)
    return make_problem(**args)
