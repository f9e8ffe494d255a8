"""Write the oracle's results for the full-size workloads to tests/golden/.

  python tests/golden/make_full_goldens.py [rank_deficient] [batched] [large] [sparse_pixels]

Calls only the seeded input generators (synth) and the FP64 CPU oracle
(oracle/); nothing here touches the GPU library.  For every problem it stores

  * beta = H^+ T from the oracle's training (Alg. 1 and Eq. 5: hidden layer,
    Gram blocks, pivoted rank decision, full-rank solve, two refinement
    steps), element by element;
  * the rank r and the rank-decision margins on the unit-diagonal scale
    (Eq. 6, Alg. 1 steps 3-4): the smallest accepted pivot and the largest
    remaining diagonal of the rejected columns, against tau = L 2^-52;
  * the conditioning of the equilibrated H1 (kappa from the eigenvalues of
    its unit-diagonal Gram) and the least-squares residual, from which the
    parity tests take the forward-error scale of each problem;
  * fingerprints of the inputs (SHA-256 of X, W, b, a; norms of T), so the
    tests can check that they see the same bytes.

The steps of the oracle's training are taken one routine at a time (as
oracle.train runs them) so that the Gram and the factor can be kept for the
margins; a self-check first confirms on a small problem that this gives
bitwise the same beta as oracle.train.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def digest(a) -> str:
    if a is None:
        return ""
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def fingerprint(p) -> dict:
    T = p["T"]
    return dict(X=digest(p["X"]), W=digest(p["W"]), b=digest(p["b"]), a=digest(p.get("a")),
                T_norm=float(np.linalg.norm(T)),
                T_wsum=float(np.sum(T * (1.0 + np.arange(T.size).reshape(T.shape) % 7))))


def train_by_steps(p):
    """oracle.train's steps one routine at a time; returns what the goldens
    keep.  Refinement: Rres = T - H beta, G = H^T Rres, beta += frsolve(G),
    twice, as orc_train does."""
    X, W, b, a, act, T = p["X"], p["W"], p["b"], p.get("a"), int(p["act"]), p["T"]
    H = oracle.hidden(X, W, b, a, act)
    S, Z = oracle.gram(H, T)
    r, perm, R = oracle.pivchol(S)
    beta = oracle.frsolve(R, r, perm, Z)
    for _ in range(2):
        Res = T - oracle.matmul_hb(H, beta)
        G = oracle.gram(H, Res)[1]
        beta = beta + oracle.frsolve(R, r, perm, G)
    L = S.shape[0]
    d = np.diag(S).copy()
    acc = np.diag(R)[:r] ** 2 / d[perm[:r]]              # accepted pivots, unit scale
    rej = 0.0
    if r < L:
        Rs = R[:r, r:] / np.sqrt(d[perm[r:]])[None, :]
        rej = float(np.max(1.0 - np.sum(Rs * Rs, axis=0)))   # remaining diagonals
    s = 1.0 / np.sqrt(d)
    Se = (S * s[:, None]) * s[None, :]
    idx = perm[:r]
    ev = np.linalg.eigvalsh(Se[np.ix_(idx, idx)])
    kappa = float(np.sqrt(ev[-1] / ev[0])) if ev[0] > 0 else float("inf")
    res = T - oracle.matmul_hb(H, beta)
    out = dict(beta=beta, rank=r, tau=oracle.default_tau(L), piv_min=float(acc.min()),
               rejected_max=rej, kappa=kappa, ev_max=float(ev[-1]), ev_min=float(ev[0]),
               res_norm=float(np.linalg.norm(res)), beta_norm=float(np.linalg.norm(beta)),
               t_norm=float(np.linalg.norm(T)), h_fro=float(np.sqrt(np.sum(d))))
    return out


def self_check():
    p = synth.make_problem(700, 12, 60, 3, n_dup=5, n_scaled=4, x_kind="uniform11",
                           act=synth.ACT_TANH)
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    g = train_by_steps(p)
    assert g["rank"] == r and np.array_equal(g["beta"], ref), "steps differ from oracle.train"


WORKLOADS = {
    "sparse_pixels": lambda: [synth.workload_sparse_pixels()],
    "rank_deficient": lambda: [synth.workload_rank_deficient()],
    "batched": lambda: synth.workload_batched(),
    "large": lambda: [synth.workload_large()],
}


def write(name):
    t0 = time.time()
    probs = WORKLOADS[name]()
    arrays = {}
    for i, p in enumerate(probs):
        g = train_by_steps(p)
        fp = fingerprint(p)
        arrays["beta_%03d" % i] = g.pop("beta")
        for k, v in g.items():
            arrays.setdefault(k, []).append(v)
        for k, v in fp.items():
            arrays.setdefault("fp_" + k, []).append(v)
        print("%s %d/%d rank %d kappa %.3g piv_min %.3g (%.0f s)"
              % (name, i + 1, len(probs), g["rank"], g["kappa"], g["piv_min"],
                 time.time() - t0), flush=True)
        del p
    for k in list(arrays):
        if not k.startswith("beta_"):
            arrays[k] = np.array(arrays[k])
    arrays["count"] = np.array(len(probs))
    path = os.path.join(HERE, "full_%s.npz" % name)
    np.savez_compressed(path, **arrays)
    print("wrote", path, "%.0f s" % (time.time() - t0), flush=True)


if __name__ == "__main__":
    self_check()
    for nm in (sys.argv[1:] or ["rank_deficient", "batched", "large"]):
        write(nm)
