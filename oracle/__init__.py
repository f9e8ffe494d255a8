"""Python access to the plain FP64 CPU oracle (oracle/elm_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the GPU smoke check and the benchmark's
CPU-baseline leg use it; the GPU library never imports it.  Every function
takes and returns numpy float64 arrays in the paper's orientation (H is
N x L, beta is L x m).  See elm_oracle.c for the passage each routine
follows.  Parity unpinned: none (every routine is pinned by
tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes as C
import os
import numpy as np

from . import build as _build

_lib = None
_d = C.POINTER(C.c_double)
_i64 = C.c_int64
_pi = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB lets the mutation test load a deliberately broken copy.
        path = os.environ.get("ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        L.orc_hidden.argtypes = [_d, _i64, _i64, _d, _i64, _d, _d, C.c_int, _d]
        L.orc_gram.argtypes = [_d, _i64, _i64, _d, _i64, _d, _d]
        L.orc_pivchol.argtypes = [_d, _i64, C.c_double, _pi, _d]
        L.orc_pivchol.restype = _i64
        L.orc_frsolve.argtypes = [_d, _i64, _i64, _pi, _d, _i64, _d]
        L.orc_frsolve.restype = C.c_int
        L.orc_train.argtypes = [_d, _i64, _i64, _d, _i64, _d, _d, C.c_int,
                                _d, _i64, C.c_double, C.c_int, _d, _pi, _d]
        L.orc_train.restype = _i64
        L.orc_pinv.argtypes = [_d, _i64, _i64, C.c_double, _d]
        L.orc_pinv.restype = _i64
        L.orc_predict.argtypes = [_d, _i64, _i64, _d, _i64, _d, _d, C.c_int,
                                  _d, _i64, _d]
        L.orc_matmul_hb.argtypes = [_d, _i64, _i64, _d, _i64, _d]
        L.orc_default_tau.argtypes = [_i64]
        L.orc_default_tau.restype = C.c_double
        L.orc_block_rbp.argtypes = [_d, _i64, _i64, _i64, _d, _i64, _d]
        L.orc_block_rbp.restype = C.c_int
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(_d)


def default_tau(L: int) -> float:
    return lib().orc_default_tau(L)


def hidden(X, W, b, a=None, act=0):
    X, W, b = _f64(X), _f64(W), _f64(b)
    a = None if a is None else _f64(a)
    N, n = X.shape
    L = W.shape[1]
    H = np.empty((N, L))
    lib().orc_hidden(_p(X), N, n, _p(W), L, _p(b), _p(a), act, _p(H))
    return H


def gram(H, T=None):
    H = _f64(H)
    N, L = H.shape
    m = 0 if T is None else T.shape[1]
    T = None if T is None else _f64(T)
    S = np.empty((L, L))
    Z = np.empty((L, max(m, 1)))
    lib().orc_gram(_p(H), N, L, _p(T), m, _p(S), _p(Z))
    return S, Z[:, :m]


def pivchol(S, tau=None):
    S = _f64(S)
    L = S.shape[0]
    perm = np.empty(L, dtype=np.int64)
    R = np.empty((L, L))
    r = lib().orc_pivchol(_p(S), L, default_tau(L) if tau is None else tau,
                          perm.ctypes.data_as(_pi), _p(R))
    return int(r), perm, R


def frsolve(R, r, perm, Z):
    R, Z = _f64(R), _f64(Z)
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    L = R.shape[0]
    m = Z.shape[1]
    beta = np.empty((L, m))
    rc = lib().orc_frsolve(_p(R), L, r, perm.ctypes.data_as(_pi), _p(Z), m, _p(beta))
    if rc != 0:
        raise RuntimeError("orc_frsolve: I + K K^T not positive definite")
    return beta


def train(X, W, b, a, act, T, tau=None, nrefine=2, return_h=False):
    """Alg. 1 end to end: returns (beta L x m, rank, perm[, H])."""
    X, W, b, T = _f64(X), _f64(W), _f64(b), _f64(T)
    a = None if a is None else _f64(a)
    N, n = X.shape
    L = W.shape[1]
    m = T.shape[1]
    beta = np.empty((L, m))
    perm = np.empty(L, dtype=np.int64)
    H = np.empty((N, L)) if return_h else None
    r = lib().orc_train(_p(X), N, n, _p(W), L, _p(b), _p(a), act, _p(T), m,
                        -1.0 if tau is None else tau, nrefine, _p(beta),
                        perm.ctypes.data_as(_pi), _p(H))
    if r < 0:
        raise RuntimeError("orc_train failed")
    return (beta, int(r), perm, H) if return_h else (beta, int(r), perm)


def pinv(H, tau=None):
    H = _f64(H)
    N, L = H.shape
    Hp = np.empty((L, N))
    r = lib().orc_pinv(_p(H), N, L, -1.0 if tau is None else tau, _p(Hp))
    return Hp, int(r)


def predict(X, W, b, a, act, beta):
    X, W, b, beta = _f64(X), _f64(W), _f64(b), _f64(beta)
    a = None if a is None else _f64(a)
    N, n = X.shape
    L = W.shape[1]
    m = beta.shape[1]
    Y = np.empty((N, m))
    lib().orc_predict(_p(X), N, n, _p(W), L, _p(b), _p(a), act, _p(beta), m, _p(Y))
    return Y


def matmul_hb(H, beta):
    H, beta = _f64(H), _f64(beta)
    N, L = H.shape
    m = beta.shape[1]
    Y = np.empty((N, m))
    lib().orc_matmul_hb(_p(H), N, L, _p(beta), m, _p(Y))
    return Y


def block_rbp(H, r1, Y):
    """Eqs. 19-23 for a full-rank H split after column r1."""
    H, Y = _f64(H), _f64(Y)
    N, L = H.shape
    m = Y.shape[1]
    beta = np.empty((L, m))
    rc = lib().orc_block_rbp(_p(H), N, L, r1, _p(Y), m, _p(beta))
    if rc != 0:
        raise np.linalg.LinAlgError("A or D singular")
    return beta
