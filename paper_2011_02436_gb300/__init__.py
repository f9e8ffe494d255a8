"""GB300 rank-based pseudoinverse ELM (arXiv 2011.02436): Python binding of
the C ABI in include/elm.h.  Arguments are marshalled to pointers and sizes;
every step of the computation runs in libelm.so's CUDA kernels.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; rows must be
contiguous (last stride 1).  Outputs not supplied by the caller are
allocated as torch tensors on the device of the first input (or as numpy
arrays for host inputs).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _lib

ACT_SIGMOID, ACT_TANH = 0, 1
F32, F64 = 0, 1
PREC_FP64, PREC_MIXED, PREC_FP64_TC = 0, 1, 2
# largest padded sample and input counts of the exact tensor-core products:
# beyond them a mixed request runs the FP64 form with tensor-core products,
# and one of that form beyond EXACT_MAX_K the FP64 form
MIXED_MAX_ROWS, MIXED_MAX_INPUTS, EXACT_MAX_K = 8257536, 64512, 212735488
OK = 0


class ElmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_lib.load().elm_status_string(status).decode(),
                                                  status, msg))
        self.status = status


def _torch():
    import torch
    return torch


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return x.data_ptr()
    return x.ctypes.data


def _ld(x):
    if x.ndim == 1:
        return x.shape[0]
    if _is_torch(x):
        if x.stride(1) != 1:
            raise ValueError("rows must be contiguous")
        return x.stride(0)
    if x.strides[1] != x.itemsize:
        raise ValueError("rows must be contiguous")
    return x.strides[0] // x.itemsize


def _xdtype(X):
    name = str(X.dtype)
    if name.endswith("float32"):
        return F32
    if name.endswith("float64"):
        return F64
    raise TypeError("X must be float32 or float64")


def _empty_like_device(ref, shape, dtype=np.float64):
    if _is_torch(ref):
        torch = _torch()
        return torch.empty(shape, dtype=torch.float64, device=ref.device)
    return np.empty(shape, dtype=dtype)


def _check(ctx, st):
    if st != OK:
        raise ElmError(st, _lib.load().elm_last_error(ctx.handle).decode())


class Context:
    """Owns an elm_ctx (device workspace, stream)."""

    def __init__(self, device: int = 0, stream=None):
        self.handle = C.c_void_p()
        self.device = device
        st = _lib.load().elm_create(C.byref(self.handle), device, _stream_ptr(stream))
        if st != OK:
            raise ElmError(st, "elm_create")

    def set_stream(self, stream):
        _lib.load().elm_set_stream(self.handle, _stream_ptr(stream))

    def close(self):
        if self.handle:
            _lib.load().elm_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def elm_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def elm_destroy(ctx: Context):
    ctx.close()


def _is_f64(x):
    return str(x.dtype).endswith("float64")


def _check_hidden_args(X, W, b, a, Ht):
    """Shapes and element types the C ABI takes on trust (it reads L
    doubles of b and a and writes L x N doubles of Ht)."""
    N, n = X.shape
    if W.ndim != 2 or W.shape[0] != n:
        raise ValueError("W must be n x L with n = X.shape[1]")
    L = W.shape[1]
    for name, v in (("W", W), ("b", b), ("a", a), ("Ht", Ht)):
        if v is not None and not _is_f64(v):
            raise ValueError("%s must be float64" % name)
    if tuple(b.shape) != (L,):
        raise ValueError("b must have shape (L,)")
    if a is not None and tuple(a.shape) != (L,):
        raise ValueError("a must have shape (L,)")
    if Ht is not None and tuple(Ht.shape) != (L, N):
        raise ValueError("Ht must have shape (L, N)")
    return N, n, L


def elm_hidden(ctx, X, W, b, a=None, act=ACT_SIGMOID, precision=PREC_FP64, Ht=None):
    """Ht (L x N) = a * g(X W + b), transposed (Eq. 1, Eq. 3)."""
    N, n, L = _check_hidden_args(X, W, b, a, Ht)
    if Ht is None:
        Ht = _empty_like_device(X, (L, N))
    st = _lib.load().elm_hidden(ctx.handle, _ptr(X), _xdtype(X), N, n, _ld(X), _ptr(W), _ld(W),
                                _ptr(b), _ptr(a), L, act, precision, _ptr(Ht), _ld(Ht))
    _check(ctx, st)
    return Ht


def elm_pinv_rank(ctx, Ht, tol_rank=0.0, perm=None, pinv=None, want_pinv=False):
    """Rank r, pivot order and optionally H^+ of H given as Ht (L x N)."""
    L, N = Ht.shape
    if perm is None:
        perm = np.empty(L, dtype=np.int32)
    if want_pinv and pinv is None:
        pinv = _empty_like_device(Ht, (L, N))
    r = C.c_int64(0)
    st = _lib.load().elm_pinv_rank(ctx.handle, _ptr(Ht), L, N, _ld(Ht), tol_rank, C.byref(r),
                                   _ptr(perm), _ptr(pinv), _ld(pinv) if pinv is not None else 0)
    _check(ctx, st)
    return int(r.value), perm, pinv


def _problem(p):
    X, W, b, T = p["X"], p["W"], p["b"], p["T"]
    a = p.get("a")
    N, n = X.shape
    L = W.shape[1]
    m = T.shape[1]
    beta = p.get("beta")
    if beta is None:
        beta = _empty_like_device(X, (L, m))
        p["beta"] = beta
    return elm_problem_struct(X, n, N, W, b, a, L, T, m, beta, p.get("act", ACT_SIGMOID))


def elm_problem_struct(X, n, N, W, b, a, L, T, m, beta, act):
    return _lib.elm_problem(X=_ptr(X), x_dtype=_xdtype(X), act=act, N=N, n=n, ldx=_ld(X),
                            W=_ptr(W), ldw=_ld(W), b=_ptr(b), a=_ptr(a), L=L, T=_ptr(T), m=m,
                            ldt=_ld(T), beta=_ptr(beta), ldb=_ld(beta))


def elm_train(ctx, problems, precision=PREC_FP64, max_refine=-1, tol_rank=0.0,
              refine_tol=0.0, check=True, flags=0, wait_limit_ns=0, block_split=0, lanes=0):
    """Train each problem (dict with X, W, b, a, act, T and optional beta
    output).  Returns a list of dicts (rank, refine_iters, status,
    rel_update, form: FORM_*); beta is written into problem['beta'].
    check: raise ElmError when the call returns a status other than OK.
    lanes: batched mixed trainings, problems whose back halves run at once
    (0: the library's default)."""
    if isinstance(problems, dict):
        problems = [problems]
    arr = (_lib.elm_problem * len(problems))(*[_problem(p) for p in problems])
    opts = _lib.elm_train_opts(precision=precision, max_refine=max_refine, tol_rank=tol_rank,
                               refine_tol=refine_tol, flags=flags, wait_limit_ns=wait_limit_ns,
                               block_split=block_split, lanes=lanes)
    res = (_lib.elm_result * len(problems))()
    st = _lib.load().elm_train(ctx.handle, arr, len(problems), C.byref(opts), res)
    if check:
        _check(ctx, st)
    return [dict(rank=r.rank, refine_iters=r.refine_iters, status=r.status,
                 rel_update=r.rel_update, form=r.form) for r in res]


def elm_autotune(ctx, problems, precision=PREC_FP64, path=None, max_refine=-1):
    """Time launch choices on these problems (trains them; beta is written)
    and keep the fastest for their shape bucket in the context, and in the
    cache file `path` if given.  Returns the choice as a dict."""
    if isinstance(problems, dict):
        problems = [problems]
    arr = (_lib.elm_problem * len(problems))(*[_problem(p) for p in problems])
    opts = _lib.elm_train_opts(precision=precision, max_refine=max_refine)
    out = _lib.elm_tune_choice()
    st = _lib.load().elm_autotune(ctx.handle, arr, len(problems), C.byref(opts),
                                  None if path is None else os.fsencode(path), C.byref(out))
    _check(ctx, st)
    return dict(panel_cluster=out.panel_cluster, panel_width=out.panel_width,
                hidden_stages=out.hidden_stages, gram_stages=out.gram_stages, lanes=out.lanes,
                best_ms=out.best_ms)


def elm_autotune_load(ctx, path):
    """Read an autotune cache file into the context."""
    _check(ctx, _lib.load().elm_autotune_load(ctx.handle, os.fsencode(path)))


FORM_FP64, FORM_MIXED, FORM_MIXED_TO_FP64, FORM_WIDE, FORM_BLOCK, FORM_FP64_TC = 0, 1, 2, 3, 4, 5


FLAG_PHASE_TIMING = 1
NOALLOC_SCRATCH_BYTES = 32 << 20


def elm_hidden_noalloc(X, W, b, a=None, act=ACT_SIGMOID, Ht=None, stream=None):
    """elm_hidden (mixed precision) without any device allocation by the
    library: scratch comes from a fixed device array inside libelm.so.  All
    arrays must be CUDA tensors of one device, which the call makes current;
    Ht is allocated here (by torch) when not given."""
    N, n, L = _check_hidden_args(X, W, b, a, Ht)
    torch = _torch()
    with torch.cuda.device(X.device):
        if Ht is None:
            Ht = _empty_like_device(X, (L, N))
        st = _lib.load().elm_hidden_noalloc(_ptr(X), _xdtype(X), N, n, _ld(X), _ptr(W), _ld(W),
                                            _ptr(b), _ptr(a), L, act, _ptr(Ht), _ld(Ht),
                                            _stream_ptr(stream))
    if st != OK:
        raise ElmError(st, "elm_hidden_noalloc")
    return Ht


def elm_hidden_noalloc_bytes(N, n, L):
    v = C.c_int64(0)
    st = _lib.load().elm_hidden_noalloc_bytes(N, n, L, C.byref(v))
    if st != OK:
        raise ElmError(st, "elm_hidden_noalloc_bytes")
    return int(v.value)


def elm_phase_times(ctx):
    """{phase name: ms} summed since the previous call (then reset)."""
    lib = _lib.load()
    buf = (C.c_double * 8)()
    n = lib.elm_phase_times(ctx.handle, buf, 8)
    if n < 0:
        raise ElmError(-n, "elm_phase_times")
    return {lib.elm_phase_name(i).decode(): buf[i] for i in range(n)}


def elm_phase_name(i):
    return _lib.load().elm_phase_name(i).decode()


def elm_launch_counter():
    return int(_lib.load().elm_launch_counter())


def elm_predict(ctx, X, W, b, a, act, beta, Y=None):
    """Y (N x m) = g(X W + b) beta (Section 2, step 3)."""
    N, n = X.shape
    L = W.shape[1]
    m = beta.shape[1]
    if Y is None:
        Y = _empty_like_device(X, (N, m))
    st = _lib.load().elm_predict(ctx.handle, _ptr(X), _xdtype(X), N, n, _ld(X), _ptr(W), _ld(W),
                                 _ptr(b), _ptr(a), L, act, _ptr(beta), m, _ld(beta), _ptr(Y),
                                 _ld(Y))
    _check(ctx, st)
    return Y


class RowBlock:
    """One row block of a problem (elm_rows_*): its hidden layer stays on the
    device; gram() gives the block's H^T H and H^T T, residual(beta) its
    H^T (T - H beta)."""

    def __init__(self, ctx, X, W, b, a, act, T, precision=PREC_MIXED):
        N, n = X.shape
        L = W.shape[1]
        m = T.shape[1]
        self.ctx, self.L, self.m, self.ref = ctx, L, m, X
        self.handle = C.c_void_p()
        st = _lib.load().elm_rows_create(ctx.handle, _ptr(X), _xdtype(X), N, n, _ld(X), _ptr(W),
                                         _ld(W), _ptr(b), _ptr(a), L, act, _ptr(T), m, _ld(T),
                                         precision, C.byref(self.handle))
        _check(ctx, st)

    def gram(self):
        S = _empty_like_device(self.ref, (self.L, self.L))
        Z = _empty_like_device(self.ref, (self.L, self.m))
        _check(self.ctx, _lib.load().elm_rows_gram(self.handle, _ptr(S), _ld(S), _ptr(Z), _ld(Z)))
        return S, Z

    def residual(self, beta):
        G = _empty_like_device(self.ref, (self.L, self.m))
        _check(self.ctx, _lib.load().elm_rows_residual(self.handle, _ptr(beta), _ld(beta),
                                                       _ptr(G), _ld(G)))
        return G

    def close(self):
        if self.handle:
            _lib.load().elm_rows_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GramFactor:
    """The pivoted factorisation of a (summed) Gram matrix (elm_factor_*);
    solve(Z) applies the full-rank route to Z (L x mc)."""

    def __init__(self, ctx, S, m, precision=PREC_MIXED, tol_rank=0.0):
        L = S.shape[0]
        self.ctx, self.L, self.ref = ctx, L, S
        self.handle = C.c_void_p()
        r = C.c_int64(0)
        st = _lib.load().elm_factor_gram(ctx.handle, _ptr(S), _ld(S), L, m, precision, tol_rank,
                                         C.byref(self.handle), C.byref(r))
        _check(ctx, st)
        self.rank = int(r.value)

    def solve(self, Z):
        out = _empty_like_device(self.ref, (self.L, Z.shape[1]))
        _check(self.ctx, _lib.load().elm_factor_solve(self.handle, _ptr(Z), _ld(Z), Z.shape[1],
                                                      _ptr(out), _ld(out)))
        return out

    def close(self):
        if self.handle:
            _lib.load().elm_factor_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
