"""Row-sharded training: the rows of H split into blocks, one or more per
process (one GPU each).  Every block forms its own H_p^T H_p and H_p^T T_p;
the blocks are summed, first within the process in block order, then over
the processes in rank order (one exchange: every rank receives the same
bits); every rank then factorises the same Gram matrix and so takes the same
rank decision; each refinement residual H^T (T - H beta) is summed the same
way.  This is the distributed setting the paper names as future work
(Section 5); the arithmetic is that of elm_train (Eqs. 5-13, Algorithm 1),
the sums over samples split by rows.

The exchange uses torch.distributed (NCCL on GPUs, gloo on CPUs); all the
arithmetic runs in the library (RowBlock, GramFactor) through `LibraryOps`.
Another object with the same two methods may stand in for it (the CPU tests
pass the FP64 oracle that way to check the reduction order and the rank
agreement on gloo ranks).
"""
from __future__ import annotations

import math

import numpy as np

from . import GramFactor, PREC_FP64, PREC_MIXED, RowBlock


class LibraryOps:
    """The library's row block and Gram factorisation on one context."""

    def __init__(self, ctx, precision=PREC_MIXED):
        self.ctx, self.precision = ctx, precision

    def block(self, X, W, b, a, act, T):
        return RowBlock(self.ctx, X, W, b, a, act, T, self.precision)

    def factor(self, S, m):
        return GramFactor(self.ctx, S, m, self.precision)

    def fp64(self):
        """The same operations in the FP64 form (the mixed form's hand-over)."""
        return LibraryOps(self.ctx, PREC_FP64)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def sum_over_ranks(x, group=None):
    """Sum of x over the ranks of `group`, rank 0's term first, then rank 1's
    and so on: an all-gather followed by a sum in rank order, so every rank
    holds bitwise the same result.  Without an initialised process group
    (or with one rank) x itself."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return x
    t = x if _is_torch(x) else torch.from_numpy(np.ascontiguousarray(x))
    t = t.contiguous()
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out if _is_torch(x) else out.numpy()


def _norm(x):
    return float(x.norm()) if _is_torch(x) else float(np.linalg.norm(x))


def train_row_blocks(ops, blocks, precision=PREC_MIXED, max_refine=None, refine_tol=None,
                     group=None, reduce=sum_over_ranks):
    """Train one problem whose rows are split into `blocks`: this process's
    blocks as (X, W, b, a, act, T) tuples, W, b, a and act the same in every
    block and on every rank.  Returns (beta, rank, info): beta (L x m) the
    same bits on every rank; info holds refine_iters, rel_update and
    converged.  Refinement as in elm_train: at most max_refine steps (2 for
    FP64, 12 for mixed), stopping once ||dbeta|| <= refine_tol ||beta||
    (1e-12 FP64, 1e-9 mixed) or, in the mixed form, once a step fails to
    halve the previous one.  As in elm_train, a mixed training whose rank
    decision the mixed Gram cannot settle, or whose refinement stops short,
    is done again in the FP64 form (info["handed_over"]); every rank takes
    the same decision, since it rests on the same summed values."""
    mixed = precision == PREC_MIXED
    if mixed and hasattr(ops, "fp64"):
        from . import ElmError
        try:
            out = _train(ops, blocks, PREC_MIXED, max_refine, refine_tol, group, reduce)
        except ElmError as e:
            if e.status != 4:            # only an unsettled rank decision is handed over
                raise
            out = None
        if out is not None and out[2]["converged"]:
            return out
        beta, rank, info = _train(ops.fp64(), blocks, PREC_FP64, None, None, group, reduce)
        info["handed_over"] = True
        return beta, rank, info
    return _train(ops, blocks, precision, max_refine, refine_tol, group, reduce)


def _train(ops, blocks, precision, max_refine, refine_tol, group, reduce):
    mixed = precision == PREC_MIXED
    if max_refine is None:
        max_refine = 12 if mixed else 2
    if refine_tol is None:
        refine_tol = 1e-9 if mixed else 1e-12
    blks = [ops.block(*blk) for blk in blocks]
    m = blocks[0][5].shape[1]

    def local_sum(xs):
        out = xs[0]
        for x in xs[1:]:
            out = out + x
        return out

    grams = [bk.gram() for bk in blks]
    S = reduce(local_sum([g[0] for g in grams]), group)
    Z = reduce(local_sum([g[1] for g in grams]), group)
    fac = ops.factor(S, m)
    beta = fac.solve(Z)
    info = dict(refine_iters=0, rel_update=0.0, converged=max_refine == 0, handed_over=False)
    prev = math.inf
    for it in range(max_refine):
        G = reduce(local_sum([bk.residual(beta) for bk in blks]), group)
        d = fac.solve(G)
        beta = beta + d
        nb = _norm(beta)
        rel = _norm(d) / nb if nb > 0 else 0.0
        info.update(refine_iters=it + 1, rel_update=rel)
        if rel <= refine_tol:
            info["converged"] = True
            break
        if mixed and it >= 1 and not rel < 0.5 * prev:
            break
        prev = rel
    for bk in blks:
        if hasattr(bk, "close"):
            bk.close()
    rank = fac.rank
    if hasattr(fac, "close"):
        fac.close()
    return beta, rank, info
