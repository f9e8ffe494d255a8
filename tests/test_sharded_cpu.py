"""Row-sharded training on CPU ranks (gloo, world size 2): the orchestration
of paper_2011_02436_gb300.sharded (blocks summed in block order within a
process, then over ranks in rank order by one exchange; one factorisation
per rank of the same summed Gram; refinement residuals summed the same way)
driven by the FP64 oracle in place of the library's kernels.  Checks: both
ranks hold bitwise the same beta and rank; rank and beta agree with the
oracle's single-process training of the whole problem."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


class OracleOps:
    """The oracle's routines behind the two methods the orchestration uses."""

    def block(self, X, W, b, a, act, T):
        import oracle

        class Blk:
            def __init__(self):
                self.H = oracle.hidden(X, W, b, a, act)
                self.T = np.ascontiguousarray(T, dtype=np.float64)

            def gram(self):
                return oracle.gram(self.H, self.T)

            def residual(self, beta):
                return oracle.gram(self.H, self.T - oracle.matmul_hb(self.H, beta))[1]
        return Blk()

    def factor(self, S, m):
        import oracle

        class Fac:
            def __init__(self):
                self.rank, self.perm, self.R = oracle.pivchol(S)

            def solve(self, Z):
                return oracle.frsolve(self.R, self.rank, self.perm, Z)
        return Fac()


def _problem():
    import synth
    return synth.make_problem(1500, 9, 70, 3, n_dup=6, n_scaled=4, x_dtype=np.float64,
                              x_kind="uniform11", act=synth.ACT_TANH)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2011_02436_gb300 import PREC_FP64
    from paper_2011_02436_gb300.sharded import train_row_blocks
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        p = _problem()
        # this rank's rows, as two blocks of unequal size
        rows = np.array_split(np.arange(p["N"]), 2 * world)[2 * rank:2 * rank + 2]
        blocks = [(p["X"][r], p["W"], p["b"], p["a"], p["act"], p["T"][r]) for r in rows]
        beta, r, info = train_row_blocks(OracleOps(), blocks, precision=PREC_FP64)
        out[rank] = (beta.tobytes(), r, info["refine_iters"])
    finally:
        dist.destroy_process_group()


def test_row_sharded_training_world2_matches_single_process_oracle():
    import oracle
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] and res[0][1] == res[1][1]     # the same bits on both ranks
    p = _problem()
    ref, r, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    beta = np.frombuffer(res[0][0]).reshape(ref.shape)
    assert res[0][1] == r == p["rank"]
    assert np.linalg.norm(beta - ref) / np.linalg.norm(ref) <= 1e-10


def test_one_process_with_blocks_equals_the_unsplit_sums():
    """Without a process group the blocks are only summed locally; split
    sums differ from the unsplit ones by rounding alone."""
    import oracle
    from paper_2011_02436_gb300 import PREC_FP64
    from paper_2011_02436_gb300.sharded import train_row_blocks
    p = _problem()
    rows = np.array_split(np.arange(p["N"]), 3)
    blocks = [(p["X"][r], p["W"], p["b"], p["a"], p["act"], p["T"][r]) for r in rows]
    beta, r, info = train_row_blocks(OracleOps(), blocks, precision=PREC_FP64)
    ref, r0, _ = oracle.train(p["X"], p["W"], p["b"], p["a"], p["act"], p["T"])
    assert r == r0 and info["converged"]
    assert np.linalg.norm(beta - ref) / np.linalg.norm(ref) <= 1e-10
