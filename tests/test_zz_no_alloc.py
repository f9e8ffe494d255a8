"""elm_hidden_noalloc: the hidden layer for callers that may not allocate
device memory (a plugin inside a framework that owns all device memory, a
service that forbids allocator calls after start-up).  Its scratch is a
fixed device array inside the library; its output must equal elm_hidden's
mixed-precision output, on consecutive calls that reuse the array."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def elm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_02436_gb300 as m
    return m


def test_noalloc_rejects_problems_beyond_the_array(elm):
    need = elm.elm_hidden_noalloc_bytes(100000, 784, 4000)
    assert need > elm.NOALLOC_SCRATCH_BYTES
    assert elm.elm_hidden_noalloc_bytes(500, 20, 90) < elm.NOALLOC_SCRATCH_BYTES


@pytest.mark.gpu
def test_noalloc_matches_elm_hidden_on_consecutive_calls(elm):
    import torch
    stream = torch.cuda.current_stream()
    ctx = elm.elm_create(0, stream)
    cases = [synth.make_problem(1500, 40, 200, 2, n_dup=10, x_kind="normal"),
             synth.make_problem(777, 13, 65, 2, n_dup=5, n_scaled=4, act=synth.ACT_TANH,
                                x_dtype=np.float64, x_kind="uniform11")]
    for p in cases:                                       # two calls in a row
        t = {k: (None if p[k] is None else torch.from_numpy(np.ascontiguousarray(p[k])).cuda())
             for k in ("X", "W", "b", "a")}
        ref = elm.elm_hidden(ctx, t["X"], t["W"], t["b"], t["a"], p["act"],
                             precision=elm.PREC_MIXED)
        got = elm.elm_hidden_noalloc(t["X"], t["W"], t["b"], t["a"], p["act"], stream=stream)
        torch.cuda.synchronize()
        assert got.shape == ref.shape
        assert float((got - ref).abs().max()) <= 1e-12
    big = synth.make_problem(20000, 784, 100, 2)
    X = torch.from_numpy(big["X"]).cuda()
    with pytest.raises(elm.ElmError) as e:                # beyond the array: rejected
        elm.elm_hidden_noalloc(X, torch.from_numpy(big["W"]).cuda(),
                               torch.from_numpy(big["b"]).cuda(), None, 0, stream=stream)
    assert e.value.status == 7
    ctx.close()
