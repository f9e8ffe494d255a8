"""Shared helpers for the GPU tests (inputs from synth, expectations from
the oracle)."""
import numpy as np


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(p, keys=("X", "W", "b", "a", "T")):
    import torch
    dev = torch.device("cuda:0")
    out = {}
    for k in keys:
        v = p.get(k)
        out[k] = None if v is None else torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    return out


def problem(p):
    t = to_dev(p)
    return dict(X=t["X"], W=t["W"], b=t["b"], a=t["a"], act=p["act"], T=t["T"])
