"""Shared helpers for the GPU parity tests (build once, move arrays, normwise errors)."""
import numpy as np

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-5, "f16": 5e-3, "bf16": 5e-3}


def built():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2411_08461_gb300 as pkg

    return pkg


def cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b) -> float:
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
