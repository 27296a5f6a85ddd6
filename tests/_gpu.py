"""Helpers shared by the GPU parity tests (host-side marshalling only)."""
import numpy as np
import torch

FP64_TOL = 1e-11   # relative 2-norm bar for float64 deterministic maps


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def context(w, **kw):
    from paper_2508_07193_b300 import flashmp as F
    return F.Context(w.grid, w.eps_cell, w.beta, w.cuts, w.overlap, **kw)
