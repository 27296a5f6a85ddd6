"""Helpers shared by the GPU parity tests (host-side marshalling only)."""
import numpy as np
import torch

FP64_TOL = 1e-11   # relative 2-norm bar for float64 deterministic maps


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel2(a, b):
    """Relative 2-norm error ||a - b|| / ||b|| (whole field)."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def maxrel(a, b):
    """Element-wise error max |a - b| / max |b|: one wrong face or block of a
    large field shows here even where the 2-norm averages it away."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    mb = np.abs(b).max()
    return float(np.abs(a - b).max() / (mb if mb > 0 else 1.0))


def rel(a, b):
    """The parity tests' error measure: the larger of the relative 2-norm and
    the element-wise max |a - b| / max |b|, so that every bound written
    against it holds element by element as well as in norm."""
    return max(rel2(a, b), maxrel(a, b))


def owned_slices(b):
    """Slices of an oracle box's owned block in a [3][nz][ny][nx] field."""
    (x0, y0, z0), (x1, y1, z1) = b.own_lo, b.own_hi
    return (slice(None), slice(z0, z1), slice(y0, y1), slice(x0, x1))


def box_rel2(z, ref, boxes):
    """Largest relative 2-norm error over the boxes' owned blocks."""
    return max(rel2(z[owned_slices(b)], ref[owned_slices(b)]) for b in boxes)


def context(w, **kw):
    from paper_2508_07193_b300 import flashmp as F
    return F.Context(w.grid, w.eps_cell, w.beta, w.cuts, w.overlap, **kw)
