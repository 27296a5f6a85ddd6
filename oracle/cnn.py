"""Small 3-D CNN for the learned initial guess / coarse correction (oracle, test-only).

Not part of the paper: the network is the learned component of the build
(4 conv layers, 3x3x3 kernels, 16 hidden channels, ReLU between layers, a
linear last layer). Inputs and outputs are channel-major voxel arrays
[C][D][H][W]; a voxel (k, j, i) carries the three edge slots (c, k, j, i) of a
field as channels 0..2 and, for the input, the cell permittivity as channel 3.

Plain float64 NumPy: convolution as a sum over the 27 taps of shifted slices
(zero padding), backward by the chain rule written out per layer, the loss as
the relative squared error, and Adam as published (Kingma & Ba 2015).
"""
from __future__ import annotations

import numpy as np

LAYERS = ((4, 16), (16, 16), (16, 16), (16, 3))
TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def init_params(seed=0, layers=LAYERS):
    """Kaiming-uniform weights W[co][ci][3][3][3] and zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for ci, co in layers:
        bound = np.sqrt(6.0 / (ci * 27))
        params.append((rng.uniform(-bound, bound, (co, ci, 3, 3, 3)), np.zeros(co)))
    return params


def shift(x, dz, dy, dx):
    """x shifted so that out[.., k, j, i] = x[.., k+dz, j+dy, i+dx] (zero outside)."""
    C, D, H, W = x.shape
    out = np.zeros_like(x)
    zs, ze = max(0, -dz), min(D, D - dz)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    out[:, zs:ze, ys:ye, xs:xe] = x[:, zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv3d(x, w, b):
    """y[o] = b[o] + sum_c sum_taps w[o, c, dz+1, dy+1, dx+1] x[c, k+dz, j+dy, i+dx]."""
    y = np.zeros((w.shape[0],) + x.shape[1:]) + b[:, None, None, None]
    for dz, dy, dx in TAPS:
        y += np.einsum("oc,cdhw->odhw", w[:, :, dz + 1, dy + 1, dx + 1], shift(x, dz, dy, dx))
    return y


def forward(params, x):
    """Returns (output, list of layer inputs) for backward."""
    acts = [x]
    h = x
    for li, (w, b) in enumerate(params):
        h = conv3d(h, w, b)
        if li < len(params) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h, acts


def conv3d_backward(x, w, dy):
    """Gradients of conv3d w.r.t. x, w and b for an upstream gradient dy."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for dz, dyy, dxx in TAPS:
        xs = shift(x, dz, dyy, dxx)
        dw[:, :, dz + 1, dyy + 1, dxx + 1] = np.einsum("odhw,cdhw->oc", dy, xs)
        # y[k] gets x[k+d] -> x[k] contributes to y[k-d]
        dx += np.einsum("oc,odhw->cdhw", w[:, :, dz + 1, dyy + 1, dxx + 1], shift(dy, -dz, -dyy, -dxx))
    db = dy.sum(axis=(1, 2, 3))
    return dx, dw, db


def loss(pred, target):
    """Relative squared error ||pred - target||^2 / ||target||^2."""
    return float(np.sum((pred - target) ** 2) / np.sum(target ** 2))


def backward(params, acts, target):
    """Loss and parameter gradients (list of (dw, db)) by the chain rule."""
    out = acts[-1]
    den = np.sum(target ** 2)
    g = 2.0 * (out - target) / den
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        w, _ = params[li]
        if li < len(params) - 1:
            g = g * (acts[li + 1] > 0.0)          # through the ReLU of layer li
        dx, dw, db = conv3d_backward(acts[li], w, g)
        grads[li] = (dw, db)
        g = dx
    return loss(out, target), grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015); state = dict(t, m, v)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    ms = state.setdefault("m", [(np.zeros_like(w), np.zeros_like(b)) for w, b in params])
    vs = state.setdefault("v", [(np.zeros_like(w), np.zeros_like(b)) for w, b in params])
    new = []
    for li, ((w, b), (dw, db)) in enumerate(zip(params, grads)):
        upd = []
        for q, (p, g) in enumerate(((w, dw), (b, db))):
            m = b1 * ms[li][q] + (1 - b1) * g
            v = b2 * vs[li][q] + (1 - b2) * g * g
            ms[li] = tuple(m if k == q else ms[li][k] for k in range(2))
            vs[li] = tuple(v if k == q else vs[li][k] for k in range(2))
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            upd.append(p - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(upd))
    return new
