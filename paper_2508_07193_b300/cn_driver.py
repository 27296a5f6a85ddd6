"""Crank-Nicolson FDTD time stepping with a dipole source: the plain
preconditioned solver against the learned initial guess / correction.

    python -m paper_2508_07193_b300.cn_driver --grid 256 --steps 200 --train-until 50

Phases (all on the GPU through the C ABI):
1. steps [0, train_until): plain steps; each records the training pair
   (r0 = R - A E^n, e = E^{n+1} - E^n), R the step's right-hand side;
2. Adam training of the CNN on random crops of those pairs;
3. steps [train_until, steps): run twice from the same saved state, once with
   the plain solver (x0 = E^n) and once with the learned component
   (use_learned = 1: learned initial guess; 2: also the in-FGMRES correction),
   recording iterations and time per step.

A checkpoint (E, H, step, CNN parameters, phase) can be written with
--checkpoint and resumed with --resume.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import flashmp as F
from . import workloads as wl


def dipole_workload(n, seed=4, beta=0.25):
    """n^3 grid, 16 eps boxes from the seed, 8^3 (or n/32) subdomains, overlap
    2; beta = (dt / 2)^2 in grid units (0.25: dt = 1)."""
    parts = max(2, n // 32)
    return wl.make_workload(f"dipole{n}", (n, n, n), seed=seed, n_eps_boxes=16,
                            cuts=[wl.even_cuts(n, parts)] * 3, overlap=2, beta=beta)


def current(w, step, dt, dev):
    J = wl.dipole_current(w.grid, step, dt)
    return torch.as_tensor(J, device=dev)


def plain_step_with_pair(ctx, E, H, J, dt, record=True, E_prev=None, ext_pairs=None):
    """One CN step from the ABI pieces (updates E, H). With record, the pair
    (R - A E^n, E^(n+1) - E^n) goes to the library's sample pool; with
    ext_pairs, the pair of the extrapolated guess G = 2 E^n - E^(n-1),
    (R - A G, E^(n+1) - G), is appended to that list."""
    R = ctx.cn_rhs(E, H, J, dt)
    r0 = ctx.curlcurl_apply(E, c_eps=-1.0, c_k=-ctx.beta)
    r0 += R
    G = None
    if ext_pairs is not None:
        G = 2.0 * E - E_prev
        rg = ctx.curlcurl_apply(G, c_eps=-1.0, c_k=-ctx.beta)
        rg += R
    E_old = E.clone()
    x, info = ctx.krylov_solve(R, E)
    ctx.h_update(H, E, E_old, dt)
    if record:
        ctx.cnn_add_sample(r0, (E - E_old).contiguous())
    if ext_pairs is not None:
        ext_pairs.append((rg, (E - G).contiguous()))
    return info


def save(path, **state):
    torch.save({k: (v.cpu() if isinstance(v, torch.Tensor) else v) for k, v in state.items()}, path)


def run(args):
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = dipole_workload(args.grid, beta=getattr(args, "beta", 0.25))
    dt = 2.0 * math.sqrt(w.beta)
    ctx = F.Context(w.grid, w.eps_cell, w.beta, w.cuts, w.overlap, precision=args.precision,
                    rtol=args.rtol, restart=30)
    E = ctx.empty_field()
    H = ctx.empty_field()
    step0 = 0
    if args.resume:
        ck = torch.load(args.resume, weights_only=False)
        E.copy_(ck["E"].to(dev)); H.copy_(ck["H"].to(dev))
        step0 = int(ck["step"])
        if ck.get("params") is not None:
            ctx.cnn_set_params(ck["params"])
    log = {"grid": list(w.grid), "beta": w.beta, "precision": args.precision, "rtol": args.rtol, "phase1": [], "plain": [],
           "learned": [], "learned_mode": args.learned_mode}
    # phase 1: plain steps with recorded pairs (E_prev: the field one step back)
    t0 = time.time()
    E_prev = E.clone()
    if args.resume and ck.get("E_prev") is not None:
        E_prev.copy_(ck["E_prev"].to(dev))
    extrapolate = getattr(args, "extrapolate", False)
    ext_pairs = [] if extrapolate else None
    for n in range(step0, min(args.train_until, args.steps)):
        cur = E.clone()
        info = plain_step_with_pair(ctx, E, H, current(w, n, dt, dev), dt, record=True, E_prev=E_prev,
                                    ext_pairs=ext_pairs if n > step0 else None)
        E_prev.copy_(cur)
        log["phase1"].append({"step": n, "iters": info["iters"], "ms": info["ms_total"]})
    torch.cuda.synchronize()
    log["phase1_s"] = time.time() - t0
    if args.checkpoint:
        save(args.checkpoint, E=E, H=H, E_prev=E_prev, step=max(step0, args.train_until), params=ctx.cnn_get_params())
    # phase 2: training (with --extrapolate, a second network from the same
    # initial parameters on the extrapolated guess's pairs)
    t0 = time.time()
    params0 = ctx.cnn_get_params()
    if ctx.cnn_num_samples() > 0 and args.train_iters > 0:
        log["train_loss"] = ctx.cnn_train(args.train_iters, args.crop, lr=args.lr, seed=args.seed)
    params_plain = ctx.cnn_get_params()
    ctx.cnn_clear_samples()
    params_ext = params_plain
    if ext_pairs:
        ctx.cnn_set_params(params0)
        for r0, e in ext_pairs:
            ctx.cnn_add_sample(r0, e)
        if args.train_iters > 0:
            log["train_loss_extrap"] = ctx.cnn_train(args.train_iters, args.crop, lr=args.lr, seed=args.seed)
        params_ext = ctx.cnn_get_params()
        ctx.cnn_clear_samples()
        ext_pairs.clear()
    torch.cuda.synchronize()
    log["train_s"] = time.time() - t0
    # phase 3: the same steps from the same state, once per initial guess:
    # E^n (plain), N on top of E^n (learned); with --extrapolate also
    # 2 E^n - E^(n-1) and N on top of that
    E0, H0, P0 = E.clone(), H.clone(), E_prev.clone()
    runs = [(0, False, "plain"), (args.learned_mode, False, "learned")]
    if extrapolate:
        runs += [(0, True, "extrap"), (args.learned_mode, True, "learned_extrap")]
        log.update({"extrap": [], "learned_extrap": []})
    for mode, extrap, key in runs:
        E.copy_(E0); H.copy_(H0); E_prev.copy_(P0)
        ctx.cnn_set_params(params_ext if extrap else params_plain)
        ctx.set_options(use_learned=mode, experimental=mode >= 2)
        torch.cuda.synchronize()
        t0 = time.time()
        for n in range(max(step0, args.train_until), args.steps):
            if extrap:
                E_cur = E.clone()
                info = ctx.cn_step(E, H, current(w, n, dt, dev), dt, E_prev=E_prev)
                E_prev.copy_(E_cur)
            else:
                info = ctx.cn_step(E, H, current(w, n, dt, dev), dt)
            log[key].append({"step": n, "iters": info["iters"], "ms": info["ms_total"],
                             "fallback": info["used_fallback"], "res": info["true_rel_res"]})
        torch.cuda.synchronize()
        log[key + "_s"] = time.time() - t0
        log[key + "_iters"] = int(sum(r["iters"] for r in log[key]))
        log[key + "_max_res"] = max((r["res"] for r in log[key]), default=0.0)
    log["energy_E"] = float((E * E).sum().item())
    ctx.close()
    return log


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--grid", type=int, default=256)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--train-until", type=int, default=50)
    p.add_argument("--train-iters", type=int, default=600)
    p.add_argument("--crop", type=int, default=32)
    p.add_argument("--lr", type=float, default=2e-3)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--precision", default="bf16")
    p.add_argument("--beta", type=float, default=0.25,
                   help="(dt / 2)^2 in grid units; the time step is dt = 2 sqrt(beta)")
    p.add_argument("--rtol", type=float, default=1e-8)
    p.add_argument("--learned-mode", type=int, default=1)
    p.add_argument("--extrapolate", action="store_true",
                   help="also run the steps from the extrapolated guess 2 E^n - E^(n-1), plain and learned")
    p.add_argument("--checkpoint", default=None)
    p.add_argument("--resume", default=None)
    p.add_argument("--out", default=None)
    args = p.parse_args()
    log = run(args)
    summary = {k: v for k, v in log.items() if not isinstance(v, list)}
    print(json.dumps(summary))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(log, f)


if __name__ == "__main__":
    main()
