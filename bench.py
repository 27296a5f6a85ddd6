"""Benchmark: one Crank-Nicolson FDTD step on the 256^3 Yee workload.

Workload (seeded, synthetic): 256^3 cells with PEC walls (50.3 M unknowns),
eps_r piecewise constant over 16 random boxes in [1, 10], beta = 0.25,
restricted additive Schwarz over 8x8x8 subdomains of 32^3 with overlap 2
(extended extents 34/36), restarted FGMRES(30) to a 1e-8 true relative
residual, float64 transforms (the plain FP64 form); the same step with the
preconditioner's transforms in the other precisions is timed beside it
(`forms`), each with its measured preconditioner error against float64.
`--workload grid128` runs the 128^3 workload (4x4x4 subdomains),
`--workload uneven` the 320x256x192 uneven one, and `--case box` times the
exact solve of the single 32^3 PEC box.
A step is one fmp_cn_step from E = H = 0 with the impressed current
J = -b/dt, so that its right-hand side is the seeded uniform field b:
right-hand-side stencil, the preconditioned Krylov solve (transform box
solves, SpMV, CGS2 orthogonalisation) and the H update.

Metric: DoF/s = 3 N^3 / step time (the paper's MDoF/s convention), whole job
(all ranks). Multi-GPU runs are independent replicas (weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CN-FDTD step time to 1e-8 residual; subdomain DoF/s vs plain FP64 form"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25   # B300 float64 (vector and tensor) nominal
# float64 pipe issue rate: 2 lane-operations (an FMA or an add each) per clock
# per SM (1.25 TFLOP/s nominal / 2 flops per FMA / 148 SMs ~ 2.1 GHz x 2)
FP64_OPS_PER_CLK_SM = 2
N_SMS = 148
SM_MAX_MHZ = 2032.0


def fp64_issue_peak_tops(sm_mhz=None):
    """Float64 operations per second the float64 pipes of all SMs issue at
    `sm_mhz` (default the maximum SM clock), in units of 1e12."""
    return FP64_OPS_PER_CLK_SM * N_SMS * (sm_mhz or SM_MAX_MHZ) * 1e6 / 1e12

# dram__bytes_read.sum + dram__bytes_write.sum of one preconditioner apply
# (all of its kernels) from an ncu capture of the current kernels, per
# (workload, precision); the capture is summarised in the profiles/ file named
# beside each entry. Absent: not captured for this kernel version.
TRAFFIC_BYTES = {
    ("yee256_ras8x8x8_ol2", "fp64"): 2965.6e6,   # transform_fp64_precond_grid256.md
    ("yee256_ras8x8x8_ol2", "bf16"): 748.3e6,    # fused_bf16_precond_grid256.md
    ("yee128_ras4x4x4_ol2", "fp64_ozaki"): 246.8e6,   # transform_fp64_ozaki_precond_grid128.md
}

WORKLOADS = ("grid128", "grid256", "uneven", "box32")


def workload(name):
    from paper_2508_07193_b300 import workloads as wl
    return {"grid128": wl.grid128, "grid256": wl.grid256, "uneven": wl.grid_uneven, "box32": wl.box32}[name]()


def bench_config(w, args):
    """The `config` object of both arms' JSON lines (same keys and values)."""
    l2 = (f"inputs exceed L2 across a step ({8 * w.n_slots / 1e6:.0f} MB per field, "
          f"{61 * 8 * w.n_slots / 1e9:.1f} GB Krylov basis)")
    return {"workload": w.name, "grid": list(w.grid), "subdomains": [len(c) for c in w.cuts],
            "overlap": w.overlap, "beta": w.beta,
            "krylov": "FGMRES(30)" if args.krylov == "fgmres" else "BiCGSTAB",
            "cuda_graph": bool(args.graph), "rtol": 1e-8, "precision": args.precision, "form": args.form,
            "l2": l2}


# one network evaluation, per voxel: 2 x 27 taps x C_in x C_out for the layers
# 4 -> 16, 16 -> 16, 16 -> 16, 16 -> 3
CNN_FLOPS_PER_VOXEL = 2 * 27 * (4 * 16 + 16 * 16 + 16 * 16 + 16 * 3)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp64")
    p.add_argument("--krylov", default="fgmres", choices=["fgmres", "bicgstab"])
    p.add_argument("--no-graph", dest="graph", action="store_false",
                   help="enqueue each Arnoldi step instead of replaying the restart cycle as one CUDA graph")
    p.add_argument("--autotune", action="store_true", help="autotune the reduced-precision work lists first")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip timing the other preconditioner precisions")
    p.add_argument("--form", default="yee", choices=["yee", "compact"],
                   help="subdomain form: Yee boxes with PEC walls, or the compact layout with the Woodbury "
                        "boundary correction (float64 only)")
    p.add_argument("--case", default="step", choices=["step", "precond", "spmv", "cnn", "box"],
                   help="precond/spmv/cnn: only W + K applies of that operator (for profiler captures), "
                        "the K timed with CUDA events; box: the exact solve of the 32^3 PEC box")
    p.add_argument("--workload", default="grid256", choices=["grid128", "grid256", "uneven", "box32"])
    p.add_argument("--fused", type=int, default=None,
                   help="bf16/fp16: largest extent of the fused cluster kernel (0: none; default 40, or 0 when "
                        "the boxes it could take are too few to fill the GPU beside larger ones)")
    p.add_argument("--streamed", type=int, default=None,
                   help="bf16/fp16 boxes outside the fused list: 1 one persistent streamed launch (default), "
                        "0 the three-pass kernels")
    p.add_argument("--orth", default=None, choices=["fixed", "float64", "split"],
                   help="Gram-Schmidt arithmetic of FGMRES: split (default: exact fixed-point products for the "
                        "oldest vectors of each pass, float64 FMAs for the rest), float64 FMAs, or exact fixed point")
    p.add_argument("--cnn-mma-sync", action="store_true",
                   help="--case cnn: the mma.sync convolution kernels instead of tcgen05")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


OZAKI_MAX_EXTENT = 80   # largest box extent of the digit-split float64 kernels


def max_over_ranks(value, world, device="cpu"):
    """The largest `value` over the ranks of the default process group (the
    value itself for one rank): the timing rule takes the slowest rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(dof, world, ms):
    """Whole-job throughput of `world` weak-scaled replicas: world x dof
    unknowns per step over the slowest rank's step time (ms)."""
    return world * dof / (ms * 1e-3)


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()

    def summary(self):
        rows = []
        try:
            for line in open(self.f.name):
                parts = [s.strip() for s in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.f.name)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def transform_flops(ctx):
    """Algorithmic flops of one preconditioner apply: per box, forward and
    inverse transforms of 3 components along 3 axes, 2 m_a flops per output
    (12 (mx+my+mz) mx my mz), plus 20 flops per mode for the 3x3 solve."""
    tot = 0
    for i in range(ctx.num_boxes()):
        mx, my, mz = ctx.box(i)["m"]
        tot += 12 * (mx + my + mz) * mx * my * mz + 20 * mx * my * mz
    return tot


def transform_bytes(ctx):
    """Algorithmic HBM bytes of one preconditioner apply: read the extended
    box of every subdomain (3 float64 components) and write the owned cells
    (3 float64 components of the whole grid)."""
    tot = 0
    for i in range(ctx.num_boxes()):
        mx, my, mz = ctx.box(i)["m"]
        tot += 3 * mx * my * mz * 8
    nx, ny, nz = ctx.grid
    return tot + 3 * nx * ny * nz * 8


def _fold2(m, dst):
    """Class structure of the library's two-level fold (Fold3 without the
    third level): rows n, input lengths len per class, the first-level pairs
    and middle, and the second-level length L (0 when it does not apply)."""
    off = 1 if dst else 0
    npair, mid = (m - off) // 2, (m - off) & 1
    s0 = 1 if dst else 0
    nks, nka = (m - s0 + 1) // 2, (m - (1 - s0) + 1) // 2
    la, lb = npair + mid, npair
    if m % 2 or m < 4:
        return dict(n=(nks, nka, 0), len=(la, lb, 0), npair=npair, mid=mid, L=0, off=off, m=m)
    if not dst:
        return dict(n=((nks + 1) // 2, nks // 2, nka), len=(la // 2 + la % 2, la // 2, lb), npair=npair, mid=mid,
                    L=la, off=off, m=m)
    return dict(n=(nka // 2, (nka - 1) // 2, nks), len=(lb // 2 + lb % 2, lb // 2, la), npair=npair, mid=mid, L=lb,
                off=off, m=m)


def _macs(f):
    return sum(n * ln for n, ln in zip(f["n"], f["len"]))


def _fold01_adds(f):
    """Additions that make the class-0 and class-1 inputs of a line (a class-0
    and a class-1 slot share their two second-level inputs)."""
    if not f["L"]:
        return f["len"][0] + f["len"][1] - f["mid"]
    L = f["L"]
    return 4 * (L // 2) + (L % 2)


def _items_ops(f, q0, g_of_q):
    """Inverse items of a line: class 0/1 products, output additions, and
    g_of_q(count) for the class-2 contributions of `count` slots."""
    n0, n1, n2 = f["n"]
    if not f["L"]:
        return (f["npair"] - q0) * (n0 + n1 + 2) + f["mid"] * n0
    L = f["L"]
    return (L // 2) * (n0 + n1 + 6 + g_of_q(2)) + (L % 2) * (n0 + 2 + g_of_q(1)) + f["mid"] * g_of_q(1)


def _inner_slot_terms(g):
    """Operations of the inner slots of g from weighted inputs (a product and
    an FMA per two-term sum; a class-0 / class-1 pair shares its two sums)."""
    if not g["L"]:
        return 2 * g["npair"] + g["mid"] + 2 * (g["len"][1])
    L = g["L"]
    return 6 * (L // 2) + 2 * (L % 2) + 2 * g["len"][2]


def _fwd_ops(m, dst):
    """Float64 operations of one forward line of the three-level fold."""
    f = _fold2(m, dst)
    if not f["L"]:
        return _macs(f) + _fold01_adds(f)
    g = _fold2(f["n"][2], False)
    N = f["n"][2]
    ops = f["n"][0] * f["len"][0] + f["n"][1] * f["len"][1] + _fold01_adds(f)
    if not dst:   # scaled differences, inner fold, inner rows, recurrence
        L2 = g["L"]
        inner_adds = (4 * (L2 // 2) + (L2 % 2) + g["len"][2]) if L2 else (N - g["mid"])
        return ops + 2 * N + inner_adds + _macs(g) + (N - 1)
    # reversed pair sums, then the inner inverse-direction items
    return ops + (N - 1) + _items_ops(g, 0, lambda cnt: cnt * g["n"][2])


def _inv_ops(m, dst, q0):
    """Float64 operations of one inverse line of the three-level fold."""
    f = _fold2(m, dst)
    if not f["L"]:
        return _items_ops(f, q0, lambda cnt: 0)
    g = _fold2(f["n"][2], False)
    N = f["n"][2]
    third = _inner_slot_terms(g) + _macs(g) + ((N - 1) if not dst else 0)
    return third + _items_ops(f, 0, lambda cnt: 0)


def transform_fp64_executed(ctx):
    """Float64 operations the three-level folded transform kernels execute
    per apply: per forward line the class-0/1 products and folds, and class
    2 through the inner DCT-II (scaled differences, inner fold, inner rows and
    the DCT-IV recurrence for DCT-II; pair sums and the inner
    inverse-direction items for DST-I); per inverse line the inner slots
    (chains of FMAs), the inner rows (and the recurrence) and the outer
    items; odd extents keep the two-level form (pairs whose two outputs lie
    outside the owned range skipped); about 11 operations per mode for the
    closed-form 3x3 with its tabulated denominator."""
    tot = 0
    for i in range(ctx.num_boxes()):
        bx = ctx.box(i)
        tot += _box_executed(bx["m"], bx["own_lo"], bx["ext_lo"], bx["own_n"])
    return tot


def _box_executed(m, own_lo, ext_lo, own_n):
    lo = [own_lo[a] - ext_lo[a] for a in range(3)]
    hi = [lo[a] + own_n[a] for a in range(3)]
    mx, my, mz = m

    def q0(ma, dst, a):
        f = _fold2(ma, dst)
        if f["L"]:
            return 0
        return max(0, min(f["npair"], min(lo[a] - f["off"], ma - hi[a])))

    tot = 0
    for c in range(3):
        sx, sy, sz = c != 0, c != 1, c != 2
        slabs = mz - (1 if c != 2 else 0)
        tot += slabs * (my * _fwd_ops(mx, sx) + mx * _fwd_ops(my, sy))                         # pass A
        tot += mx * my * (_fwd_ops(mz, sz) + _inv_ops(mz, sz, q0(mz, sz, 2)))                 # pass B
        own_z = hi[2] - lo[2]
        tot += own_z * (mx * _inv_ops(my, sy, q0(my, sy, 1)) + (hi[1] - lo[1]) * _inv_ops(mx, sx, q0(mx, sx, 0)))
    return tot + 9 * mx * my * mz   # the per-mode 3x3 (Eq. 12): nine float64 operations


def _rup(v, a):
    return (v + a - 1) // a * a


def ozaki_mma_flops(ctx):
    """bf16 tensor-core flops the digit-split float64 kernels execute per
    apply: every 16-line x 8-mode tile and 16-deep k-step runs the 21 digit-
    plane products (p + q <= 5), 21 * 2 * 16 * 8 * 16 flops; the tile counts
    follow the kernels (lines padded to 16, modes to 8, contraction to 16;
    inverse passes on the owned mode tiles only)."""
    per = 21 * 2 * 16 * 8 * 16
    tiles = 0
    for i in range(ctx.num_boxes()):
        bx = ctx.box(i)
        mx, my, mz = bx["m"]
        lo = [bx["own_lo"][a] - bx["ext_lo"][a] for a in range(3)]
        on = bx["own_n"]
        kx, ky, kz = _rup(mx, 16) // 16, _rup(my, 16) // 16, _rup(mz, 16) // 16
        # pass A: every z-slab, stage x (lines y) then stage y (lines kx)
        tiles += 3 * mz * (ky * (_rup(mx, 8) // 8) * kx + kx * (_rup(my, 8) // 8) * ky)
        # pass B: 16-column tiles, forward z on all modes, inverse z on the owned slabs
        ncolt = -(-(mx * my) // 16)
        nn = _rup(lo[2] + on[2], 8) // 8 - lo[2] // 8
        tiles += ncolt * 3 * ((_rup(mz, 8) // 8) + nn) * kz
        # pass C: owned z-slabs, inverse y (lines kx, owned y) then inverse x (owned lines y, owned x)
        nn1 = _rup(lo[1] + on[1], 8) // 8 - lo[1] // 8
        nn2 = _rup(lo[0] + on[0], 8) // 8 - lo[0] // 8
        tiles += 3 * on[2] * (kx * nn1 * ky + (_rup(on[1], 16) // 16) * nn2 * kx)
    return tiles * per


def compact_apply_flops(ctx):
    """Float64 flops of one compact-layout preconditioner apply (Algorithm 1
    with Step 4): two dense transform solves, 12 (mx+my+mz) mx my mz flops per
    box each, and the correction GEMV, 2 np^2 per box, np = the slots on each
    component's two low transverse faces."""
    dense = gemv = 0
    for i in range(ctx.num_boxes()):
        mx, my, mz = ctx.box(i)["m"]
        dense += 12 * (mx + my + mz) * mx * my * mz
        np_ = (mx * (my * mz - (my - 1) * (mz - 1)) + my * (mx * mz - (mx - 1) * (mz - 1))
               + mz * (mx * my - (mx - 1) * (my - 1)))
        gemv += 2 * np_ * np_
    return 2 * dense + gemv


def orth_flops(n, iters, restart=30):
    """Float64 flops of classical Gram-Schmidt over FGMRES(restart) for
    `iters` Arnoldi steps: per step j of a cycle, <V_i, w> and <w, w>
    (2 (j + 2) n) and w -= V h with ||w||^2 (2 (j + 2) n); the basis stays
    unnormalised (no scaling pass) and re-orthogonalisation passes are not
    counted."""
    tot, done = 0, 0
    while done < iters:
        for j in range(min(restart, iters - done)):
            tot += 4 * (j + 2) * n
        done += restart
    return tot


class OracleIteration:
    """One Arnoldi iteration of the float64 CPU oracle on a workload, as a
    bounded sample: the oracle's exact box solves of `n_boxes` of the
    subdomains (their time scaled to all of them), one sparse SpMV with the
    oracle's assembled operator and modified Gram-Schmidt of the result
    against `basis` vectors (the mean basis size of a restart-30 cycle).
    The operator, the partition and the basis are built once (untimed)."""

    def __init__(self, w, n_boxes=8, basis=15):
        import numpy as np

        from oracle import ras, yee
        self.w = w
        self.ee = yee.edge_eps(w.grid, w.eps_cell)
        self.boxes = ras.partition(w.grid, w.cuts, w.overlap)
        self.A = yee.system_matrix(w.grid, self.ee, w.beta)
        self.sample = self.boxes[:: max(1, len(self.boxes) // n_boxes)][:n_boxes]
        self.x = w.rhs.reshape(-1)
        rng = np.random.default_rng(0)
        self.V = [rng.standard_normal(self.x.size) / np.sqrt(self.x.size) for _ in range(basis)]

    def seconds(self):
        """(total, box-solve part scaled to all boxes, SpMV + MGS part)."""
        import numpy as np

        from oracle import box as obox, ras
        w = self.w
        t0 = time.perf_counter()
        for b in self.sample:
            obox.exact_solve(ras.restrict(w.rhs, b), ras.eps_bar(self.ee, b), w.beta)
        t_pre = (time.perf_counter() - t0) * len(self.boxes) / len(self.sample)
        t0 = time.perf_counter()
        y = self.A @ self.x
        for v in self.V:
            h = float(np.dot(y, v))
            y = y - h * v
        t_rest = time.perf_counter() - t0
        return t_pre + t_rest, t_pre, t_rest

    def describe(self, t_it, iters, src):
        return (f"one oracle Arnoldi iteration: {len(self.sample)} of {len(self.boxes)} box solves (scaled to all), "
                f"sparse SpMV, MGS against {len(self.V)} vectors ({t_it:.2f} s); scaled to {iters} iterations "
                f"({src})")


def oracle_iters(w, iters_gpu=None):
    """FGMRES(30) iteration count of the workload for scaling the oracle's
    per-iteration time: the oracle's own recorded run where one exists
    (oracle/record_fgmres.py), else the GPU float64 run's count, stated as an
    extrapolation."""
    name = {"yee128_ras4x4x4_ol2": "grid128", "yee256_ras8x8x8_ol2": "grid256"}.get(w.name)
    path = os.path.join(ROOT, "oracle", "recorded", f"{name}_fgmres.json")
    if name and os.path.exists(path):
        rec = json.load(open(path))
        return rec["iters"], f"the oracle's own FGMRES(30) count on this workload, oracle/recorded/{name}_fgmres.json"
    if iters_gpu is None:
        raise RuntimeError(f"no recorded oracle iteration count for {w.name}")
    return iters_gpu, "extrapolation: the GPU float64 run's iteration count (no recorded oracle run)"


def run_reference(args):
    """Reference arm: the float64 CPU oracle on the host cores, same workload,
    metric, unit and config; one timed step = one sampled oracle Arnoldi
    iteration, scaled to a full solve by the oracle's recorded FGMRES(30)
    iteration count on that workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(args.workload)
    iters, src = oracle_iters(w)
    it = OracleIteration(w)
    for _ in range(args.warmup):
        it.seconds()
    ts = [it.seconds()[0] for _ in range(args.steps)]
    t_it = sum(ts) / len(ts)
    nx, ny, nz = w.grid
    dof = 3 * nx * ny * nz
    value = dof / (iters * t_it)
    unit = "DoF/s"
    sample = ("per timed step (ms_per_step): " + it.describe(t_it, iters, src) +
              "; value = DoF / the extrapolated solve time")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_it * 1e3, "ms_per_solve_extrapolated": iters * t_it * 1e3,
           "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded eps boxes and uniform rhs)",
           "config": bench_config(w, args),
           "cpu_baseline": {"value": value, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def precond_error(z, ref, boxes):
    """Error of a preconditioner output z against the float64 kernels' ref:
    relative 2-norm, max |z - ref| / max |ref|, and the largest relative
    2-norm over the boxes' owned blocks."""
    d = z - ref
    worst = 0.0
    for b in boxes:
        (x0, y0, z0), n = b["own_lo"], b["own_n"]
        sl = (slice(None), slice(z0, z0 + n[2]), slice(y0, y0 + n[1]), slice(x0, x0 + n[0]))
        worst = max(worst, float(d[sl].norm() / ref[sl].norm()))
    return {"rel_2norm": float(d.norm() / ref.norm()), "max_rel": float(d.abs().max() / ref.abs().max()),
            "max_box_rel_2norm": worst}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2508_07193_b300 import flashmp as F
    from paper_2508_07193_b300 import workloads as wl

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    nx, ny, nz = w.grid
    dof = 3 * nx * ny * nz
    stream = torch.cuda.current_stream(dev)
    ctx = F.Context(w.grid, w.eps_cell, w.beta, w.cuts, w.overlap, precision=args.precision, restart=30,
                    rtol=1e-8, stream=stream, device=dev, krylov=args.krylov, use_graph=args.graph)
    dt = 2.0 * math.sqrt(w.beta)
    setup_s = None
    if args.form != "yee":
        t0 = time.time()
        ctx.set_subdomain_form(args.form)
        setup_s = time.time() - t0
    if args.fused is not None:
        ctx.set_fused(args.fused)
    if args.streamed is not None:
        ctx.set_streamed(args.streamed)
    if args.orth is not None:
        ctx.set_orth(args.orth)
    tuning = None
    if args.autotune and args.precision != "fp64":
        tuning = ctx.autotune(args.precision, reps=3)
    b = torch.as_tensor(w.rhs, device=dev)
    J = (-b / dt).contiguous()
    E = ctx.empty_field()
    H = ctx.empty_field()
    infos = []

    def step():
        E.zero_(); H.zero_()
        infos.append(ctx.cn_step(E, H, J, dt))

    for _ in range(args.warmup):
        step()
    infos.clear()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch0 = ctx.launch_count()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = ctx.launch_count() - n_launch0
    clocks = clk.summary()
    ms = max_over_ranks(ms, world, dev)
    iters = [i["iters"] for i in infos]
    true_res = max(i["true_rel_res"] for i in infos)

    # -- dominant kernel group: the preconditioner apply (3 transform passes) --
    r = b.clone()
    z = ctx.empty_field()
    for _ in range(3):
        ctx.precond_apply(r, z)
    n_p = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n_p):
        ctx.precond_apply(r, z)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1) / n_p
    flops = transform_flops(ctx)
    # SpMV
    e0.record(stream)
    for _ in range(n_p):
        ctx.curlcurl_apply(r, z)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_spmv = e0.elapsed_time(e1) / n_p
    spmv_bytes = 72 * nx * ny * nz      # per cell: read x and eps_edge, write y (3 float64 each)
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6400.0)
    tb = transform_bytes(ctx)
    traffic = TRAFFIC_BYTES.get((w.name, args.precision))
    if args.form == "compact":
        cf = compact_apply_flops(ctx) / (ms_p * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": cf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": cf / FP64_NOMINAL_TFLOPS, "traffic": None,
                "correction_matrix_bytes": ctx.get_subdomain_form()[1],
                "kernel": "compact-layout box solve: two dense float64 transform solves and the Woodbury "
                          "correction GEMV (one preconditioner apply)",
                "peak_source": "B300 nominal float64 rate from the recipe (measured DFMA 1.13 TFLOP/s)"}
    elif args.precision == "fp64_ozaki":
        tf = ozaki_mma_flops(ctx) / (ms_p * 1e-3) / 1e12
        pbf = pk.get("bf16_tflops", 1778.0)
        roof = {"bound": "tensor", "achieved": tf, "peak": pbf, "unit": "TFLOP/s", "frac": tf / pbf,
                "traffic": traffic, "algorithmic_bytes": tb,
                "kernel": "digit-split float64 transform solve (k_oz_fwd_xy + k_oz_z_solve + k_oz_inv_xy, "
                          "bf16 mma.sync digit planes; one preconditioner apply)",
                "peak_source": "of measured (MEASURED_PEAKS.json bf16_tflops, a tcgen05 cuBLAS GEMM)",
                "note": "achieved counts the bf16 flops of the 21 digit-plane products per tile; the kernels "
                        "are bound by the integer issue of cutting and recombining digits, not by the tensor pipe",
                "dense_fp64_equivalent_tflops": flops / (ms_p * 1e-3) / 1e12}
    elif args.precision == "fp64":
        ops = transform_fp64_executed(ctx)
        sm_mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
        peak_ops = fp64_issue_peak_tops(sm_mhz)
        achieved = ops / (ms_p * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Top/s (float64 operations)",
                "frac": achieved / peak_ops, "traffic": traffic, "algorithmic_bytes": tb,
                "kernel": "float64 transform solve (passes A+B+C = one preconditioner apply)",
                "peak_source": f"float64 issue rate derived from the recipe's unit counts and clocks: "
                               f"{FP64_OPS_PER_CLK_SM} operations per clock per SM x {N_SMS} SMs x {sm_mhz:.0f} MHz "
                               f"(the median SM clock sampled in the timed region)",
                "executed_ops_per_apply": ops,
                "dense_equivalent_tflops": flops / (ms_p * 1e-3) / 1e12,
                "note": "achieved counts the float64 operations (FMAs, multiplications and additions) the "
                        "three-level folded kernels execute, from a per-line model within 2-7 % of ncu's count "
                        "per pass; dense_equivalent_tflops counts the dense 12(mx+my+mz)mxmymz formula, whose "
                        "FMAs the folded kernels' operations number about a third of"}
    else:
        achieved = tb / (ms_p * 1e-3) / 1e9
        kern = ("fused cluster kernel (one 3-CTA cluster per box)" if args.precision != "tf32"
                else "three-pass kernels")
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "algorithmic_bytes": tb,
                "kernel": f"{args.precision} transform solve, {kern} (one preconditioner apply)",
                "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    spmv_gbs = spmv_bytes / (ms_spmv * 1e-3) / 1e9
    roof_spmv = {"bound": "hbm", "achieved": spmv_gbs, "peak": hbm, "unit": "GB/s", "frac": spmv_gbs / hbm,
                 "kernel": "k_curlcurl (SpMV)", "peak_source": "of measured"}

    # -- e2e: the step's input J from pinned host memory (H2D) and its result
    # E back to the host (D2H), every step; one untimed pass first so that
    # first-use costs of the copies stay out of the timed region --
    # The copies overlap the compute the way a time-stepping caller would run
    # them: step n+1's J uploads on a copy stream while step n solves, and
    # step n's E, snapshotted on the device, downloads while step n+1 solves.
    # Two buffers each; events order every reuse; all copies complete inside
    # the timed region.
    hJ = torch.empty_like(J, device="cpu").pin_memory()
    hJ.copy_(J.cpu())
    hE = [torch.empty_like(hJ).pin_memory() for _ in range(2)]
    Jd = [torch.empty_like(J) for _ in range(2)]
    Es = [torch.empty_like(E) for _ in range(2)]
    cps = torch.cuda.Stream(device=dev)
    ev = lambda: torch.cuda.Event()
    up, used, snap, down = [ev(), ev()], [ev(), ev()], [ev(), ev()], [ev(), ev()]

    def e2e_run(k):
        with torch.cuda.stream(cps):
            Jd[0].copy_(hJ, non_blocking=True)
            up[0].record(cps)
        for n in range(k):
            b = n % 2
            if n + 1 < k:   # upload the next step's input once step n-1 no longer reads that buffer
                with torch.cuda.stream(cps):
                    if n >= 1:
                        cps.wait_event(used[1 - b])
                    Jd[1 - b].copy_(hJ, non_blocking=True)
                    up[1 - b].record(cps)
            stream.wait_event(up[b])
            if n >= 2:
                stream.wait_event(down[b])   # Es[b] free again
            E.zero_(); H.zero_()
            ctx.cn_step(E, H, Jd[b], dt)
            used[b].record(stream)
            Es[b].copy_(E)
            snap[b].record(stream)
            with torch.cuda.stream(cps):
                cps.wait_event(snap[b])
                hE[b].copy_(Es[b], non_blocking=True)
                down[b].record(cps)
        stream.wait_stream(cps)

    e2e_run(2)
    torch.cuda.synchronize()
    e0.record(stream)
    n_e = max(2, min(4, args.steps))
    e2e_run(n_e)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / n_e, world, dev)

    out = {
        "metric": METRIC,
        "value": job_value(dof, world, ms),
        "unit": "DoF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64" if args.precision == "fp64" else
                  "f64 (preconditioner transforms float64-accurate on bf16 digit planes, exact fp32 accumulation)"
                  if args.precision == "fp64_ozaki" else f"f64 (preconditioner transforms {args.precision})"),
        "data": "synthetic (seeded eps boxes and uniform rhs)",
        "config": bench_config(w, args),
        "iters_per_step": iters,
        "true_rel_res_max": true_res,
        "precond_ms": ms_p,
        "subdomain_dof_per_s": dof / (ms_p * 1e-3),
        "spmv_ms": ms_spmv,
        "roofline": roof,
        "roofline_spmv": roof_spmv,
        "e2e": {"value": job_value(dof, world, ms_e2e), "unit": "DoF/s", "h2d_bytes_per_step": J.numel() * 8,
                "d2h_bytes_per_step": E.numel() * 8, "ms_per_step": ms_e2e,
                "copies": "pinned host J in and E out every step, on a copy stream overlapping the neighbouring "
                          "steps' compute (double buffers), all complete inside the timed region"},
        "gpu_launches": launches,
        "form_setup_s": setup_s,
        "tuning": list(tuning) if tuning else list(ctx.get_tuning()),
        "clocks": clocks,
    }
    # phase breakdown from one extra (untimed) step with CUDA-event phase timers
    ctx.set_options(timing=True)
    E.zero_(); H.zero_()
    ph = ctx.cn_step(E, H, J, dt)
    ctx.set_options(timing=False)
    out["phase_ms"] = {k: ph[k] for k in ("ms_precond", "ms_spmv", "ms_orth", "ms_total")}
    if args.krylov == "fgmres" and ph["ms_orth"] > 0:
        of = orth_flops(dof, ph["iters"]) / 2 / (ph["ms_orth"] * 1e-3) / 1e12
        pk_ops = fp64_issue_peak_tops(clocks.get("sm_mhz"))
        ob = orth_flops(dof, ph["iters"]) / 2 * 8 / (ph["ms_orth"] * 1e-3) / 1e9
        if ctx.get_orth() == ctx.ORTH_MODES["split"]:
            out["roofline_orth"] = {
                "bound": "hbm", "achieved": ob, "peak": hbm, "unit": "GB/s", "frac": ob / hbm,
                "fp64_fma_equiv_tops": of, "fp64_issue_frac": of / pk_ops,
                "kernel": "Gram-Schmidt basis passes k_dots_sp / k_update_sp (one step)",
                "note": "algorithmic bytes: one 8-byte read of every basis element and of w per pass (the "
                        "update's write of w not counted); the oldest vectors of each pass take exact "
                        "fixed-point products on the integer pipes, the rest float64 FMAs, so the float64 "
                        "pipe's time is brought down to about HBM's"}
        else:
            out["roofline_orth"] = {"bound": "alu", "achieved": of, "peak": pk_ops, "unit": "Top/s (float64 FMAs)",
                                    "frac": of / pk_ops, "achieved_gbs": ob, "hbm_frac": ob / hbm,
                                    "kernel": "Gram-Schmidt basis passes k_dots / k_update (one step)",
                                    "note": "one float64 FMA per 8-byte basis element read: the float64 pipe, "
                                            "not HBM, bounds them"}
    # the other preconditioner precisions on the same workload, same protocol,
    # each with its preconditioner error against the float64 kernels (which
    # the parity tests hold within 1e-11 of the float64 oracle) on r = b
    if not args.no_forms and args.form == "yee":
        forms = {}
        max_ext = max(max(ctx.box(i)["m"]) for i in range(ctx.num_boxes()))
        ctx.set_options(precision="fp64")
        ctx.precond_apply(r, z)
        z64 = z.clone()
        owned = [ctx.box(i) for i in range(ctx.num_boxes())]
        # (form, transform precision, Krylov method): every precision with the
        # run's method, and the reduced-precision transforms with BiCGSTAB
        # (two applies and two SpMVs per iteration, no Gram-Schmidt) beside an
        # FGMRES run
        runs = [(p, p, args.krylov) for p in ("fp64", "fp64_ozaki", "bf16", "fp16", "tf32")]
        if args.krylov == "fgmres":
            runs += [(p + "_bicgstab", p, "bicgstab") for p in ("bf16", "fp16")]
        for name, p, kr in runs:
            if p == "fp64_ozaki" and max_ext > OZAKI_MAX_EXTENT:
                continue
            if p == args.precision and kr == args.krylov:
                forms[name] = {"ms_per_step": ms, "iters": iters[0] if iters else None, "true_rel_res_max": true_res,
                               "precond_ms": ms_p}
            else:
                ctx.set_options(precision=p, krylov=kr)
                infos.clear()
                for _ in range(args.warmup):
                    step()
                infos.clear()
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(args.steps):
                    step()
                e1.record(stream)
                torch.cuda.synchronize()
                fm = e0.elapsed_time(e1) / args.steps
                for _ in range(3):
                    ctx.precond_apply(r, z)
                e0.record(stream)
                for _ in range(n_p):
                    ctx.precond_apply(r, z)
                e1.record(stream)
                torch.cuda.synchronize()
                forms[name] = {"ms_per_step": fm, "iters": infos[0]["iters"],
                               "true_rel_res_max": max(i["true_rel_res"] for i in infos),
                               "precond_ms": e0.elapsed_time(e1) / n_p}
                if kr != args.krylov:
                    forms[name]["krylov"] = "BiCGSTAB" if kr == "bicgstab" else "FGMRES(30)"
            if forms[name]["iters"]:
                # iteration counts of BiCGSTAB with a 16-bit preconditioner move with the summation
                # order of its dot products; the time per iteration is the kernels' measure
                forms[name]["ms_per_iteration"] = forms[name]["ms_per_step"] / forms[name]["iters"]
            if p != "fp64":
                ctx.set_options(precision=p, krylov=kr)
                ctx.precond_apply(r, z)
                forms[name]["precond_err_vs_fp64"] = precond_error(z, z64, owned)
            if p == "fp64_ozaki":
                forms[name]["mma_tflops"] = ozaki_mma_flops(ctx) / (forms[name]["precond_ms"] * 1e-3) / 1e12
        ctx.set_options(precision=args.precision, krylov=args.krylov)
        out["forms"] = forms
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, iters[0] if iters else 1)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    ctx.close()


def cpu_baseline(w, iters_gpu):
    """The float64 CPU oracle as it stands, timed on a bounded sample of the
    step (one Arnoldi iteration with 8 of the box solves), scaled to the
    oracle's own recorded iteration count (or the GPU run's, stated)."""
    it = OracleIteration(w)
    t_it = it.seconds()[0]
    iters, src = oracle_iters(w, iters_gpu)
    nx, ny, nz = w.grid
    return {"value": 3 * nx * ny * nz / (iters * t_it), "unit": "DoF/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": it.describe(t_it, iters, src)}


def run_case(args):
    """W + K applies of one operator on a workload, for profiler captures;
    `--case box` times the exact solve of the single 32^3 PEC box (the plain
    float64 transform solve of one box, fmp_box_solve)."""
    import numpy as np
    import torch

    from paper_2508_07193_b300 import flashmp as F

    name = "box32" if args.case == "box" else args.workload
    w = workload(name)
    ctx = F.Context(w.grid, w.eps_cell, w.beta, w.cuts, w.overlap, precision=args.precision)
    if args.form != "yee":
        ctx.set_subdomain_form(args.form)
    if args.fused is not None:
        ctx.set_fused(args.fused)
    if args.streamed is not None:
        ctx.set_streamed(args.streamed)
    r = torch.as_tensor(w.rhs, device="cuda")
    z = ctx.empty_field()
    if args.case == "box":
        op = lambda a, b: ctx.box_solve(0, a, b)
    else:
        op = {"precond": ctx.precond_apply, "spmv": ctx.curlcurl_apply, "cnn": ctx.cnn_apply}[args.case]
    if args.case == "cnn":
        ctx.cnn_set_params(np.random.default_rng(0).normal(0.0, 0.05, ctx.cnn_num_params()).astype(np.float32))
        ctx.cnn_set_tc(not args.cnn_mma_sync)
    for _ in range(args.warmup):
        op(r, z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for _ in range(args.steps):
        op(r, z)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    out = {"case": args.case, "workload": w.name, "applies": args.warmup + args.steps, "ms_per_apply": ms}
    nx, ny, nz = w.grid
    if args.case == "cnn":
        flops = CNN_FLOPS_PER_VOXEL * nx * ny * nz
        out.update({"tflops": flops / (ms * 1e-3) / 1e12, "flops_per_apply": flops,
                    "kernels": "mma.sync" if args.cnn_mma_sync else "tcgen05 (all four layers)"})
    if args.case in ("box", "precond"):
        out.update({"fused": ctx.get_fused(), "streamed": ctx.get_streamed()})
        out.update({"subdomain_dof_per_s": 3 * nx * ny * nz / (ms * 1e-3),
                    "dense_equivalent_tflops": transform_flops(ctx) / (ms * 1e-3) / 1e12,
                    "precision": args.precision})
        if args.precision == "fp64":
            ops = transform_fp64_executed(ctx)
            out.update({"executed_ops_per_apply": ops, "executed_tops": ops / (ms * 1e-3) / 1e12,
                        "fp64_issue_frac_at_max_clock": ops / (ms * 1e-3) / 1e12 / fp64_issue_peak_tops()})
    print(json.dumps(out))
    ctx.close()


def main():
    args = parse()
    if args.case != "step":
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
