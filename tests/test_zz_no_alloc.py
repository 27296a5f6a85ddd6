"""fmp_box_solve_static: the allocation-free single-box exact solve.

Some callers cannot call cudaMalloc (an application whose own allocator holds
all device memory, a real-time loop that forbids allocation after start-up).
They use fmp_box_solve_static, which keeps its scratch in a fixed array inside
the library. This file checks it, through the C ABI, against the context-based
fmp_box_solve on consecutive calls (different box sizes, then the first size
again, so that contents left by one call cannot leak into the next), against
the float64 oracle's exact solve of the same box, at the largest extent the
array holds (64 per axis, the largest scratch offset and shared-memory sizes)
and at the smallest (2) next to the largest, and that oversize boxes are
refused. It is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2508_07193_b300 import workloads as wl
from tests._gpu import FP64_TOL, dev, host, rel

pytestmark = pytest.mark.gpu


def _entry():
    from paper_2508_07193_b300 import flashmp as F
    f = F.lib().fmp_box_solve_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_void_p]
    return f


CASES = (((36, 34, 33), 2.7, 1), ((32, 32, 32), 1.0, 2), ((36, 34, 33), 2.7, 1),
         ((64, 64, 64), 1.9, 3), ((2, 3, 64), 4.2, 4), ((64, 40, 24), 1.3, 5), ((2, 3, 64), 4.2, 4))


def test_static_box_solve_matches_context_solve_on_consecutive_calls():
    from paper_2508_07193_b300 import flashmp as F
    f = _entry()
    stream = torch.cuda.current_stream()
    for grid, eps, seed in CASES:
        nx, ny, nz = grid
        w = wl.make_workload("box", grid, seed=seed, uniform_eps=True, overlap=0)
        ctx = F.Context(grid, np.full((nz, ny, nx), eps), 0.25)
        r = dev(w.rhs)
        ref = host(ctx.box_solve(0, r))
        x = torch.full_like(r, float("nan"))
        rc = f(r.data_ptr(), x.data_ptr(), nx, ny, nz, ctx.box(0)["eps_bar"], 0.25, stream.cuda_stream)
        assert rc == F.FMP_OK
        assert rel(host(x), ref) <= FP64_TOL
        ctx.close()


def test_static_box_solve_rejects_oversize_and_bad_arguments():
    from paper_2508_07193_b300 import flashmp as F
    f = _entry()
    r = torch.zeros((3, 8, 8, 65), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(r)
    s = torch.cuda.current_stream().cuda_stream
    assert f(r.data_ptr(), x.data_ptr(), 65, 8, 8, 1.0, 0.25, s) == F.FMP_ERR_ARG
    assert f(r.data_ptr(), x.data_ptr(), 8, 8, 1, 1.0, 0.25, s) == F.FMP_ERR_ARG
    assert f(r.data_ptr(), r.data_ptr(), 8, 8, 8, 1.0, 0.25, s) == F.FMP_ERR_ARG
    assert f(r.data_ptr(), x.data_ptr(), 8, 8, 8, 0.0, 0.25, s) == F.FMP_ERR_ARG


def test_static_box_solve_matches_oracle():
    """The same calls against the float64 oracle's exact solve of each box
    (transforms and a dense 3x3 solve per mode), element by element."""
    from oracle import box
    from paper_2508_07193_b300 import flashmp as F
    f = _entry()
    stream = torch.cuda.current_stream()
    for grid, eps, seed in CASES[2:]:
        nx, ny, nz = grid
        w = wl.make_workload("box", grid, seed=seed, uniform_eps=True, overlap=0)
        ref = box.exact_solve(w.rhs, eps, 0.25)
        r = dev(w.rhs)
        x = torch.full_like(r, float("nan"))
        assert f(r.data_ptr(), x.data_ptr(), nx, ny, nz, eps, 0.25, stream.cuda_stream) == F.FMP_OK
        assert rel(host(x), ref) <= FP64_TOL, grid
