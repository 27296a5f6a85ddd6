"""CN steps started from the extrapolated guess 2 E^n - E^(n-1)
(fmp_cn_step_guess): the same steps as the oracle's direct-solve CN steps
(Sec. II-A, Eqs. 2-4) within the solve tolerance, with fewer iterations on a
smooth source than the plain guess E^n."""
import numpy as np
import pytest

from oracle import cn, yee
from paper_2508_07193_b300 import workloads as wl
from tests._gpu import context, dev, host, rel

pytestmark = pytest.mark.gpu


def test_extrapolated_guess_matches_oracle_steps():
    w = wl.small(grid=(10, 9, 8), cuts=((5, 5), (4, 5), (8,)), overlap=2, seed=31, n_eps_boxes=3)
    g = w.grid
    ee = yee.edge_eps(g, w.eps_cell)
    dt = 2.0 * np.sqrt(w.beta)
    ctx = context(w, rtol=1e-12)
    E = np.zeros_like(w.rhs); H = np.zeros_like(E)
    Ed, Hd, Pd = dev(E), dev(H), dev(E)
    for n in range(5):
        J = wl.dipole_current(g, n, dt) * 10
        cur = Ed.clone()
        ctx.cn_step(Ed, Hd, dev(J), dt, E_prev=Pd)
        Pd.copy_(cur)
        E, H = cn.step(g, ee, E, H, J, dt)
    assert rel(host(Ed), E) <= 1e-9 and rel(host(Hd), H) <= 1e-9


def test_extrapolation_saves_iterations_on_a_smooth_source():
    w = wl.make_workload("dipole24", (24, 24, 24), seed=4, n_eps_boxes=6, cuts=[wl.even_cuts(24, 2)] * 3, overlap=2)
    dt = 2.0 * np.sqrt(w.beta)
    out = {}
    for extrap in (False, True):
        ctx = context(w, rtol=1e-10)
        E, H = ctx.empty_field(), ctx.empty_field()
        P = ctx.empty_field()
        its = 0
        for n in range(30):
            J = dev(wl.dipole_current(w.grid, n, dt))
            cur = E.clone()
            info = ctx.cn_step(E, H, J, dt, E_prev=P if extrap else None)
            P.copy_(cur)
            if n >= 10:
                its += info["iters"]
            assert info["true_rel_res"] <= 1e-10
        out[extrap] = (its, host(E), host(H))
    assert out[True][0] < out[False][0]
    assert rel(out[True][1], out[False][1]) <= 1e-8 and rel(out[True][2], out[False][2]) <= 1e-8
