"""Record the oracle's FGMRES(30) iteration count on a benchmark workload.

Test infrastructure: runs only the float64 CPU oracle and writes
oracle/recorded/<workload>_fgmres.json, which the CPU reference arm of the
benchmark reads to scale its per-iteration timing to a full step, and which
the GPU tests compare the library's iteration count against. The 128^3
workload takes about three minutes on 8 cores; the 256^3 one about half an
hour and 45 GB of host memory (basis V and Z of 31 and 30 vectors of 50.3 M
unknowns, plus the sparse operator).

    python -m oracle.record_fgmres [grid128|grid256]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import krylov, ras, yee  # noqa: E402
from paper_2508_07193_b300 import workloads as wl  # noqa: E402


def main(name="grid128"):
    w = {"grid128": wl.grid128, "grid256": wl.grid256}[name]()
    ee = yee.edge_eps(w.grid, w.eps_cell)
    A = yee.system_matrix(w.grid, ee, w.beta)
    boxes = ras.partition(w.grid, w.cuts, w.overlap)
    shp = w.rhs.shape
    M = lambda r: ras.precond_apply(r.reshape(shp), boxes, ee, w.beta).reshape(-1)
    t0 = time.time()
    x, info = krylov.fgmres(lambda v: A @ v, M, w.rhs.reshape(-1), restart=30, rtol=1e-8)
    out = {"workload": w.name, "krylov": "FGMRES(30), modified Gram-Schmidt", "rtol": 1e-8,
           "iters": info["iters"], "restarts": info["restarts"], "true_rel_res": info["true_rel_res"],
           "seconds": time.time() - t0, "cores": os.cpu_count()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "recorded", f"{name}_fgmres.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main(*sys.argv[1:2])
