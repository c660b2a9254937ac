"""Record the oracle's own work counts on a map workload (TEST INFRASTRUCTURE ONLY).

For a sample of incident-energy rows, runs the oracle's per-row pipeline in
full (independent BiCGStab solve to 1e-13, continued fraction to cf_tol) and
writes the matrix-vector product counts and continued-fraction depths, plus the
ground-state Lanczos step count, to a JSON file.  The CPU-baseline leg of the
benchmark times a bounded part of the same pipeline and scales it to a whole
map with these counts.

    python -m oracle.measure_costs hubbard-L12-fp64 out.json [rows...]
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np


def _row(args):
    name, k, E_G = args
    import scipy.sparse as sp
    import workloads
    from oracle import hubbard, solvers, spectrum
    wl = {w.name: w for w in (workloads.CHAIN8, workloads.CHAIN12, workloads.CHAIN14)}[name]
    m = hubbard.RixsModel(wl.L, wl.n_up, wl.n_dn, wl.t, wl.U, wl.Uc, wl.core_site)
    E_G, G, _ = solvers.ground_state(m.H, workloads.lanczos_start(m.H.shape[0], wl.lanczos_seed), kmax=300)
    n = m.Hp.shape[0]
    A = (m.Hp - (E_G + 1j * wl.Gamma) * sp.identity(n)).tocsr()
    t0 = time.perf_counter()
    X, nmv = solvers.solve_shifted(A, m.O2 @ G, np.array([wl.w_in[k]]), tol=1e-13, method="bicgstab")
    t1 = time.perf_counter()
    I, depth = spectrum.lanczos_cf(m.H, m.O1 @ X[0], E_G, wl.w, wl.eta, cf_tol=1e-13)
    t2 = time.perf_counter()
    return dict(row=int(k), w_in=float(wl.w_in[k]), solve_matvecs=int(nmv), cf_depth=int(depth),
                solve_seconds=t1 - t0, cf_seconds=t2 - t1)


def main():
    name, out = sys.argv[1], sys.argv[2]
    rows = [int(r) for r in sys.argv[3:]] or [0, 20, 40, 60, 80, 100]
    import workloads
    from oracle import hubbard, solvers
    wl = {w.name: w for w in (workloads.CHAIN8, workloads.CHAIN12, workloads.CHAIN14)}[name]
    t0 = time.perf_counter()
    m = hubbard.RixsModel(wl.L, wl.n_up, wl.n_dn, wl.t, wl.U, wl.Uc, wl.core_site)
    t_build = time.perf_counter() - t0
    steps = {}

    class Counting:
        def __init__(self, H):
            self.H, self.n = H, 0
            self.shape = H.shape

        def __matmul__(self, v):
            self.n += 1
            return self.H @ v

    cH = Counting(m.H)
    t0 = time.perf_counter()
    E_G, G, _ = solvers.ground_state(cH, workloads.lanczos_start(m.H.shape[0], wl.lanczos_seed), kmax=300)
    t_gs = time.perf_counter() - t0
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(rows), os.cpu_count() or 1)) as pool:
        res = pool.map(_row, [(name, k, E_G) for k in rows])
    rec = dict(workload=name, rows=res, ground_state_matvecs=cH.n, build_seconds=t_build, ground_state_seconds=t_gs,
               mean_solve_matvecs=float(np.mean([r["solve_matvecs"] for r in res])),
               mean_cf_depth=float(np.mean([r["cf_depth"] for r in res])),
               command="python -m oracle.measure_costs " + " ".join(sys.argv[1:]))
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main()
