"""Oracle jobs for the GPU parity tests, run in worker processes (TEST INFRASTRUCTURE).

The plain per-incident-energy oracle (an independent BiCGStab solve of Eq. 2,
phi = O1 Psi, and the continued fraction of Eq. 1) costs minutes per row at the
full workload sizes, so the tests spread rows (or shifts) over a process pool.
The pool uses the "spawn" start method, since a process forked after CUDA is
initialised can hang, and one BLAS thread per worker.  Every function here only
calls `oracle/`; nothing comes from the CUDA path.
"""
from __future__ import annotations

import multiprocessing as mp
import os


def pool(n_jobs: int):
    """A spawn process pool of min(n_jobs, host cores) single-threaded workers."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return mp.get_context("spawn").Pool(max(1, min(n_jobs, cores)))


def map_row(job):
    """I(w_in, w) of one incident energy by the plain definition (Eqs. 1-2).

    job = (L, n_up, n_dn, core_site, Gamma, eta, E_G, G, w_in, w, solve_tol, cf_tol)."""
    import numpy as np
    import scipy.sparse as sp

    from oracle import hubbard, solvers, spectrum
    L, n_up, n_dn, core, Gamma, eta, E_G, G, w_in, w, solve_tol, cf_tol = job
    gsec = hubbard.Sector(L, n_up, n_dn)
    isec = hubbard.Sector(L, n_up + 1, n_dn)
    H = hubbard.hamiltonian_kron(gsec, 1.0, 8.0)
    Hp = hubbard.hamiltonian_kron(isec, 1.0, 8.0, 4.0, core)
    O2 = hubbard.creation_operator(gsec, isec, core, 0)
    O1 = hubbard.annihilation_operator(isec, gsec, core, 0)
    n = Hp.shape[0]
    A = (Hp - (E_G + w_in + 1j * Gamma) * sp.identity(n, format="csr")).tocsr()
    psi, _ = solvers.bicgstab(lambda v: A @ v, (O2 @ G).astype(np.complex128), solve_tol)
    I, _ = spectrum.lanczos_cf(H, O1 @ psi, E_G, np.asarray(w), eta, cf_tol=cf_tol)
    return I


def csr_shift_solve(job):
    """x = (A - sigma I)^{-1} b by BiCGStab for the random sparse workload.  A's CSR
    arrays and b are read from .npy files memory-mapped by every worker (one copy
    in the page cache).  job = (directory, sigma, tol)."""
    import numpy as np
    import scipy.sparse as sp

    from oracle import solvers
    d, sigma, tol = job
    rowptr = np.load(os.path.join(d, "rowptr.npy"), mmap_mode="r")
    col = np.load(os.path.join(d, "col.npy"), mmap_mode="r")
    val = np.load(os.path.join(d, "val.npy"), mmap_mode="r")
    b = np.load(os.path.join(d, "b.npy"))
    n = len(rowptr) - 1
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n), copy=False)
    x, nmv = solvers.bicgstab(lambda v: A @ v - sigma * v, b, tol)
    return x, nmv
