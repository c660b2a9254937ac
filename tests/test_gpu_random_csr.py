"""The random complex-symmetric stress workload at full size (n = 2^22, 256 shifts
sigma_k + 0.3i).  Every 16th shift (16 of the 256) is checked three ways: its true
residual, recomputed by an independent sparse product on the host, meets the
tolerance; its solution equals the oracle's independent BiCGStab solve of that one
system to 1e-8 (FP64); and the FP32-mixed solution equals the oracle's to 1e-4.
The 16 oracle solves run in a spawn process pool while the GPU solves."""
import os
import tempfile

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle_pool
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    wl = workloads.RANDOM_CSR
    rowptr, col, val = workloads.random_symmetric_csr(wl.n, wl.half_nnz_per_row, wl.diag_range, wl.matrix_seed)
    b = workloads.random_complex_rhs(wl.n, wl.rhs_seed)
    sig = workloads.random_shifts(wl.n_shifts, *wl.shift_range, wl.shift_imag, wl.shift_seed)
    return wl, rowptr, col, val, b, sig


def test_full_size_fp64_and_mixed(cuda, problem):
    from paper_2506_09551_gb300 import api
    wl, rowptr, col, val, b, sig = problem
    sample = list(range(0, wl.n_shifts, 16))
    with tempfile.TemporaryDirectory() as d:
        for name, arr in (("rowptr", rowptr), ("col", col), ("val", val), ("b", b)):
            np.save(os.path.join(d, name + ".npy"), arr)
        with oracle_pool.pool(len(sample)) as pool:
            pending = pool.map_async(oracle_pool.csr_shift_solve, [(d, complex(sig[k]), 1e-12) for k in sample])
            A = sp.csr_matrix((val, col, rowptr), shape=(wl.n, wl.n))
            seed = int(np.argsort(sig.real)[len(sig) // 2])
            op = api.Operator.csr(rowptr, col, val)
            bt = torch.tensor(b, device="cuda")
            x, per, info, st = op.multishift_solve(bt, sig - sig[seed], -sig[seed], tol=1e-10, maxit=20000)
            assert st == 0 and per["converged"].all()
            nb = np.linalg.norm(b)
            X = {}
            for k in sample:
                xk = x[k].cpu().numpy()
                X[k] = xk
                r = b - (A @ xk - sig[k] * xk)
                assert np.linalg.norm(r) <= 10 * 1e-10 * nb, (k, np.linalg.norm(r) / nb)
            del x
            xm, per_m, info_m, st_m = op.multishift_solve(bt, sig - sig[seed], -sig[seed], tol=1e-7, maxit=20000,
                                                          prec=api.FP32_MIXED)
            assert per_m["converged"].all()
            XM = {k: xm[k].cpu().numpy().astype(np.complex128) for k in sample}
            del xm
            ref = pending.get()
    for i, k in enumerate(sample):
        xr = ref[i][0]
        e64 = np.linalg.norm(X[k] - xr) / np.linalg.norm(xr)
        e32 = np.linalg.norm(XM[k] - xr) / np.linalg.norm(xr)
        print(f"shift {k} ({sig[k]:.3f}): FP64 {e64:.2e}, FP32-mixed {e32:.2e} vs the oracle's own solve")
        assert e64 <= 1e-8, (k, e64)
        assert e32 <= 1e-4, (k, e32)
