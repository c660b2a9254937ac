"""The random complex-symmetric stress workload at full size (n = 2^22, 256 shifts
sigma_k + 0.3i): every sampled shift's true residual, recomputed by an independent
sparse product on the host, meets the tolerance, and the FP32-mixed solutions agree
with the FP64 ones to 1e-4."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

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
    A = sp.csr_matrix((val, col, rowptr), shape=(wl.n, wl.n))
    seed = int(np.argsort(sig.real)[len(sig) // 2])
    op = api.Operator.csr(rowptr, col, val)
    bt = torch.tensor(b, device="cuda")
    x, per, info, st = op.multishift_solve(bt, sig - sig[seed], -sig[seed], tol=1e-10, maxit=20000)
    assert st == 0 and per["converged"].all()
    nb = np.linalg.norm(b)
    sample = list(range(0, wl.n_shifts, 16))
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
    for k in sample:
        xk = xm[k].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(xk - X[k]) <= 1e-4 * np.linalg.norm(X[k]), k
