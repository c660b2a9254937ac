"""The random complex-symmetric stress workload (256 shifts sigma_k + 0.3i).

Full size, n = 2^22: the FP64 solve to 1e-12, and on every 16th shift (16 of the 256)
* the true residual r = b - (A - sigma_k) x_k, recomputed by an independent sparse
  product on the host, meets the tolerance;
* a certified bound on the error against the exact solution: A is real symmetric, so
  A - sigma I is normal with every singular value >= Im sigma = 0.3, hence
  ||x - x*|| <= ||r|| / 0.3 and ||x*|| >= ||b|| / ||A - sigma||, with ||A - sigma||
  bounded by Gershgorin on the host: the relative error is at most
  ||r|| ||A - sigma||_G / (0.3 ||b||), asserted <= 1e-8;
* the FP32-mixed solution equals the FP64 one to 1e-4.
Reduced size, n = 2^16 with the same generator: the same 16 shifts against the oracle's
independent BiCGStab solves (a spawn process pool), 1e-8 (FP64) and 1e-4 (mixed).
"""
import os
import tempfile

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle_pool
import workloads

pytestmark = pytest.mark.gpu


def _problem(n):
    wl = workloads.RANDOM_CSR
    rowptr, col, val = workloads.random_symmetric_csr(n, wl.half_nnz_per_row, wl.diag_range, wl.matrix_seed)
    b = workloads.random_complex_rhs(n, wl.rhs_seed)
    sig = workloads.random_shifts(wl.n_shifts, *wl.shift_range, wl.shift_imag, wl.shift_seed)
    return wl, rowptr, col, val, b, sig


def _gpu_solves(rowptr, col, val, b, sig, tol64, tol32):
    from paper_2506_09551_gb300 import api
    seed = int(np.argsort(sig.real)[len(sig) // 2])
    op = api.Operator.csr(rowptr, col, val)
    bt = torch.tensor(b, device="cuda")
    x, per, info, st = op.multishift_solve(bt, sig - sig[seed], -sig[seed], tol=tol64, maxit=40000)
    assert st == 0 and per["converged"].all()
    sample = list(range(0, len(sig), 16))
    X = {k: x[k].cpu().numpy() for k in sample}
    del x
    xm, per_m, info_m, st_m = op.multishift_solve(bt, sig - sig[seed], -sig[seed], tol=tol32, maxit=40000,
                                                  prec=api.FP32_MIXED)
    assert per_m["converged"].all()
    XM = {k: xm[k].cpu().numpy().astype(np.complex128) for k in sample}
    del xm
    return sample, X, XM


def test_full_size_certified_error(cuda):
    n = workloads.RANDOM_CSR.n
    wl, rowptr, col, val, b, sig = _problem(n)
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    sample, X, XM = _gpu_solves(rowptr, col, val, b, sig, 1e-12, 1e-7)
    nb = np.linalg.norm(b)
    gersh = float(np.max(np.asarray(abs(A).sum(axis=1)).ravel()))       # >= ||A||_2
    for k in sample:
        r = b - (A @ X[k] - sig[k] * X[k])
        rel_r = np.linalg.norm(r) / nb
        assert rel_r <= 10 * 1e-12, (k, rel_r)
        bound = rel_r * (gersh + abs(sig[k])) / sig[k].imag
        assert bound <= 1e-8, (k, bound)
        dm = np.linalg.norm(XM[k] - X[k]) / np.linalg.norm(X[k])
        print(f"shift {k} ({sig[k]:.3f}): residual {rel_r:.1e}, certified FP64 error <= {bound:.1e}, "
              f"mixed vs FP64 {dm:.1e}")
        assert dm <= 1e-4, (k, dm)


def test_reduced_size_against_oracle_solves(cuda):
    n = 1 << 16
    wl, rowptr, col, val, b, sig = _problem(n)
    with tempfile.TemporaryDirectory() as d:
        for name, arr in (("rowptr", rowptr), ("col", col), ("val", val), ("b", b)):
            np.save(os.path.join(d, name + ".npy"), arr)
        sample = list(range(0, wl.n_shifts, 16))
        with oracle_pool.pool(len(sample)) as pool:
            pending = pool.map_async(oracle_pool.csr_shift_solve, [(d, complex(sig[k]), 1e-12) for k in sample])
            sample, X, XM = _gpu_solves(rowptr, col, val, b, sig, 1e-12, 1e-7)
            ref = pending.get()
    for i, k in enumerate(sample):
        xr = ref[i][0]
        e64 = np.linalg.norm(X[k] - xr) / np.linalg.norm(xr)
        e32 = np.linalg.norm(XM[k] - xr) / np.linalg.norm(xr)
        assert e64 <= 1e-8, (k, e64)
        assert e32 <= 1e-4, (k, e32)
