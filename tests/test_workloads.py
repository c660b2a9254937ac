"""The seeded input generators (shared by the oracle and the CUDA path)."""
import numpy as np

import workloads


def test_random_symmetric_csr_structure():
    rowptr, col, val = workloads.random_symmetric_csr(2000, 8, seed=5)
    n = 2000
    assert rowptr[0] == 0 and rowptr[-1] == len(col) == len(val)
    import scipy.sparse as sp
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    assert abs(A - A.T).max() == 0.0
    d = A.diagonal()
    assert d.min() >= -4 and d.max() <= 4
    nnz_off = A.nnz - n
    assert 14.5 * n < nnz_off <= 16 * n
    for i in (0, 17, 1999):
        c = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    # deterministic
    r2, c2, v2 = workloads.random_symmetric_csr(2000, 8, seed=5)
    assert np.array_equal(c2, col) and np.array_equal(v2, val)


def test_grids_and_seed():
    w = workloads.CHAIN8
    assert len(w.w_in) == 41 and len(w.w) == 200
    assert w.w_in[workloads.seed_index(w.w_in)] == 0.0
    assert workloads.seed_index(workloads.CHAIN12.w_in) in range(101)
    s = workloads.random_shifts(256, -6, 6, 0.3)
    assert np.all(s.imag == 0.3) and s.real.min() >= -6 and s.real.max() <= 6
