"""GPU parity of the operator kernels against the oracle's explicit CSR matrices."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import hubbard
import workloads

pytestmark = pytest.mark.gpu

CASES = [  # (L, n_up, n_dn, periodic, intermediate, core)
    (4, 2, 2, True, False, 0),
    (6, 3, 3, True, True, 2),
    (7, 3, 2, False, True, 6),
    (8, 4, 4, True, False, 0),
    (8, 4, 4, True, True, 0),
    (10, 5, 5, True, True, 3),
    (11, 6, 5, True, False, 0),
]


def _oracle_op(L, nu, nd, periodic, inter, core):
    sec = hubbard.Sector(L, nu + (1 if inter else 0), nd)
    return hubbard.hamiltonian(sec, 1.0, 8.0, 4.0, core if inter else None, periodic)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_hubbard_apply_matches_oracle(cuda, case, prec):
    from paper_2506_09551_gb300 import api
    L, nu, nd, periodic, inter, core = case
    m = api.model(L, nu, nd, core_site=core, periodic=periodic)
    op = api.Operator.hubbard(m, inter)
    H = _oracle_op(*case)
    assert op.dim == H.shape[0]
    X = workloads.random_complex_vectors(op.dim, 3, seed=L)
    c0 = -1.7 - 0.3j
    ref = (H @ X.T).T + c0 * X
    x = torch.tensor(X, dtype=api.cdtype(prec), device="cuda")
    y = op.apply(x, c0, prec).cpu().numpy()
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err <= (1e-15 if prec == 0 else 2e-7), err


def test_csr_apply_matches_scipy(cuda):
    from paper_2506_09551_gb300 import api
    rowptr, col, val = workloads.random_symmetric_csr(5003, 8, seed=9)
    A = sp.csr_matrix((val, col, rowptr), shape=(5003, 5003))
    op = api.Operator.csr(rowptr, col, val)
    X = workloads.random_complex_vectors(5003, 2, seed=3)
    c0 = 0.25 + 0.3j
    y = op.apply(torch.tensor(X, device="cuda"), c0).cpu().numpy()
    ref = (A @ X.T).T + c0 * X
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-15


@pytest.mark.parametrize("L,nu,nd,site", [(4, 2, 2, 0), (6, 3, 3, 4), (8, 4, 4, 7), (9, 4, 5, 3)])
def test_sector_maps_are_exact(cuda, L, nu, nd, site):
    from paper_2506_09551_gb300 import api
    om = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, site)
    m = api.model(L, nu, nd, core_site=site)
    D, Dp = om.gsec.dim, om.isec.dim
    X = workloads.random_complex_vectors(D, 2, seed=1)
    y = api.apply_cdag_up(m, site, torch.tensor(X, device="cuda"), Dp).cpu().numpy()
    assert np.array_equal(y, (om.O2 @ X.T).T)          # +-1 entries: bit-exact
    Xp = workloads.random_complex_vectors(Dp, 2, seed=2)
    z = api.apply_c_up(m, site, torch.tensor(Xp, device="cuda"), D).cpu().numpy()
    assert np.array_equal(z, (om.O1 @ Xp.T).T)
