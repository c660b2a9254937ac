"""The dual-space multi-shift BiCG (App. A) on the GPU, for a complex Hermitian H: the
Hubbard ring with Peierls phases (a flux through the ring).  Every shift's solution is
checked against the oracle's independent sparse-LU solve of that system."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import hubbard, solvers
import workloads

pytestmark = pytest.mark.gpu

SHIFTS = np.linspace(-4.0, 12.0, 9)


def _flux_system(L, nu, nd, flux, core=0):
    """A = H'(flux) - E0 - i Gamma on the intermediate sector, a seeded complex b."""
    sec = hubbard.Sector(L, nu + 1, nd)
    Hp = hubbard.hamiltonian(sec, 1.0, 8.0, 4.0, core, flux=flux)
    E0 = -3.0
    A = (Hp - (E0 + 0.3j) * sp.identity(Hp.shape[0])).tocsr()
    b = workloads.random_complex_vectors(Hp.shape[0], 1, seed=0xF1)[0]
    return A, b, E0


@pytest.mark.parametrize("L,nu,nd,flux", [(6, 3, 3, 0.9), (7, 2, 3, 2.4), (8, 3, 4, -1.7)])
def test_dual_solve_matches_independent_solves(cuda, L, nu, nd, flux):
    from paper_2506_09551_gb300 import api, native
    A, b, E0 = _flux_system(L, nu, nd, flux)
    assert abs(A - A.T).max() > 1e-3                  # not complex symmetric
    ref, _ = solvers.solve_shifted(A, b, SHIFTS, method="lu")
    op = api.Operator.hubbard(api.model(L, nu, nd, flux=flux), True)
    bt = torch.tensor(b, device="cuda")
    seed = workloads.seed_index(SHIFTS)
    c0 = -(E0 + 0.3j) - SHIFTS[seed]
    x, per, info, st = op.multishift_solve(bt, SHIFTS - SHIFTS[seed], c0=c0, tol=1e-11, maxit=20000, dual=True)
    assert st == 0 and per["converged"].all()
    assert info["matvecs"] == 2 * info["iterations"]
    err = np.linalg.norm(x.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-8, err
    x32, per32, _, st32 = op.multishift_solve(bt, SHIFTS - SHIFTS[seed], c0=c0, tol=1e-7, maxit=20000, dual=True,
                                              prec=api.FP32_MIXED)
    assert per32["converged"].all()
    e32 = np.linalg.norm(x32.cpu().numpy().astype(np.complex128) - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert e32.max() <= 1e-4, e32
    # the bilinear (complex-symmetric) solver refuses this operator
    with pytest.raises(native.MsbError):
        op.multishift_solve(bt, SHIFTS, c0=c0, tol=1e-10)


def test_dual_solve_on_a_real_symmetric_operator_gives_the_same_solutions(cuda):
    from paper_2506_09551_gb300 import api
    A, b, E0 = _flux_system(6, 3, 3, 0.0)
    op = api.Operator.hubbard(api.model(6, 3, 3), True)
    bt = torch.tensor(b, device="cuda")
    c0 = -(E0 + 0.3j)
    xd, _, infod, _ = op.multishift_solve(bt, SHIFTS, c0=c0, tol=1e-11, dual=True)
    xp, _, infop, _ = op.multishift_solve(bt, SHIFTS, c0=c0, tol=1e-11)
    d = np.linalg.norm(xd.cpu().numpy() - xp.cpu().numpy(), axis=1) / np.linalg.norm(xp.cpu().numpy(), axis=1)
    assert d.max() <= 1e-8
    assert infod["matvecs"] == 2 * infod["iterations"] and infop["matvecs"] == infop["iterations"]
