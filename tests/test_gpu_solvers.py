"""GPU parity of the ground state and of the multi-shift solve against the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import hubbard, solvers
import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,nu,nd", [(6, 3, 3), (8, 4, 4), (10, 5, 5)])
def test_ground_state(cuda, L, nu, nd):
    from paper_2506_09551_gb300 import api
    om = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, 0)
    E_o, G_o, _ = solvers.ground_state(om.H, workloads.lanczos_start(om.H.shape[0], 1))
    op = api.Operator.hubbard(api.model(L, nu, nd))
    E, g, res = op.ground_state(1e-12, 300)
    g = g.cpu().numpy()
    assert abs(E - E_o) <= 1e-12 * abs(E_o)
    assert res <= 1e-12 * max(1, abs(E))
    assert abs(abs(g @ G_o) - 1) <= 1e-11
    # true residual by the oracle's own matrix
    assert np.linalg.norm(om.H @ g - E * g) <= 2e-12 * max(1, abs(E))


def _chain8_problem():
    wl = workloads.CHAIN8
    om = hubbard.RixsModel(wl.L, wl.n_up, wl.n_dn, 1.0, 8.0, 4.0, 0)
    E_G, G, _ = solvers.ground_state(om.H, workloads.lanczos_start(om.H.shape[0], 1))
    return wl, om, E_G, G


@pytest.fixture(scope="module")
def chain8():
    return _chain8_problem()


@pytest.mark.parametrize("block", [1, 2, 4, 8, 16])
def test_multishift_matches_independent_solves(cuda, chain8, block):
    from paper_2506_09551_gb300 import api
    wl, om, E_G, G = chain8
    E = om.O2 @ G
    s0 = workloads.seed_index(wl.w_in)
    shifts = wl.w_in - wl.w_in[s0]
    n = om.Hp.shape[0]
    A = (om.Hp - (E_G + wl.w_in[s0] + 1j * wl.Gamma) * sp.identity(n)).tocsr()
    X_ref, _ = solvers.solve_shifted(A, E, shifts, tol=1e-13)
    op = api.Operator.hubbard(api.model(wl.L, wl.n_up, wl.n_dn), intermediate=True)
    c0 = -E_G - wl.w_in[s0] - 1j * wl.Gamma
    x, per, info, st = op.multishift_solve(torch.tensor(E, dtype=torch.complex128, device="cuda"), shifts, c0,
                                           tol=1e-12, maxit=3000, block=block)
    x = x.cpu().numpy()
    assert st == 0 and per["converged"].all()
    for k in range(len(shifts)):
        err = np.linalg.norm(x[k] - X_ref[k]) / np.linalg.norm(X_ref[k])
        assert err <= 1e-9, (k, err)
        rt = E - (A - shifts[k] * sp.identity(n)) @ x[k]
        assert np.linalg.norm(rt) <= 20 * 1e-12 * np.linalg.norm(E)
    assert info["iterations"] == per["iters"].max()


def test_lagged_update_is_bitwise_identical(cuda, chain8):
    """The lagged per-shift update performs the same operations in the same order."""
    from paper_2506_09551_gb300 import api
    wl, om, E_G, G = chain8
    E = torch.tensor(om.O2 @ G, dtype=torch.complex128, device="cuda")
    op = api.Operator.hubbard(api.model(wl.L, wl.n_up, wl.n_dn), intermediate=True)
    shifts = np.linspace(-4, 12, 17)
    outs = [op.multishift_solve(E, shifts, -E_G - 0.3j, tol=1e-11, block=b)[0].cpu().numpy() for b in (1, 4, 16)]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_mixed_precision_solve(cuda, chain8):
    from paper_2506_09551_gb300 import api
    wl, om, E_G, G = chain8
    E = om.O2 @ G
    n = om.Hp.shape[0]
    shifts = np.array([-4.0, -1.0, 0.0, 2.0, 7.0, 12.0])
    A = (om.Hp - (E_G + 1j * wl.Gamma) * sp.identity(n)).tocsr()
    X_ref, _ = solvers.solve_shifted(A, E, shifts, tol=1e-13)
    op = api.Operator.hubbard(api.model(wl.L, wl.n_up, wl.n_dn), intermediate=True)
    x, per, info, st = op.multishift_solve(torch.tensor(E, device="cuda"), shifts, -E_G - 1j * wl.Gamma,
                                           tol=1e-6, block=8, prec=api.FP32_MIXED)
    assert x.dtype == torch.complex64
    x = x.cpu().numpy().astype(np.complex128)
    for k in range(len(shifts)):
        assert np.linalg.norm(x[k] - X_ref[k]) / np.linalg.norm(X_ref[k]) <= 1e-4


def test_random_complex_symmetric_csr(cuda):
    """Small stand-in of the random stress workload: sigma_k + 0.3i shifts, seed in the middle."""
    from paper_2506_09551_gb300 import api
    n = 4000
    rowptr, col, val = workloads.random_symmetric_csr(n, 8, seed=21)
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    b = workloads.random_complex_rhs(n, seed=22)
    sig = workloads.random_shifts(24, -6, 6, 0.3, seed=23)
    seed = int(np.argsort(sig.real)[len(sig) // 2])
    op = api.Operator.csr(rowptr, col, val)
    x, per, info, st = op.multishift_solve(torch.tensor(b, device="cuda"), sig - sig[seed], -sig[seed],
                                           tol=1e-10, maxit=20000, block=8)
    x = x.cpu().numpy()
    assert per["converged"].all()
    Ac = sp.csc_matrix(A, dtype=np.complex128)
    for k in range(0, 24, 5):
        xr = sp.linalg.spsolve((Ac - sig[k] * sp.identity(n, format="csc")).tocsc(), b)
        assert np.linalg.norm(x[k] - xr) / np.linalg.norm(xr) <= 1e-8


def test_edge_cases(cuda, chain8):
    from paper_2506_09551_gb300 import api, native
    wl, om, E_G, G = chain8
    op = api.Operator.hubbard(api.model(wl.L, wl.n_up, wl.n_dn), intermediate=True)
    n = op.dim
    # zero right-hand side: zero solutions, all converged, no iteration
    x, per, info, st = op.multishift_solve(torch.zeros(n, dtype=torch.complex128, device="cuda"), [0.0, 1.0],
                                           -E_G - 0.3j)
    assert st == 0 and per["converged"].all() and info["iterations"] == 0
    assert torch.count_nonzero(x).item() == 0
    # iteration cap: MSB_EMAXITER, partial results written and finite
    E = torch.tensor(om.O2 @ G, dtype=torch.complex128, device="cuda")
    x, per, info, st = op.multishift_solve(E, [0.0, 3.0], -E_G - 0.3j, tol=1e-14, maxit=5,
                                           allow_status=(native.MSB_EMAXITER,))
    assert st == native.MSB_EMAXITER and info["iterations"] == 5
    assert torch.isfinite(torch.view_as_real(x)).all()
    # a single shift equal to the seed
    x1, per, info, st = op.multishift_solve(E, [0.0], -E_G - 0.3j, tol=1e-12)
    n2 = om.Hp.shape[0]
    A = (om.Hp - (E_G + 0.3j) * sp.identity(n2)).tocsr()
    xr = sp.linalg.spsolve(sp.csc_matrix(A), om.O2 @ G)
    assert np.linalg.norm(x1.cpu().numpy()[0] - xr) / np.linalg.norm(xr) <= 1e-9
    # invalid arguments are rejected before any work
    with pytest.raises(native.MsbError):
        op.multishift_solve(E, [0.0], 0.0, block=3)


def test_atomic_limit_terminates_after_one_step(cuda):
    """t = 0: E = O2 G is an eigenvector of H', so the seed residual vanishes at m = 1."""
    from paper_2506_09551_gb300 import api
    L = 6
    m = api.model(L, 3, 3, t=0.0)
    om = hubbard.RixsModel(L, 3, 3, 0.0, 8.0, 4.0, 0)
    sec = om.gsec
    mask = ((sec.u & sec.d) == 0) & ((sec.u | sec.d) == (1 << L) - 1)
    G = np.where(mask, workloads.lanczos_start(sec.dim, 4), 0.0)
    G /= np.linalg.norm(G)
    E = torch.tensor(om.O2 @ G, dtype=torch.complex128, device="cuda")
    op = api.Operator.hubbard(m, intermediate=True)
    x, per, info, st = op.multishift_solve(E, np.linspace(-4, 12, 9), -0.3j, tol=1e-12)
    assert info["iterations"] <= 2
    lam = 8.0 - 2 * 4.0 - 0.3j - np.linspace(-4, 12, 9)
    ref = (om.O2 @ G)[None, :] / lam[:, None]
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
