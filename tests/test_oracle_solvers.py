"""Pins of the oracle's ground state and shifted solvers (Sec. III, App. A-D)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hubbard, solvers


def _model(L=6, nu=3, nd=3, j=0):
    return hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, core_site=j)


@pytest.mark.parametrize("L,nu,nd,periodic", [(4, 2, 2, True), (6, 3, 3, True), (5, 3, 2, False),
                                              (8, 4, 4, True)])
def test_ground_state_vs_dense(L, nu, nd, periodic):
    m = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, 0, periodic)
    E, G, res = solvers.ground_state(m.H, np.random.default_rng(1).standard_normal(m.H.shape[0]))
    ev, V = np.linalg.eigh(m.H.toarray())
    assert ev[1] - ev[0] > 1e-6                       # unique ground state
    assert abs(E - ev[0]) <= 1e-12 * max(1, abs(ev[0]))
    assert abs(abs(G @ V[:, 0]) - 1) < 1e-12
    assert res <= 1e-12 * max(1, abs(E))


def test_ground_state_dimer_closed_form():
    sec = hubbard.Sector(2, 1, 1)
    H = hubbard.hamiltonian(sec, 1.0, 8.0, periodic=False)
    E, G, _ = solvers.ground_state(H, np.array([1.0, 0.3, -0.2, 0.5]))
    assert abs(E - (4 - np.sqrt(16 + 4))) < 1e-13


def _shifted_problem(L=6, nu=3, nd=3, Gamma=0.3):
    m = _model(L, nu, nd)
    E_G, G, _ = solvers.ground_state(m.H, np.random.default_rng(1).standard_normal(m.H.shape[0]))
    n = m.Hp.shape[0]
    A = (m.Hp - E_G * sp.identity(n) - 1j * Gamma * sp.identity(n)).tocsr()
    return A, m.O2 @ G


def test_lu_bicgstab_dense_agree():
    A, b = _shifted_problem()
    shifts = np.linspace(-4, 12, 7)
    Xl, _ = solvers.solve_shifted(A, b, shifts, method="lu")
    Xb, nmv = solvers.solve_shifted(A, b, shifts, tol=1e-13, method="bicgstab")
    Ad = A.toarray()
    for k, s in enumerate(shifts):
        xd = np.linalg.solve(Ad - s * np.eye(len(b)), b)
        assert np.linalg.norm(Xl[k] - xd) <= 1e-12 * np.linalg.norm(xd)
        assert np.linalg.norm(Xb[k] - xd) <= 1e-10 * np.linalg.norm(xd)
    assert nmv > 0


def _random_complex_symmetric(n, seed, Gamma=0.3):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    H = (M + M.T) / 2
    return H - 1j * Gamma * np.eye(n), rng.standard_normal(n)


@pytest.mark.parametrize("case", ["hubbard", "random"])
def test_msbicg_matches_independent_solves(case):
    if case == "hubbard":
        A, b = _shifted_problem()
        A = A.toarray()
    else:
        A, b = _random_complex_symmetric(60, 7)
    shifts = np.array([-3.0, -0.5, 0.0, 0.7, 2.5, 6.0, 11.0])
    out = solvers.msbicg(A, b, shifts, tol=1e-12, maxit=2000)
    assert out["converged"].all()
    for k, s in enumerate(shifts):
        xd = np.linalg.solve(A - s * np.eye(len(b)), b)
        assert np.linalg.norm(out["x"][k] - xd) <= 1e-9 * np.linalg.norm(xd), k
        # true residual of every shift, by an independent product
        rt = b - (A - s * np.eye(len(b))) @ out["x"][k]
        assert np.linalg.norm(rt) <= 10 * 1e-12 * np.linalg.norm(b)


def test_paper_printed_zeta_sign_is_wrong():
    """Planted mistake: Eq. (5)/(C8) as printed, (1 + alpha s), solves (A + sI) instead."""
    A, b = _random_complex_symmetric(60, 7)
    shifts = np.array([-2.0, 1.5, 4.0])
    out = solvers.msbicg(A, b, shifts, tol=1e-12, maxit=400, zeta_sign=+1.0)
    errs = [np.linalg.norm(out["x"][k] - np.linalg.solve(A - s * np.eye(60), b)) for k, s in enumerate(shifts)]
    assert max(errs) > 1e-3 * np.linalg.norm(np.linalg.solve(A - shifts[0] * np.eye(60), b))
    # ... and what it does solve is the system with the opposite shift
    for k, s in enumerate(shifts):
        x_plus = np.linalg.solve(A + s * np.eye(60), b)
        if out["converged"][k]:
            assert np.linalg.norm(out["x"][k] - x_plus) <= 1e-8 * np.linalg.norm(x_plus)


def test_hermitian_product_is_wrong():
    """Planted mistake: conjugated products in alpha/beta break the Galerkin condition."""
    A, b = _random_complex_symmetric(60, 11)
    b = b + 0.5j * np.random.default_rng(3).standard_normal(60)   # complex RHS
    shifts = np.array([0.0, 2.0])
    out = solvers.msbicg(A, b, shifts, tol=1e-12, maxit=120, product="hermitian")
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(out["x"][0] - xd) > 1e-4 * np.linalg.norm(xd)


@pytest.mark.parametrize("m_stop", [1, 3, 8, 20])
def test_residual_collinearity(m_stop):
    """Eq. (4)/(B4): the true residual of each shifted system equals r_m / zeta_m."""
    A, b = _random_complex_symmetric(50, 5)
    shifts = np.array([-1.0, 0.4, 3.0])
    out = solvers.msbicg(A, b, shifts, tol=0.0, maxit=m_stop)
    for k, s in enumerate(shifts):
        rt = b - (A - s * np.eye(50)) @ out["x"][k]
        assert np.linalg.norm(rt - out["r"] / out["zeta"][k]) <= 1e-10 * np.linalg.norm(b)


def test_residual_polynomial_identities():
    """Eq. (C1): r_m = P_m(A) r_0, and Eq. (C3): zeta_m = P_m(s), with P_m built by the
    three-term recurrence (C6-C7) from the seed's alpha/beta."""
    A, b = _random_complex_symmetric(40, 9)
    s = 1.7
    M = 12
    out = solvers.msbicg(A, b, np.array([s]), tol=0.0, maxit=M, record=True)
    h = out["hist"]
    # matrix polynomial P_M(A) b by the same three-term recurrence, on vectors
    Pp, P = b.copy(), b.copy()
    a_prev = 1.0
    for k in range(M):
        bk = h["beta"][k - 1] if k > 0 else 0.0
        c = h["alpha"][k] * bk / a_prev
        Pp, P = P, -h["alpha"][k] * (A @ P) + (1 + c) * P - c * Pp
        a_prev = h["alpha"][k]
    assert np.linalg.norm(P - out["r"]) <= 1e-9 * np.linalg.norm(b)
    z = solvers.residual_polynomial(h["alpha"], h["beta"], s, M)
    assert abs(z - out["zeta"][0]) <= 1e-9 * abs(z)


def test_dual_residual_is_conjugate():
    """App. A: for A = H' - E_G - i Gamma with H' real symmetric and E real, the dual
    residual of full BiCG equals conj(r_m), so no A^dagger products are needed."""
    A, b = _random_complex_symmetric(30, 4)
    R, RT = solvers.dual_bicg(A, b, 15)
    for r, rt in zip(R, RT):
        assert np.linalg.norm(rt - np.conj(r)) <= 1e-9 * np.linalg.norm(b)
    # ... and it does not hold for a complex non-symmetric matrix
    rng = np.random.default_rng(2)
    B = rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))
    R, RT = solvers.dual_bicg(B, b, 5)
    assert np.linalg.norm(RT[3] - np.conj(R[3])) > 1e-3 * np.linalg.norm(b)


@pytest.mark.parametrize("n", [8, 20, 36])
def test_finite_termination(n):
    """At most n steps solve an n x n system exactly (up to rounding)."""
    A, b = _random_complex_symmetric(n, 100 + n, Gamma=2.0)
    shifts = np.array([-1.0, 0.5, 2.0])
    out = solvers.msbicg(A, b, shifts, tol=1e-13, maxit=3 * n)
    for k, s in enumerate(shifts):
        xd = np.linalg.solve(A - s * np.eye(n), b)
        assert np.linalg.norm(out["x"][k] - xd) <= 1e-8 * np.linalg.norm(xd)


def test_two_by_two_toy_collinearity():
    """Fig. 2(c): after one step the CG/BiCG residuals of different shifts are collinear
    (all orthogonal to r_0 in 2D); the MINRES residuals are not."""
    A = np.array([[2.0, 0.6], [0.6, 1.0]])
    b = np.array([1.0, 0.3])
    res_cg, res_mr = [], []
    for s in (0.0, -0.5, 0.7):
        As = A - s * np.eye(2)
        out = solvers.msbicg(As, b, np.array([0.0]), tol=0.0, maxit=1)
        res_cg.append(b - As @ out["x"][0].real)
        v = As @ b
        res_mr.append(b - (v @ b) / (v @ v) * v)         # one MINRES step: min ||b - g A b||
    cross = lambda u, v: (u[0] * v[1] - u[1] * v[0]) / (np.linalg.norm(u) * np.linalg.norm(v))
    assert all(abs(cross(res_cg[0], r)) < 1e-13 for r in res_cg[1:])
    assert any(abs(cross(res_mr[0], r)) > 1e-3 for r in res_mr[1:])
