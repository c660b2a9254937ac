"""Pins of the oracle's adaptive reseeding (App. E) against independent solves."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import hubbard, solvers
import workloads


def _system():
    """A = H' - E_G - i Gamma of the L = 6 ring and b = O2 |G> (the map's seed system)."""
    om = hubbard.RixsModel(6, 3, 3, 1.0, 8.0, 4.0, 0, True)
    E_G, G, _ = solvers.ground_state(om.H, workloads.lanczos_start(om.H.shape[0], 1))
    n = om.Hp.shape[0]
    A = (om.Hp - (E_G + 0.3j) * sp.identity(n)).tocsr()
    return A, (om.O2 @ G).astype(np.complex128)


def _direct(A, b, shifts):
    n = A.shape[0]
    return np.array([spla.spsolve((A - s * sp.identity(n)).tocsc(), b) for s in shifts])


SHIFTS = np.linspace(-4.0, 12.0, 17)


def test_no_reseed_on_an_accurate_run():
    A, b = _system()
    out = solvers.msbicg_reseeded(A, b, SHIFTS, 1e-10, 2000, reseed_tol=1e-8, seed_index=4)
    assert out["seeds"] == [4] and out["accepted"].all()
    ref = solvers.msbicg(lambda v: A @ v - SHIFTS[4] * v, b, SHIFTS - SHIFTS[4], 1e-10, 2000)
    assert np.array_equal(out["x"], ref["x"])
    assert np.max(out["dr"]) <= 1e-8 * np.linalg.norm(b)


def test_planted_round_off_is_detected_and_repaired():
    """Round-off planted in the shifted recursions (growing with the distance from the
    seed) leaves far shifts with small recursive but large true residuals: single-seed
    MSBiCG gets them wrong, the Delta r test rejects them, and reseeding solves them."""
    A, b = _system()
    nb = np.linalg.norm(b)
    ref = _direct(A, b, SHIFTS)
    kw = dict(zeta_noise=1e-7, noise_seed=3)
    reseed_tol = 1e-6

    def true_res(x):
        return np.array([np.linalg.norm(b - (A @ x[k] - s * x[k])) for k, s in enumerate(SHIFTS)]) / nb

    single = solvers.msbicg(lambda v: A @ v - SHIFTS[0] * v, b, SHIFTS - SHIFTS[0], 1e-10, 2000, **kw)
    assert single["converged"].all()                     # the recursive residuals look fine ...
    assert true_res(single["x"]).max() > 2 * reseed_tol   # ... but the solutions are not
    out = solvers.msbicg_reseeded(A, b, SHIFTS, 1e-10, 2000, reseed_tol=reseed_tol, seed_index=0,
                                  max_seeds=17, **kw)
    assert out["accepted"].all()
    assert 2 <= len(out["seeds"]) < len(SHIFTS)           # targeted, not one seed per shift
    assert true_res(out["x"]).max() <= 1.01 * (reseed_tol + 1e-10)
    err = np.linalg.norm(out["x"] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    err_single = np.linalg.norm(single["x"] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < err_single.max()
    # each new seed is a shift rejected by the previous run, the one nearest its seed
    for (s_prev, solved), s_next in zip(out["runs"][:-1], out["seeds"][1:]):
        assert s_next in solved and s_next != s_prev


def test_unconverged_shifts_are_reseeded():
    A, b = _system()
    out = solvers.msbicg_reseeded(A, b, SHIFTS, 1e-10, 25, reseed_tol=1e-8, seed_index=0, max_seeds=17)
    assert len(out["seeds"]) >= 2
    ref = _direct(A, b, SHIFTS)
    acc = out["accepted"]
    assert acc.any()
    err = np.linalg.norm(out["x"][acc] - ref[acc], axis=1) / np.linalg.norm(ref[acc], axis=1)
    assert err.max() <= 1e-7
