"""Pins of the oracle's second step and of the whole map (Eqs. 1-2) against full
diagonalisation, closed forms, limits and symmetries."""
import numpy as np
import pytest

from oracle import hubbard, rixs, solvers, spectrum
from workloads import tiny

W_IN = np.linspace(-4, 12, 9)
W = np.linspace(-1, 10, 25)


def _map(L, nu, nd, j=0, **kw):
    return rixs.rixs_map(L, nu, nd, 1.0, 8.0, 4.0, j, 0.3, 0.1, W_IN, W, **kw)


def test_cf_matches_direct_solves():
    m = hubbard.RixsModel(6, 3, 3, 1.0, 8.0, 4.0, 0)
    res = _map(6, 3, 3, model=m)
    for k in (0, 3, 6):
        I_cf, depth = spectrum.lanczos_cf(m.H, res.phi[k], res.E_G, W, 0.1)
        I_d = spectrum.direct_second_step(m.H, res.phi[k], res.E_G, W, 0.1)
        assert np.max(np.abs(I_cf - I_d)) <= 1e-11 * np.max(np.abs(I_d))


@pytest.mark.parametrize("L,nu,nd,periodic", [(4, 2, 2, True), (6, 3, 3, True), (5, 3, 2, False)])
def test_whole_map_vs_lehmann_sum(L, nu, nd, periodic):
    m = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, 0, periodic)
    res = _map(L, nu, nd, model=m, periodic=periodic)
    I_l = spectrum.lehmann_map(m.H, m.Hp, m.O2, m.O1, res.G, res.E_G, W_IN, W, 0.3, 0.1)
    assert rixs.relative_l2(res.I, I_l) <= 1e-11


def test_planted_missing_core_hole_is_caught():
    """Planted mistake: dropping the core-hole term of Eq. (10) from H' moves the
    resonance; the Lehmann comparison with the right H' then fails."""
    m = hubbard.RixsModel(4, 2, 2, 1.0, 8.0, 4.0, 0)
    bad = hubbard.RixsModel(4, 2, 2, 1.0, 8.0, 0.0, 0)
    res = _map(4, 2, 2, model=bad)
    I_l = spectrum.lehmann_map(m.H, m.Hp, m.O2, m.O1, res.G, res.E_G, W_IN, W, 0.3, 0.1)
    assert rixs.relative_l2(res.I, I_l) > 1e-2


@pytest.mark.parametrize("L,nu", [(4, 2), (6, 3)])
def test_atomic_limit_closed_form(L, nu):
    """t = 0 at half filling: I = (1/pi) w / |U - 2Uc - w_in - i Gamma|^2 * eta / (w^2 + eta^2),
    w = ||c^dag_{j,up} G||^2, for any G in the singly-occupied ground manifold (E_G = 0)."""
    U, Uc, Gamma, eta = 8.0, 4.0, 0.3, 0.1
    m = hubbard.RixsModel(L, nu, nu, 0.0, U, Uc, 1)
    sec = m.gsec
    mask = ((sec.u & sec.d) == 0) & ((sec.u | sec.d) == (1 << L) - 1)
    G = np.where(mask, np.random.default_rng(4).standard_normal(sec.dim), 0.0)
    G /= np.linalg.norm(G)
    res = rixs.rixs_map(L, nu, nu, 0.0, U, Uc, 1, Gamma, eta, W_IN, W, G=G, E_G=0.0, model=m)
    wgt = np.linalg.norm(m.O2 @ G) ** 2
    ref = (wgt / np.abs(U - 2 * Uc - W_IN - 1j * Gamma) ** 2)[:, None] * (eta / (W ** 2 + eta ** 2))[None, :] / np.pi
    assert rixs.relative_l2(res.I, ref) <= 1e-13


def test_kubo_limit():
    """Gamma -> infinity: Gamma^2 I(w_in, w) -> (1/pi) Im <G|O2^dag O1^dag R(w) O1 O2|G>,
    the two-point spectrum of O1 O2.  The O(1/Gamma) term of the expansion of Eq. (2)
    is real and drops out of Im, so the deviation falls like 1/Gamma^2."""
    m = hubbard.RixsModel(4, 2, 2, 1.0, 8.0, 4.0, 0)
    E_G, G, _ = solvers.ground_state(m.H, np.random.default_rng(1).standard_normal(m.H.shape[0]))
    S, _ = spectrum.lanczos_cf(m.H, m.O1 @ (m.O2 @ G), E_G, W, 0.1)
    errs = []
    for Gamma in (1e2, 1e3, 1e4):
        res = rixs.rixs_map(4, 2, 2, 1.0, 8.0, 4.0, 0, Gamma, 0.1, np.array([0.0, 3.0]), W,
                            G=G, E_G=E_G, model=m)
        errs.append(np.max(np.abs(Gamma ** 2 * res.I - S[None, :])) / np.max(S))
    assert errs[2] < 1e-6
    assert 50 < errs[0] / errs[1] < 200 and 50 < errs[1] / errs[2] < 200


def test_nonnegative_and_sum_rule():
    m = hubbard.RixsModel(6, 3, 3, 1.0, 8.0, 4.0, 0)
    w = np.arange(-60.0, 90.0, 0.005)
    res = rixs.rixs_map(6, 3, 3, 1.0, 8.0, 4.0, 0, 0.3, 0.1, np.array([-2.0, 0.0, 5.0]), w, model=m)
    assert res.I.min() >= -1e-14 * res.I.max()
    for k in range(3):
        integral = np.sum(res.I[k]) * 0.005
        n2 = np.linalg.norm(res.phi[k]) ** 2
        assert abs(integral - n2) <= 2e-3 * n2


def test_translation_invariance_of_core_site():
    maps = [_map(6, 3, 3, j=j).I for j in range(6)]
    for I in maps[1:]:
        assert rixs.relative_l2(I, maps[0]) <= 1e-10


def test_spin_symmetry_and_ordering_independence():
    ref = _map(6, 3, 3).I
    assert rixs.relative_l2(_map(6, 3, 3, spin=1).I, ref) <= 1e-10
    assert rixs.relative_l2(_map(6, 3, 3, order="site-major").I, ref) <= 1e-10
    assert rixs.relative_l2(_map(6, 3, 3, order="site-major", spin=1).I, ref) <= 1e-10
