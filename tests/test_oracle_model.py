"""Pins of the oracle's Hubbard model (Eqs. 9-10) against closed forms and invariants."""
from itertools import combinations
from math import comb

import numpy as np
import pytest

from oracle import hubbard


@pytest.mark.parametrize("L,n", [(4, 2), (6, 3), (8, 4), (12, 6), (14, 8)])
def test_sector_enumeration(L, n):
    s = hubbard.sector_states(L, n)
    assert len(s) == comb(L, n)
    assert np.all(np.diff(s) > 0)
    # brute force over subsets
    ref = sorted(sum(1 << i for i in c) for c in combinations(range(L), n))
    assert np.array_equal(s, np.array(ref))


def test_popcount_table():
    x = np.array([0, 1, 3, 0xFF, (1 << 40) - 1, 0x5555_5555_5555], dtype=np.int64)
    assert hubbard.popcount(x).tolist() == [bin(int(v)).count("1") for v in x]


@pytest.mark.parametrize("order", ["up-first", "site-major"])
@pytest.mark.parametrize("L,nu,nd,periodic", [(4, 2, 2, True), (6, 3, 2, True), (5, 2, 3, False)])
def test_hamiltonian_symmetric(order, L, nu, nd, periodic):
    sec = hubbard.Sector(L, nu, nd, order)
    H = hubbard.hamiltonian(sec, 1.0, 8.0, 4.0, 0, periodic)
    assert abs(H - H.T).max() == 0.0
    # hop entries are exactly -t * (+-1)
    off = H - hubbard.sp.diags(H.diagonal())
    assert set(np.unique(np.abs(off.data)).tolist()) <= {1.0}


def _free_fermion_levels(L, n_up, n_dn, t, periodic):
    """Many-body U=0 spectrum as sums of single-particle energies.

    Periodic ring of true fermions: eps_k = -2t cos(2 pi m / L).  Open chain:
    eps_k = -2t cos(pi m / (L + 1)), m = 1..L.  (Textbook tight binding.)"""
    if periodic:
        eps = -2 * t * np.cos(2 * np.pi * np.arange(L) / L)
    else:
        eps = -2 * t * np.cos(np.pi * np.arange(1, L + 1) / (L + 1))
    up = [sum(eps[list(c)]) for c in combinations(range(L), n_up)]
    dn = [sum(eps[list(c)]) for c in combinations(range(L), n_dn)]
    return np.sort(np.add.outer(up, dn).ravel())


@pytest.mark.parametrize("order", ["up-first", "site-major"])
@pytest.mark.parametrize("L,nu,nd,periodic", [(4, 2, 2, True), (6, 2, 3, True), (6, 4, 3, True),
                                              (5, 2, 2, False)])
def test_u0_spectrum_matches_single_particle_sums(order, L, nu, nd, periodic):
    """Even N_sigma on the ring exercises the boundary Jordan-Wigner sign."""
    sec = hubbard.Sector(L, nu, nd, order)
    H = hubbard.hamiltonian(sec, 1.0, 0.0, periodic=periodic)
    ev = np.linalg.eigvalsh(H.toarray())
    ref = _free_fermion_levels(L, nu, nd, 1.0, periodic)
    assert np.allclose(ev, ref, atol=1e-12)


def test_wrong_boundary_sign_is_caught():
    """Planted mistake: dropping the boundary JW sign (treating fermions as hard-core
    bosons) changes the U=0 spectrum at even filling, so the pin above would fail."""
    sec = hubbard.Sector(4, 2, 2)
    H = hubbard.hamiltonian(sec, 1.0, 0.0).toarray()
    off = H - np.diag(np.diag(H))
    Hb = -np.abs(off) + np.diag(np.diag(H))     # every hop amplitude -t: bosonic signs
    ref = _free_fermion_levels(4, 2, 2, 1.0, True)
    assert not np.allclose(np.linalg.eigvalsh(Hb), ref, atol=1e-6)


@pytest.mark.parametrize("U", [0.0, 2.0, 8.0])
def test_two_site_closed_form(U):
    """Hubbard dimer at half filling: E_0 = U/2 - sqrt(U^2/4 + 4 t^2) (textbook)."""
    sec = hubbard.Sector(2, 1, 1)
    H = hubbard.hamiltonian(sec, 1.0, U, periodic=False)
    ev = np.linalg.eigvalsh(H.toarray())
    assert abs(ev[0] - (U / 2 - np.sqrt(U * U / 4 + 4.0))) < 1e-13
    # full dimer spectrum: {E_-, 0, U, E_+}
    ref = np.sort([U / 2 - np.sqrt(U * U / 4 + 4), 0.0, U, U / 2 + np.sqrt(U * U / 4 + 4)])
    assert np.allclose(ev, ref, atol=1e-13)


def test_core_hole_diagonal():
    """H' - H is -Uc (n_{j,up} + n_{j,dn}) on the intermediate sector (Eq. 10)."""
    sec = hubbard.Sector(6, 4, 3)
    H = hubbard.hamiltonian(sec, 1.0, 8.0).toarray()
    Hp = hubbard.hamiltonian(sec, 1.0, 8.0, 4.0, 2).toarray()
    d = Hp - H
    assert np.count_nonzero(d - np.diag(np.diag(d))) == 0
    ref = -4.0 * (sec.occupation(2, 0) + sec.occupation(2, 1))
    assert np.array_equal(np.diag(d), ref)


@pytest.mark.parametrize("order", ["up-first", "site-major"])
def test_o1_is_o2_transpose_and_anticommutator(order):
    m = hubbard.RixsModel(6, 3, 3, 1.0, 8.0, 4.0, core_site=3, order=order)
    assert abs(m.O1 - m.O2.T).max() == 0.0
    # {c, c^dag} = 1 on the ground sector: c c^dag + c^dag c, via the N_up-1 sector
    lower = hubbard.Sector(6, 2, 3, order)
    mid = hubbard.Sector(6, 3, 3, order)
    c_dn_to = hubbard.annihilation_operator(mid, lower, 3, 0)
    cd_back = hubbard.creation_operator(lower, mid, 3, 0)
    anti = (m.O1 @ m.O2 + cd_back @ c_dn_to).toarray()
    assert np.allclose(anti, np.eye(mid.dim))


@pytest.mark.parametrize("L,nu,nd,core,periodic", [(8, 4, 4, None, True), (8, 5, 4, 0, True),
                                                   (7, 3, 2, 2, False), (9, 5, 4, 4, True), (6, 0, 3, None, True)])
def test_kronecker_form_equals_generic_construction(L, nu, nd, core, periodic):
    """hamiltonian_kron (per-species hop matrices in a Kronecker sum, used for the large
    sectors of the full-size parity tests) equals the generic Jordan-Wigner construction
    entry by entry, with and without the core hole, on rings and open chains."""
    sec = hubbard.Sector(L, nu, nd)
    A = hubbard.hamiltonian(sec, 1.0, 8.0, 4.0, core, periodic)
    B = hubbard.hamiltonian_kron(sec, 1.0, 8.0, 4.0, core, periodic)
    assert A.shape == B.shape and A.nnz == B.nnz
    assert abs(A - B).max() == 0.0


@pytest.mark.parametrize("L,nu,nd,flux", [(5, 2, 2, 0.7), (6, 3, 2, 2.1), (4, 1, 2, -1.3)])
def test_flux_hamiltonian_is_hermitian_with_twisted_u0_spectrum(L, nu, nd, flux):
    """Peierls phases (a flux through the ring): H is complex Hermitian, and at U = 0 its
    levels are sums of the twisted single-particle energies -2t cos(2 pi m / L + flux / L)."""
    sec = hubbard.Sector(L, nu, nd)
    H = hubbard.hamiltonian(sec, 1.0, 0.0, flux=flux).toarray()
    assert np.iscomplexobj(H) and np.abs(H.imag).max() > 0
    assert np.allclose(H, H.conj().T, atol=1e-14)
    eps = -2.0 * np.cos(2 * np.pi * np.arange(L) / L + flux / L)
    up = [sum(eps[list(c)]) for c in combinations(range(L), nu)]
    dn = [sum(eps[list(c)]) for c in combinations(range(L), nd)]
    assert np.allclose(np.linalg.eigvalsh(H), np.sort(np.add.outer(up, dn).ravel()), atol=1e-11)


def test_flux_on_an_open_chain_is_a_gauge():
    """On an open chain the phases can be gauged away: the spectrum does not depend on them."""
    sec = hubbard.Sector(5, 2, 2)
    H0 = hubbard.hamiltonian(sec, 1.0, 8.0, periodic=False).toarray()
    H1 = hubbard.hamiltonian(sec, 1.0, 8.0, periodic=False, flux=1.9).toarray()
    assert np.allclose(np.linalg.eigvalsh(H0), np.linalg.eigvalsh(H1), atol=1e-12)
