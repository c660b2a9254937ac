"""Pins of the oracle's spin channels and 2D clusters (Sec. III's channels and lattices at
sizes that fit): the U = 0 spectrum of a periodic 2D cluster with diagonal hopping against
its single-particle levels, and the spin-flip and 2D maps against the Kramers-Heisenberg
sum by full diagonalisation."""
from itertools import combinations

import numpy as np
import pytest

from oracle import hubbard, rixs, spectrum

W_IN = np.linspace(-4, 12, 7)
W = np.linspace(-1, 10, 25)


def _single_particle_levels(L, lx, t, tp):
    """Eigenvalues of the one-body hopping matrix of the periodic lx x (L / lx) cluster,
    built here from the lattice geometry alone (plane waves: eps(k) = -2t(cos kx + cos ky)
    - 2t'(cos(kx + ky) + cos(kx - ky)))."""
    ly = L // lx
    eps = []
    for mx in range(lx):
        for my in range(ly):
            kx, ky = 2 * np.pi * mx / lx, 2 * np.pi * my / ly
            eps.append(-2 * t * (np.cos(kx) + np.cos(ky)) - 2 * tp * (np.cos(kx + ky) + np.cos(kx - ky)))
    return np.array(eps)


@pytest.mark.parametrize("lx,L,nu,nd,tp", [(3, 9, 2, 1, -0.3), (3, 9, 2, 2, 0.0), (3, 12, 1, 2, 0.25)])
def test_2d_u0_spectrum_matches_single_particle_sums(lx, L, nu, nd, tp):
    bl = hubbard.cluster_bonds(L, True, 1.0, lx, tp)
    sec = hubbard.Sector(L, nu, nd)
    H = hubbard.hamiltonian(sec, 1.0, 0.0, bond_list=bl)
    ev = np.linalg.eigvalsh(H.toarray())
    eps = _single_particle_levels(L, lx, 1.0, tp)
    up = [sum(eps[list(c)]) for c in combinations(range(L), nu)]
    dn = [sum(eps[list(c)]) for c in combinations(range(L), nd)]
    ref = np.sort(np.add.outer(up, dn).ravel())
    assert np.allclose(ev, ref, atol=1e-11)
    # and the Kronecker assembly agrees with the generic one on the same bonds
    assert abs(hubbard.hamiltonian_kron(sec, 1.0, 0.0, bond_list=bl) - H).max() == 0.0


def test_2d_bond_count_and_rejections():
    assert len(hubbard.cluster_bonds(12, True, 1.0, 3, 0.0)) == 24
    assert len(hubbard.cluster_bonds(12, True, 1.0, 3, -0.2)) == 48
    with pytest.raises(ValueError):
        hubbard.cluster_bonds(8, True, 1.0, 2, 0.0)       # a 2 x 4 torus doubles its bonds


@pytest.mark.parametrize("L,nu,nd,spin,spin_out,lx,tp", [
    (4, 2, 2, 1, 0, 0, 0.0),       # spin flip: c^dag_{down} in, c_{up} out
    (6, 3, 3, 0, 1, 0, 0.0),       # spin flip: c^dag_{up} in, c_{down} out
    (5, 2, 3, 1, 1, 0, 0.0),       # spin-conserving, down channel
    (9, 2, 1, 0, 0, 3, -0.3),      # 3 x 3 cluster with diagonal hopping
    (9, 1, 2, 0, 1, 3, 0.2),       # spin flip on the 3 x 3 cluster
])
def test_channel_maps_vs_lehmann_sum(L, nu, nd, spin, spin_out, lx, tp):
    m = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, 1, True, spin=spin, spin_out=spin_out, lx=lx, tp=tp)
    res = rixs.rixs_map(L, nu, nd, 1.0, 8.0, 4.0, 1, 0.3, 0.1, W_IN, W, model=m)
    I_l = spectrum.lehmann_map(m.Hf, m.Hp, m.O2, m.O1, res.G, res.E_G, W_IN, W, 0.3, 0.1)
    assert rixs.relative_l2(res.I, I_l) <= 1e-10
    if spin != spin_out:
        assert (m.fsec.n_up, m.fsec.n_dn) != (nu, nd)


def test_spin_flip_final_sector_and_planted_wrong_sector():
    """The spin-flip final states carry one spin_out electron fewer and one spin electron
    more than the ground state; evaluating the second step with the ground-sector H
    instead (a planted mistake) cannot even be formed for N_up != N_dn and gives a
    different map when the sectors happen to have equal size."""
    m = hubbard.RixsModel(6, 3, 2, 1.0, 8.0, 4.0, 0, True, spin=1, spin_out=0)
    assert (m.fsec.n_up, m.fsec.n_dn) == (2, 3)
    res = rixs.rixs_map(6, 3, 2, 1.0, 8.0, 4.0, 0, 0.3, 0.1, W_IN, W, model=m)
    assert res.I.min() >= -1e-12 * res.I.max()
    # sum rule over a wide window: the weight is ||phi||^2
    wide = np.linspace(-40, 80, 6001)
    I_w, _ = spectrum.lanczos_cf(m.Hf, res.phi[3], res.E_G, wide, 0.1)
    integral = np.sum(I_w) * (wide[1] - wide[0])
    assert abs(integral - np.vdot(res.phi[3], res.phi[3]).real) <= 5e-3 * np.vdot(res.phi[3], res.phi[3]).real
