"""Oracle: Hubbard-model Hilbert space and operators (TEST INFRASTRUCTURE ONLY).

What is computed, and where the paper defines it
------------------------------------------------
* Eq. (9): H = -sum_{<ij>,s} t (c^dag_{js} c_{is} + h.c.) + U sum_i n_{i,up} n_{i,dn},
  here on a 1D chain with nearest-neighbour bonds only (periodic or open).
* Eq. (10): H' = H + E_edge sum h h^dag - U_c sum n_{i,s} h h^dag.  The core hole
  sits on the site j where O2 acted, E_edge is absorbed into w_in, so
  H' = H - U_c (n_{j,up} + n_{j,dn}) acting on the (n_up + 1, n_dn) sector.
* Eqs. (1)-(2) with the dipole operators reduced to O2 = c^dag_{j,up} and
  O1 = c_{j,up} (the 2p matrix elements of Sec. III are not given).

The basis is the occupation-number basis of each spin sector: the L-bit strings
with the right popcount in ascending order; a many-body basis state has index
rank(u) * D_dn + rank(d).  Fermionic signs are computed from scratch for every
operator application with the textbook Jordan-Wigner rule
    c_o |n> = (-1)^(number of occupied orbitals ordered before o) |n - o>
over a chosen orbital ordering.  Two orderings are provided: "up-first"
(orbital (i, up) = i, (i, dn) = L + i) and "site-major" ((i, s) = 2 i + s).
The spectrum I(w_in, w) must not depend on the ordering; the tests use that.

Parity: every function here is pinned by tests/test_oracle_model.py (sector
sizes, Hermiticity, the U=0 spectrum against single-particle energies, the
two-site closed form, O1 = O2^T).  hamiltonian_kron, the Kronecker-sum assembly
used for the large sectors (L = 14) of the full-size parity tests, is pinned
there as equal to the generic construction entry by entry.
"""
from __future__ import annotations

from dataclasses import dataclass
from math import comb

import numpy as np
import scipy.sparse as sp


_BYTE_POPCOUNT = np.array([bin(b).count("1") for b in range(256)], dtype=np.int64)


def popcount(a: np.ndarray) -> np.ndarray:
    """Number of set bits of each non-negative int64 entry (byte-table lookup)."""
    a = np.asarray(a, dtype=np.int64)
    out = np.zeros(a.shape, dtype=np.int64)
    for k in range(8):
        out += _BYTE_POPCOUNT[(a >> (8 * k)) & 0xFF]
    return out


def sector_states(L: int, n: int) -> np.ndarray:
    """All L-bit strings with n set bits, ascending (bit i = site i occupied)."""
    if not (0 <= n <= L):
        raise ValueError("need 0 <= n <= L")
    allv = np.arange(1 << L, dtype=np.int64)
    s = allv[popcount(allv) == n]
    assert len(s) == comb(L, n)
    return s


def orbital(L: int, site: int, spin: int, order: str) -> int:
    """Position of orbital (site, spin) in the Jordan-Wigner string; spin 0 = up."""
    if order == "up-first":
        return site + spin * L
    if order == "site-major":
        return 2 * site + spin
    raise ValueError(order)


@dataclass
class Sector:
    """Many-body basis of the (n_up, n_dn) sector of an L-site chain."""
    L: int
    n_up: int
    n_dn: int
    order: str = "up-first"

    def __post_init__(self):
        self.up = sector_states(self.L, self.n_up)
        self.dn = sector_states(self.L, self.n_dn)
        self.D_up, self.D_dn = len(self.up), len(self.dn)
        self.dim = self.D_up * self.D_dn
        # occupation of every basis state, per spin (dim,)
        self.u = np.repeat(self.up, self.D_dn)
        self.d = np.tile(self.dn, self.D_up)
        # full Jordan-Wigner occupation string of each basis state
        self.jw = self._to_jw(self.u, self.d)
        # rank of every L-bit string within its species' sector (-1 if outside)
        self._rank_up = np.full(1 << self.L, -1, dtype=np.int64)
        self._rank_up[self.up] = np.arange(self.D_up)
        self._rank_dn = np.full(1 << self.L, -1, dtype=np.int64)
        self._rank_dn[self.dn] = np.arange(self.D_dn)

    def _to_jw(self, u: np.ndarray, d: np.ndarray) -> np.ndarray:
        out = np.zeros_like(u)
        for i in range(self.L):
            out |= ((u >> i) & 1) << orbital(self.L, i, 0, self.order)
            out |= ((d >> i) & 1) << orbital(self.L, i, 1, self.order)
        return out

    def _from_jw(self, jw: np.ndarray):
        u = np.zeros_like(jw)
        d = np.zeros_like(jw)
        for i in range(self.L):
            u |= ((jw >> orbital(self.L, i, 0, self.order)) & 1) << i
            d |= ((jw >> orbital(self.L, i, 1, self.order)) & 1) << i
        return u, d

    def index_of_jw(self, jw: np.ndarray) -> np.ndarray:
        """Basis index rank(u) * D_dn + rank(d) of each JW string (must lie in the sector)."""
        u, d = self._from_jw(jw)
        iu, idn = self._rank_up[u], self._rank_dn[d]
        if np.any(iu < 0) or np.any(idn < 0):
            raise ValueError("state outside sector")
        return iu * self.D_dn + idn

    def occupation(self, site: int, spin: int) -> np.ndarray:
        occ = self.u if spin == 0 else self.d
        return (occ >> site) & 1


def annihilate(jw: np.ndarray, o: int):
    """c_o on JW strings: returns (mask of states where it acts, sign, new strings)."""
    bit = np.int64(1) << o
    acts = (jw & bit) != 0
    below = jw & (bit - 1)
    sign = np.where(popcount(below) % 2 == 0, 1.0, -1.0)
    return acts, sign, jw ^ bit


def create(jw: np.ndarray, o: int):
    """c^dag_o on JW strings: returns (mask, sign, new strings)."""
    bit = np.int64(1) << o
    acts = (jw & bit) == 0
    below = jw & (bit - 1)
    sign = np.where(popcount(below) % 2 == 0, 1.0, -1.0)
    return acts, sign, jw | bit


def bonds(L: int, periodic: bool):
    """Nearest-neighbour bonds (i, i+1) of the chain; the periodic ring adds (L-1, 0)."""
    if periodic and L < 3:
        raise ValueError("a periodic chain needs L >= 3 (L = 2 would double the bond)")
    nb = L if periodic else L - 1
    return [(i, (i + 1) % L) for i in range(nb)]


def cluster_bonds(L: int, periodic: bool = True, t: float = 1.0, lx: int = 0, tp: float = 0.0):
    """Bonds (i, j, t_ij) of the lattice.  lx = 0: the 1D chain of `bonds` with hopping t.
    lx > 0: the periodic lx x ly cluster (ly = L / lx, site x + lx y) with hopping t on
    the nearest-neighbour bonds and t' = tp on the diagonal (next-nearest) bonds; both
    sides must be at least 3 so that no bond is doubled by the wrap-around."""
    if lx == 0:
        return [(i, j, t) for (i, j) in bonds(L, periodic)]
    if L % lx:
        raise ValueError("L must be a multiple of lx")
    ly = L // lx
    if lx < 3 or ly < 3:
        raise ValueError("a periodic 2D cluster needs both sides >= 3")
    site = lambda x, y: (x % lx) + lx * (y % ly)  # noqa: E731
    out = []
    for y in range(ly):
        for x in range(lx):
            out.append((site(x, y), site(x + 1, y), t))
            out.append((site(x, y), site(x, y + 1), t))
            if tp != 0.0:
                out.append((site(x, y), site(x + 1, y + 1), tp))
                out.append((site(x, y), site(x - 1, y + 1), tp))
    return out


def hop_term(sec: Sector, i: int, j: int, spin: int):
    """COO triplets of c^dag_{j,s} c_{i,s} on `sec`: rows (new), cols (old), values."""
    oi = orbital(sec.L, i, spin, sec.order)
    oj = orbital(sec.L, j, spin, sec.order)
    a1, s1, mid = annihilate(sec.jw, oi)
    a2, s2, new = create(mid, oj)
    ok = a1 & a2
    cols = np.nonzero(ok)[0]
    rows = sec.index_of_jw(new[ok])
    return rows, cols, (s1 * s2)[ok]


def hamiltonian(sec: Sector, t: float, U: float, Uc: float = 0.0, core_site: int | None = None,
                periodic: bool = True, bond_list=None, flux: float = 0.0) -> sp.csr_matrix:
    """H of Eq. (9) on `sec`, plus -Uc (n_{j,up} + n_{j,dn}) of Eq. (10) when core_site is set.
    bond_list: (i, j, t_ij) bonds (cluster_bonds); default the chain's bonds with hopping t.
    flux: a magnetic flux through the ring (Peierls phases): the hop of an electron from
    i to j = i + 1 (mod L) carries exp(+i flux / L), the reverse hop exp(-i flux / L),
    which makes H complex Hermitian (chain bonds only)."""
    R, C, V = [], [], []
    theta = flux / sec.L
    for (i, j, tij) in (bond_list if bond_list is not None else [(i, j, t) for (i, j) in bonds(sec.L, periodic)]):
        for s in (0, 1):
            for (a, b), ph in (((i, j), theta), ((j, i), -theta)):   # c^dag_b c_a and its h.c.
                r, c, v = hop_term(sec, a, b, s)
                amp = -tij * (np.exp(1j * ph) if flux != 0.0 else 1.0)
                R.append(r); C.append(c); V.append(amp * v)
    diag = np.zeros(sec.dim)
    for i in range(sec.L):
        diag += U * (sec.occupation(i, 0) * sec.occupation(i, 1))
    if core_site is not None:
        diag -= Uc * (sec.occupation(core_site, 0) + sec.occupation(core_site, 1))
    idx = np.arange(sec.dim)
    R.append(idx); C.append(idx); V.append(diag)
    H = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                      shape=(sec.dim, sec.dim)).tocsr()
    H.sum_duplicates()
    H.eliminate_zeros()
    return H


def species_hops(L: int, n: int, t: float, periodic: bool = True, bond_list=None) -> sp.csr_matrix:
    """Hopping matrix of one spin species alone: -t sum_<ij> (c^dag_j c_i + h.c.)
    on the L-bit strings with n set bits (rank order), with the textbook
    Jordan-Wigner sign computed by `annihilate` / `create` on those strings."""
    states = sector_states(L, n)
    rank = np.full(1 << L, -1, dtype=np.int64)
    rank[states] = np.arange(len(states))
    R, C, V = [], [], []
    for (i, j, tij) in (bond_list if bond_list is not None else [(i, j, t) for (i, j) in bonds(L, periodic)]):
        for (a, b) in ((i, j), (j, i)):
            a1, s1, mid = annihilate(states, a)
            a2, s2, new = create(mid, b)
            ok = a1 & a2
            R.append(rank[new[ok]]); C.append(np.nonzero(ok)[0]); V.append(-tij * (s1 * s2)[ok])
    D = len(states)
    T = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(D, D)).tocsr()
    T.sum_duplicates()
    return T


def hamiltonian_kron(sec: Sector, t: float, U: float, Uc: float = 0.0, core_site: int | None = None,
                     periodic: bool = True, bond_list=None) -> sp.csr_matrix:
    """The same H (Eq. 9, plus the core-hole term of Eq. 10) assembled as
    T_up (x) I + I (x) T_dn + diag.  With the "up-first" orbital order every
    orbital strictly between two up orbitals is an up orbital (and likewise for
    down), so a hop's Jordan-Wigner sign involves its own species only and each
    hop term factorises into one species' hop matrix times the identity on the
    other.  A faster construction for large sectors; equal to `hamiltonian`
    entry by entry (pinned in tests/test_oracle_model.py)."""
    if sec.order != "up-first":
        raise ValueError("the Kronecker form needs the up-first orbital order")
    Tu = species_hops(sec.L, sec.n_up, t, periodic, bond_list)
    Td = species_hops(sec.L, sec.n_dn, t, periodic, bond_list)
    diag = U * popcount(sec.u & sec.d).astype(np.float64)
    if core_site is not None:
        diag -= Uc * (sec.occupation(core_site, 0) + sec.occupation(core_site, 1))
    H = (sp.kron(Tu, sp.identity(sec.D_dn), format="csr") + sp.kron(sp.identity(sec.D_up), Td, format="csr")
         + sp.diags(diag, format="csr"))
    H.sum_duplicates()
    H.eliminate_zeros()
    return H.tocsr()


def creation_operator(src: Sector, dst: Sector, site: int, spin: int) -> sp.csr_matrix:
    """Matrix of c^dag_{site,spin} from sector `src` to sector `dst` (dst.dim x src.dim)."""
    o = orbital(src.L, site, spin, src.order)
    acts, sign, new = create(src.jw, o)
    cols = np.nonzero(acts)[0]
    rows = dst.index_of_jw(new[acts])
    return sp.csr_matrix((sign[acts], (rows, cols)), shape=(dst.dim, src.dim))


def annihilation_operator(src: Sector, dst: Sector, site: int, spin: int) -> sp.csr_matrix:
    """Matrix of c_{site,spin} from sector `src` to sector `dst` (dst.dim x src.dim)."""
    o = orbital(src.L, site, spin, src.order)
    acts, sign, new = annihilate(src.jw, o)
    cols = np.nonzero(acts)[0]
    rows = dst.index_of_jw(new[acts])
    return sp.csr_matrix((sign[acts], (rows, cols)), shape=(dst.dim, src.dim))


@dataclass
class RixsModel:
    """H on the ground sector, H' on the intermediate sector, O2 and O1, and the
    final-state H (Eqs. 1, 2, 9, 10).

    O2 = c^dag_{j,spin} creates the excited electron with spin `spin`; O1 =
    c_{j,spin_out} fills the core hole from the valence orbital with spin
    `spin_out` (default: the same spin).  spin_out == spin is the spin-conserving
    channel, whose final states lie in the ground sector; spin_out != spin is the
    spin-flip channel, whose final states lie in the sector with one `spin_out`
    electron fewer and one `spin` electron more (Sec. III's polarisation
    channels, with the 2p orbitals reduced to one spin orbital).  lx > 0 makes
    the lattice the periodic lx x (L / lx) cluster with diagonal hopping tp
    (cluster_bonds)."""
    L: int
    n_up: int
    n_dn: int
    t: float
    U: float
    Uc: float
    core_site: int = 0
    periodic: bool = True
    order: str = "up-first"
    spin: int = 0            # spin of the created electron: 0 = up (c^dag_{j,up})
    spin_out: int | None = None
    lx: int = 0
    tp: float = 0.0

    def __post_init__(self):
        if self.spin_out is None:
            self.spin_out = self.spin
        self.bonds = cluster_bonds(self.L, self.periodic, self.t, self.lx, self.tp)
        dn_shift = (1 if self.spin == 1 else 0)
        up_shift = (1 if self.spin == 0 else 0)
        self.gsec = Sector(self.L, self.n_up, self.n_dn, self.order)
        self.isec = Sector(self.L, self.n_up + up_shift, self.n_dn + dn_shift, self.order)
        fu = self.isec.n_up - (1 if self.spin_out == 0 else 0)
        fd = self.isec.n_dn - (1 if self.spin_out == 1 else 0)
        self.H = hamiltonian(self.gsec, self.t, self.U, bond_list=self.bonds)
        self.Hp = hamiltonian(self.isec, self.t, self.U, self.Uc, self.core_site, bond_list=self.bonds)
        if (fu, fd) == (self.n_up, self.n_dn):
            self.fsec, self.Hf = self.gsec, self.H
        else:
            self.fsec = Sector(self.L, fu, fd, self.order)
            self.Hf = hamiltonian(self.fsec, self.t, self.U, bond_list=self.bonds)
        self.O2 = creation_operator(self.gsec, self.isec, self.core_site, self.spin)
        self.O1 = annihilation_operator(self.isec, self.fsec, self.core_site, self.spin_out)
