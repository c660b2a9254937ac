"""Oracle: the whole RIXS map of Eqs. (1)-(2) (TEST INFRASTRUCTURE ONLY).

Pipeline (every step is the plain definition; nothing is fused or reordered):
  1. H, H', O2, O1 as CSR matrices (hubbard.RixsModel; Eqs. 9-10).
  2. |G>, E_G by Lanczos (solvers.ground_state), unless the caller passes G.
  3. E = O2 |G> (Eq. 2).
  4. Psi_k = (H' - E_G - w_in_k - i Gamma)^{-1} E, each k solved on its own
     (Eq. 2 / Eq. A1; solvers.solve_shifted).
  5. phi_k = O1 Psi_k (Eq. 1).
  6. I(w_in_k, w) = (1/pi) Im <phi_k|(H_f - E_G - w - i eta)^{-1}|phi_k> by the
     continued fraction (spectrum.lanczos_cf), or by direct solves; H_f is H on
     the final sector (the ground sector in the spin-conserving channel).

Parity: pinned by tests/test_oracle_spectrum.py against the Lehmann sum at
L = 4 and 6, the atomic limit, the Kubo limit and the model's symmetries.
rixs_map_q (the momentum-resolved map, a coherent sum over core sites): pinned by
tests/test_oracle_momentum.py (sum over the L momenta = L x the sum of the single-site
maps; reflection symmetry q -> -q; non-negativity).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import hubbard, solvers, spectrum


@dataclass
class MapResult:
    I: np.ndarray                 # (n_in, n_w)
    E_G: float
    G: np.ndarray
    Psi: np.ndarray               # (n_in, D')
    phi: np.ndarray               # (n_in, D)
    matvecs: int
    cf_depth: list
    seconds: dict = field(default_factory=dict)


def rixs_map(L, n_up, n_dn, t, U, Uc, core_site, Gamma, eta, w_in, w, *, periodic=True,
             order="up-first", spin=0, spin_out=None, lx=0, tp=0.0, G=None, E_G=None, gs_tol=1e-12,
             gs_start=None, solve_tol=1e-13, solve_method="auto", second_step="cf", cf_tol=1e-13,
             model=None) -> MapResult:
    sec = {}
    t0 = time.perf_counter()
    m = model or hubbard.RixsModel(L, n_up, n_dn, t, U, Uc, core_site, periodic, order, spin, spin_out, lx, tp)
    sec["build"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    if G is None:
        v0 = gs_start if gs_start is not None else np.random.default_rng(1).standard_normal(m.H.shape[0])
        E_G, G, _ = solvers.ground_state(m.H, v0, gs_tol)
    elif E_G is None:
        E_G = float(G @ (m.H @ G)) / float(G @ G)
    sec["ground_state"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    E = m.O2 @ G
    A = m.Hp - E_G * _eye(m.Hp.shape[0]) - 1j * Gamma * _eye(m.Hp.shape[0])
    Psi, nmv = solvers.solve_shifted(A, E, np.asarray(w_in, dtype=float), tol=solve_tol,
                                     method=solve_method)
    sec["solve"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    phi = (m.O1 @ Psi.T).T
    I = np.zeros((len(w_in), len(w)))
    depths = []
    for k in range(len(w_in)):
        if second_step == "cf":
            I[k], d = spectrum.lanczos_cf(m.Hf, phi[k], E_G, np.asarray(w), eta, cf_tol=cf_tol)
            depths.append(d)
        else:
            I[k] = spectrum.direct_second_step(m.Hf, phi[k], E_G, np.asarray(w), eta)
            depths.append(0)
    sec["second_step"] = time.perf_counter() - t0
    return MapResult(I, E_G, G, Psi, phi, nmv, depths, sec)


@dataclass
class QMapResult:
    I: np.ndarray                 # (n_q, n_in, n_w) coherent maps
    I_site: np.ndarray            # (L, n_in, n_w) single-site maps (core hole at j)
    E_G: float
    qs: np.ndarray


def rixs_map_q(L, n_up, n_dn, t, U, Uc, Gamma, eta, w_in, w, qs, *, periodic=True, gs_start=None,
               gs_tol=1e-12, solve_tol=1e-13, cf_tol=1e-13) -> QMapResult:
    """Momentum-resolved map: the coherent sum over core sites j of Eqs. (1)-(2).

    For every site j the intermediate state Psi_j(w_in) is solved with the core hole on
    j (H'_j, Eq. 10) and mapped back, phi_j = c_{j,up} Psi_j (Eq. 1).  The momentum-q
    final-state vector is phi_q = sum_j exp(i q j) phi_j (dipole operators summed with the
    phase of momentum transfer q, Sec. III), and
        I_q(w_in, w) = (1/pi) Im <phi_q|(H - E_G - w - i eta)^{-1}|phi_q>
    by the continued fraction.  Over the L momenta q = 2 pi k / L the phases sum to
    L delta_{jj'}, so sum_q I_q = L sum_j I_j with I_j the single-site maps.
    """
    w_in = np.asarray(w_in, dtype=float)
    w = np.asarray(w, dtype=float)
    qs = np.asarray(qs, dtype=float)
    m0 = hubbard.RixsModel(L, n_up, n_dn, t, U, Uc, 0, periodic)
    v0 = gs_start if gs_start is not None else np.random.default_rng(1).standard_normal(m0.H.shape[0])
    E_G, G, _ = solvers.ground_state(m0.H, v0, gs_tol)
    phis = []
    I_site = np.zeros((L, len(w_in), len(w)))
    for j in range(L):
        mj = hubbard.RixsModel(L, n_up, n_dn, t, U, Uc, j, periodic)
        A = mj.Hp - E_G * _eye(mj.Hp.shape[0]) - 1j * Gamma * _eye(mj.Hp.shape[0])
        Psi, _ = solvers.solve_shifted(A, mj.O2 @ G, w_in, tol=solve_tol)
        phi = (mj.O1 @ Psi.T).T
        phis.append(phi)
        for k in range(len(w_in)):
            I_site[j, k], _ = spectrum.lanczos_cf(m0.H, phi[k], E_G, w, eta, cf_tol=cf_tol)
    I = np.zeros((len(qs), len(w_in), len(w)))
    for iq, q in enumerate(qs):
        for k in range(len(w_in)):
            phi_q = sum(np.exp(1j * q * j) * phis[j][k] for j in range(L))
            I[iq, k], _ = spectrum.lanczos_cf(m0.H, phi_q, E_G, w, eta, cf_tol=cf_tol)
    return QMapResult(I, I_site, E_G, qs)


def _eye(n):
    import scipy.sparse as sp
    return sp.identity(n, format="csr")


def relative_l2(I: np.ndarray, I_ref: np.ndarray) -> float:
    """||I - I_ref||_F / ||I_ref||_F over the whole (w_in, w) map."""
    return float(np.linalg.norm(I - I_ref) / np.linalg.norm(I_ref))
