"""Oracle: the second step of Eq. (1) (TEST INFRASTRUCTURE ONLY).

What is computed, and where the paper defines it
------------------------------------------------
For each intermediate state Psi_k and phi_k = O1 Psi_k,
    I(w_in_k, w) = (1/pi) Im <phi_k| (H - E_G - w - i eta)^{-1} |phi_k>     (Eq. 1)
with the paper's i0+ replaced by a finite broadening eta and the
proportionality constant taken as 1/pi (so that the integral over w of I is
||phi_k||^2 as eta -> 0).

* lanczos_cf: the continued-fraction expansion the paper uses for this step
  (Sec. II and the memory discussion of Sec. III): a Hermitian Lanczos
  tridiagonalisation of H started from phi/||phi|| (no reorthogonalisation),
  G(z) = n0 / (z - a_0 - b_1^2 / (z - a_1 - b_2^2 / ...)), z = E_G + w + i eta,
  and I = -(1/pi) Im G(z).  The depth grows in blocks of 50 until no I(w)
  moves by more than cf_tol relative to max|I| between successive blocks, or
  the Krylov space is exhausted (b_k tiny).
* direct_second_step: the plain definition, one sparse solve per loss energy.
* lehmann_map: the Kramers-Heisenberg sum over eigenstates of H' and H by
  full diagonalisation (the textbook form of Eqs. 1-2), for tiny clusters.

Parity: pinned by tests/test_oracle_spectrum.py (CF vs direct solves; the
Lehmann sum vs the whole oracle map; the atomic limit; the Kubo limit;
non-negativity; the sum rule).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class _Lanczos:
    """Hermitian Lanczos on real symmetric H from complex phi, no reorthogonalisation,
    advanced on demand.  a[k] = <q_k|H|q_k>, b[k] = b_{k+1} = ||H q_k - a_k q_k - b_k q_{k-1}||."""

    def __init__(self, H, phi: np.ndarray):
        self.H = H
        self.n0 = float(np.vdot(phi, phi).real)
        self.a, self.b = [], []
        self.done = self.n0 == 0.0
        if not self.done:
            self.q = phi / np.sqrt(self.n0)
            self.q_prev = np.zeros_like(self.q)
            self.b_prev = 0.0
            self.scale = None

    def advance(self, steps: int):
        for _ in range(steps):
            if self.done:
                return
            w = self.H @ self.q - self.b_prev * self.q_prev
            a = float(np.vdot(self.q, w).real)
            w = w - a * self.q
            b = float(np.linalg.norm(w))
            self.a.append(a)
            self.b.append(b)
            if self.scale is None:
                self.scale = max(abs(a), b, 1.0)
            if b <= 1e-14 * self.scale:        # invariant Krylov space: exact termination
                self.done = True
                return
            self.q_prev, self.q = self.q, w / b
            self.b_prev = b


def lanczos_coefficients(H, phi: np.ndarray, kmax: int):
    """(n0, a[0..K-1], b[1..K]) of the Hermitian Lanczos run from phi (K <= kmax)."""
    lz = _Lanczos(H, phi)
    lz.advance(kmax)
    return lz.n0, np.array(lz.a), np.array(lz.b)


def cf_green(n0: float, a: np.ndarray, b: np.ndarray, z: np.ndarray, depth: int | None = None):
    """G(z) = n0 / (z - a_0 - b_1^2 / (z - a_1 - ...)) truncated after `depth`
    levels with a zero tail, evaluated bottom-up."""
    K = len(a) if depth is None else depth
    z = np.asarray(z, dtype=np.complex128)
    g = np.zeros_like(z)
    for k in range(K - 1, -1, -1):
        tail = b[k] ** 2 * g if k < K - 1 else 0.0
        g = 1.0 / (z - a[k] - tail)
    return n0 * g


def lanczos_cf(H, phi: np.ndarray, E_G: float, w: np.ndarray, eta: float,
               kmax: int = 6000, cf_tol: float = 1e-13, block: int = 50):
    """I(w) = -(1/pi) Im G(E_G + w + i eta) by a continued fraction of converged depth.

    The depth grows by `block` levels at a time; it stops when no I(w) moved
    by more than cf_tol * max|I| since the previous block, or when the Krylov
    space is exhausted.  Returns (I, depth_used)."""
    lz = _Lanczos(H, phi)
    z = E_G + np.asarray(w) + 1j * eta
    if lz.done:
        return np.zeros(len(w)), 0
    prev = None
    while True:
        lz.advance(block)
        K = len(lz.a)
        I = -np.imag(cf_green(lz.n0, np.array(lz.a), np.array(lz.b), z, K)) / np.pi
        if lz.done or K >= kmax:
            return I, K
        if prev is not None and np.max(np.abs(I - prev)) <= cf_tol * max(np.max(np.abs(I)), 1e-300):
            return I, K
        prev = I


def direct_second_step(H, phi: np.ndarray, E_G: float, w: np.ndarray, eta: float):
    """(1/pi) Im <phi|(H - E_G - w - i eta)^{-1}|phi> by one sparse LU solve per w."""
    n = H.shape[0]
    Hc = sp.csc_matrix(H, dtype=np.complex128)
    I = sp.identity(n, dtype=np.complex128, format="csc")
    out = np.zeros(len(w))
    for i, wi in enumerate(w):
        x = spla.splu((Hc - (E_G + wi + 1j * eta) * I).tocsc()).solve(phi.astype(np.complex128))
        out[i] = np.imag(np.vdot(phi, x)) / np.pi
    return out


def lehmann_map(H, Hp, O2, O1, G: np.ndarray, E_G: float, w_in: np.ndarray, w: np.ndarray,
                Gamma: float, eta: float):
    """Kramers-Heisenberg sum by full diagonalisation of H (final) and H' (intermediate):
    I = (1/pi) sum_f |sum_n <f|O1|n><n|O2|G> / (E'_n - E_G - w_in - i Gamma)|^2
        * eta / ((E_f - E_G - w)^2 + eta^2)."""
    Ei, Vi = np.linalg.eigh(Hp.toarray())
    Ef, Vf = np.linalg.eigh(H.toarray())
    amp = Vi.T @ (O2 @ G)                       # <n|O2|G>
    M = Vf.T @ (O1 @ Vi)                        # <f|O1|n>
    out = np.zeros((len(w_in), len(w)))
    lor = eta / ((Ef[None, :] - E_G - np.asarray(w)[:, None]) ** 2 + eta ** 2)   # (n_w, n_f)
    for k, win in enumerate(w_in):
        A = M @ (amp / (Ei - E_G - win - 1j * Gamma))    # (n_f,)
        out[k] = lor @ (np.abs(A) ** 2) / np.pi
    return out
