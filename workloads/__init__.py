"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module holds input generation only: model parameters, energy grids, seeds,
random start vectors, the random sparse stress matrix and its right-hand side.
It contains none of the method's arithmetic (no Hamiltonian, no solver, no
spectrum), so both the CPU oracle and the CUDA path may take their inputs from
it without sharing any computation.

The paper's own workloads (doped 2D Betts clusters with intermediate-state
dimensions of 1e8-1e9, Sec. III) cannot be held on one GPU and their data is
not available; the 1D Hubbard chains below keep the paper's energy scales
(U = 8t, U_c = 4t, Gamma of order t; Sec. III) and a dense incident-energy grid
(200-300 points in Sec. III) and stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass(frozen=True)
class HubbardWorkload:
    """One RIXS-map workload on a periodic 1D Hubbard chain.

    The ground state lives in the (n_up, n_dn) sector; the intermediate state
    after O2 = c^dagger_{j,up} lives in (n_up + 1, n_dn) (Eqs. 1-2, Sec. III).
    """
    name: str
    L: int
    n_up: int
    n_dn: int
    t: float = 1.0
    U: float = 8.0
    Uc: float = 4.0
    core_site: int = 0
    periodic: bool = True
    Gamma: float = 0.3
    eta: float = 0.1
    n_in: int = 41
    w_in_range: tuple = (-4.0, 12.0)
    n_w: int = 200
    w_range: tuple = (-1.0, 10.0)
    gs_tol: float = 1e-12
    solve_tol: float = 1e-10
    lanczos_seed: int = 1

    @property
    def w_in(self) -> np.ndarray:
        return np.linspace(self.w_in_range[0], self.w_in_range[1], self.n_in)

    @property
    def w(self) -> np.ndarray:
        return np.linspace(self.w_range[0], self.w_range[1], self.n_w)


# The named workloads.  Sizes: D = C(L,n_up) C(L,n_dn), D' = C(L,n_up+1) C(L,n_dn).
CHAIN8 = HubbardWorkload("hubbard-L8-fp64", L=8, n_up=4, n_dn=4, n_in=41, n_w=200)
CHAIN12 = HubbardWorkload("hubbard-L12-fp64", L=12, n_up=6, n_dn=6, n_in=101, n_w=400)
CHAIN14 = HubbardWorkload("hubbard-L14-mixed", L=14, n_up=7, n_dn=7, n_in=201, n_w=400)

# Batched workload: one L=12 chain with one right-hand side per core site
# j = 0..11, plus three clusters of uneven size, 64 incident energies each.
BATCH_SITES = HubbardWorkload("hubbard-L12x12rhs", L=12, n_up=6, n_dn=6, n_in=64, n_w=400)
BATCH_CLUSTERS = (
    HubbardWorkload("hubbard-L10", L=10, n_up=5, n_dn=5, n_in=64, n_w=400),
    HubbardWorkload("hubbard-L11", L=11, n_up=6, n_dn=5, n_in=64, n_w=400),
    HubbardWorkload("hubbard-L12", L=12, n_up=6, n_dn=6, n_in=64, n_w=400),
)

# Small cases for tests (tiny clusters that full diagonalisation handles).
def tiny(L: int, n_up: int, n_dn: int, **kw) -> HubbardWorkload:
    base = dict(n_in=9, n_w=25)
    base.update(kw)
    return HubbardWorkload(f"hubbard-L{L}-tiny", L=L, n_up=n_up, n_dn=n_dn, **base)


def seed_index(w_in: np.ndarray) -> int:
    """Index of the incident energy used as the seed system: the grid point
    nearest to the atomic resonance w_in = E_edge, i.e. w_in = 0 once E_edge is
    absorbed into w_in (Sec. III picks the atomic resonance as the seed)."""
    return int(np.argmin(np.abs(np.asarray(w_in))))


def lanczos_start(n: int, seed: int = 1) -> np.ndarray:
    """Seeded real random start vector for the ground-state Lanczos (unnormalised)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n)


# ---------------------------------------------------------------------------
# Random complex-symmetric stress workload.
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class RandomCSRWorkload:
    name: str = "random-csr-2^22"
    n: int = 1 << 22
    half_nnz_per_row: int = 8          # 8 drawn columns, mirrored -> ~16 per row
    diag_range: tuple = (-4.0, 4.0)
    n_shifts: int = 256
    shift_range: tuple = (-6.0, 6.0)
    shift_imag: float = 0.3
    matrix_seed: int = 0x5EED0001
    rhs_seed: int = 0x5EED0002
    shift_seed: int = 0x5EED0003
    solve_tol: float = 1e-10


RANDOM_CSR = RandomCSRWorkload()


def random_symmetric_csr(n: int, half_nnz_per_row: int, diag_range=(-4.0, 4.0), seed: int = 0x5EED0001):
    """Real symmetric sparse matrix in CSR form (rowptr int64, col int32, val float64).

    For each row i draw `half_nnz_per_row` columns j != i uniformly and one
    N(0,1) value each; the value is placed at (i,j) and (j,i) and duplicates
    are summed.  The diagonal is U[diag_range].  Columns within a row are
    sorted ascending and the diagonal is stored as an explicit entry.
    """
    rng = np.random.default_rng(seed)
    k = half_nnz_per_row
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    cols = rng.integers(0, n - 1, size=n * k, dtype=np.int64)
    cols = cols + (cols >= rows)            # uniform over j != i
    vals = rng.standard_normal(n * k)
    diag = rng.uniform(diag_range[0], diag_range[1], size=n)
    r = np.concatenate([rows, cols, np.arange(n, dtype=np.int64)])
    c = np.concatenate([cols, rows, np.arange(n, dtype=np.int64)])
    v = np.concatenate([vals, vals, diag])
    # sort by (row, col) and sum duplicates
    key = r * n + c
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    uniq, start = np.unique(key, return_index=True)
    vsum = np.add.reduceat(v, start)
    rr = (uniq // n).astype(np.int64)
    cc = (uniq % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rr + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cc, vsum


def random_complex_rhs(n: int, seed: int = 0x5EED0002) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def random_shifts(k: int, lo: float, hi: float, imag: float, seed: int = 0x5EED0003) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=k) + 1j * imag


def random_complex_vectors(n: int, k: int, seed: int) -> np.ndarray:
    """(k, n) complex test vectors with N(0,1) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
