"""Pins of the cluster batch (several independent clusters in one multi-shift solve).

The library solves the clusters' systems (H'_c - E_G,c - w_seed - i Gamma - s_k) x = b_c
together, as one system on the block-diagonal direct sum with the concatenated
right-hand side.  These tests check that reading against the oracle alone: the oracle's
MSBiCG on the direct sum reproduces each cluster's independent solves, and the joint
residual bound tol * min_c ||b_c|| meets every cluster's own bound."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import hubbard, solvers
import workloads


def _cluster_systems():
    out = []
    for (L, nu, nd) in ((4, 2, 2), (5, 2, 3), (6, 3, 3)):
        om = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, 0, True)
        E_G, G, _ = solvers.ground_state(om.H, workloads.lanczos_start(om.H.shape[0], 1))
        out.append((om, E_G, om.O2 @ G))
    return out


def test_direct_sum_solve_equals_independent_solves():
    Gamma, w_seed = 0.3, 0.0
    shifts = np.array([-3.0, -1.0, 0.0, 2.5, 7.0])
    systems = _cluster_systems()
    blocks = [(om.Hp - E_G * sp.identity(om.Hp.shape[0])).tocsr() for om, E_G, _ in systems]
    A = sp.block_diag(blocks, format="csr") - (w_seed + 1j * Gamma) * sp.identity(sum(b.shape[0] for b in blocks))
    b = np.concatenate([bc for _, _, bc in systems])
    norms = np.array([np.linalg.norm(bc) for _, _, bc in systems])
    tol = 1e-10
    joint_tol = tol * norms.min() / np.linalg.norm(b)
    res = solvers.msbicg(A, b, shifts, joint_tol, 2000)
    assert res["converged"].all()
    off = np.cumsum([0] + [blk.shape[0] for blk in blocks])
    for c, (om, E_G, bc) in enumerate(systems):
        n = blocks[c].shape[0]
        for k, s in enumerate(shifts):
            Ac = (blocks[c] - (w_seed + 1j * Gamma + s) * sp.identity(n)).tocsc()
            ref = spla.spsolve(Ac, bc)
            xc = res["x"][k, off[c]:off[c + 1]]
            # each cluster's own residual meets its own bound
            r = np.linalg.norm(bc - Ac @ xc)
            assert r <= 1.01 * tol * np.linalg.norm(bc), (c, k, r)
            assert np.linalg.norm(xc - ref) <= 1e-7 * np.linalg.norm(ref), (c, k)


def test_direct_sum_blocks_do_not_mix():
    """A right-hand side living in one block gives solutions that vanish in the others
    (the block-diagonal operator keeps the clusters apart)."""
    systems = _cluster_systems()
    blocks = [(om.Hp - E_G * sp.identity(om.Hp.shape[0])).tocsr() for om, E_G, _ in systems]
    n = sum(blk.shape[0] for blk in blocks)
    A = sp.block_diag(blocks, format="csr") - 0.3j * sp.identity(n)
    b = np.zeros(n, dtype=complex)
    off = blocks[0].shape[0]
    b[off:off + blocks[1].shape[0]] = systems[1][2]
    res = solvers.msbicg(A, b, np.array([-1.0, 2.0]), 1e-12, 2000)
    x = res["x"]
    assert np.abs(x[:, :off]).max() == 0.0
    assert np.abs(x[:, off + blocks[1].shape[0]:]).max() == 0.0
