"""Pins of the oracle's momentum-resolved map (coherent sum over core sites)."""
import numpy as np

from oracle import rixs as orixs
import workloads


def _qmap(L, nu, nd, qs):
    return orixs.rixs_map_q(L, nu, nd, 1.0, 8.0, 4.0, 0.3, 0.1, np.linspace(-4, 12, 5),
                            np.linspace(-1, 10, 40), qs, cf_tol=1e-13)


def test_momentum_sum_rule_and_reflection():
    L = 4
    qs = 2 * np.pi * np.arange(L) / L
    r = _qmap(L, 2, 2, qs)
    # sum over the L momenta = L x sum of the single-site maps (phases sum to L delta_jj')
    lhs = r.I.sum(axis=0)
    rhs = L * r.I_site.sum(axis=0)
    assert np.max(np.abs(lhs - rhs)) <= 1e-10 * np.max(np.abs(rhs))
    # reflection j -> -j of the ring: I_q = I_{-q} (q = pi/2 and 3 pi/2)
    assert np.max(np.abs(r.I[1] - r.I[3])) <= 1e-10 * np.max(np.abs(r.I[1]))
    assert r.I.min() >= -1e-12 * r.I.max()
    # translation invariance: every single-site map is the same
    for j in range(1, L):
        assert np.max(np.abs(r.I_site[j] - r.I_site[0])) <= 1e-10 * np.max(r.I_site[0])


def test_q_zero_is_not_the_incoherent_sum():
    """The coherent sum has interference: at q = 0 it differs from L x a single-site
    map (it would equal it only without inter-site terms)."""
    r = _qmap(4, 2, 2, np.array([0.0]))
    inc = 4 * r.I_site[0]
    assert np.max(np.abs(r.I[0] - inc)) > 1e-3 * np.max(inc)
