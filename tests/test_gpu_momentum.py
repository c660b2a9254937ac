"""Momentum-resolved maps on the GPU (coherent sum over core sites) against the oracle."""
import numpy as np
import pytest

from oracle import rixs as orixs

pytestmark = pytest.mark.gpu


def test_momentum_maps_match_oracle_and_sum_rule(cuda):
    from paper_2506_09551_gb300 import api
    L = 6
    qs = 2 * np.pi * np.arange(L) / L
    w_in = np.linspace(-4, 12, 5)
    w = np.linspace(-1, 10, 40)
    m = api.model(L, 3, 3)
    p = api.map_params(Gamma=0.3, eta=0.1, solve_tol=1e-11, cf_tol=1e-11, precision=0)
    I, info, st = api.rixs_map_q(m, p, qs, w_in, w)
    assert st == 0 and I.shape == (L, 5, 40)
    ref = orixs.rixs_map_q(L, 3, 3, 1.0, 8.0, 4.0, 0.3, 0.1, w_in, w, qs, cf_tol=1e-13)
    err = orixs.relative_l2(I, ref.I)
    assert err <= 1e-8, err
    sites, _, _ = api.rixs_map_sites(m, p, list(range(L)), w_in, w)
    lhs, rhs = I.sum(axis=0), L * sites.sum(axis=0)
    assert np.max(np.abs(lhs - rhs)) <= 1e-8 * np.max(np.abs(rhs))
