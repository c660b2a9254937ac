"""Clusters of uneven size computed together (one solve on the direct sum of their H',
one continued fraction over all their columns): GPU parity against separate maps and
against the oracle."""
import numpy as np
import pytest
import torch

from oracle import rixs as orixs
import workloads

pytestmark = pytest.mark.gpu


def _rand(n, nvec, seed):
    g = np.random.default_rng(seed)
    x = g.standard_normal((nvec, n)) + 1j * g.standard_normal((nvec, n))
    return torch.tensor(x, dtype=torch.complex128, device="cuda")


def test_direct_sum_apply_matches_parts(cuda):
    from paper_2506_09551_gb300 import api
    parts = [api.Operator.hubbard(api.model(6, 3, 3), True),
             api.Operator.hubbard(api.model(7, 3, 4, core_site=2), True),
             api.Operator.hubbard(api.model(8, 4, 4, periodic=False), True)]
    shifts = [-1.5, 0.25, 3.0]
    S = api.Operator.direct_sum(parts, shifts)
    assert S.dim == sum(p.dim for p in parts)
    x = _rand(S.dim, 2, 7)
    y = S.apply(x, c0=0.5 - 0.3j)
    off = 0
    for p, s in zip(parts, shifts):
        xp = x[:, off:off + p.dim].contiguous()
        ref = p.apply(xp, c0=s + 0.5 - 0.3j)
        got = y[:, off:off + p.dim]
        assert torch.max(torch.abs(got - ref)).item() <= 1e-13 * torch.max(torch.abs(ref)).item()
        off += p.dim


def test_direct_sum_rejections(cuda):
    from paper_2506_09551_gb300 import api, native
    a = api.Operator.hubbard(api.model(6, 3, 3), True)
    S = api.Operator.direct_sum([a, a], [0.0, 1.0])
    with pytest.raises(native.MsbError):
        S.ground_state()
    phi = _rand(S.dim, 1, 1)
    with pytest.raises(native.MsbError):
        S.continued_fraction(phi, 0.0, np.linspace(0, 1, 5), 0.1)
    rowptr, col, val = np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0, 2.0])
    csr = api.Operator.csr(rowptr, col, val)
    with pytest.raises(native.MsbError):
        api.Operator.direct_sum([a, csr])
    with pytest.raises(native.MsbError):
        api.Operator.direct_sum([a] * 17)


def test_cluster_map_matches_separate_maps_and_oracle(cuda):
    """Three uneven clusters in one call (FP64) = three separate maps, and the first
    one = the oracle's independent solves and continued fraction."""
    from paper_2506_09551_gb300 import api
    models = [api.model(6, 3, 3), api.model(7, 4, 3, core_site=1), api.model(8, 4, 4, periodic=False)]
    p = api.map_params(Gamma=0.3, eta=0.1, solve_tol=1e-11, cf_tol=1e-11, precision=0)
    w_in = np.linspace(-4, 12, 17)
    w = np.linspace(-1, 10, 120)
    I, E, info, st = api.rixs_map_clusters(models, p, w_in, w)
    assert st == 0 and info["n_converged"] == len(w_in)
    for c, m in enumerate(models):
        Ic, infoc, stc = api.rixs_map(m, p, w_in, w)
        assert abs(E[c] - infoc["E_G"]) <= 1e-11 * abs(E[c])
        err = orixs.relative_l2(I[c], Ic)
        assert err <= 1e-8, (c, err)
    ref = orixs.rixs_map(6, 3, 3, 1.0, 8.0, 4.0, 0, 0.3, 0.1, w_in, w, cf_tol=1e-13,
                         gs_start=workloads.lanczos_start(400, 1))
    assert orixs.relative_l2(I[0], ref.I) <= 1e-8


def test_cluster_map_mixed_matches_fp64(cuda):
    """Uneven clusters L = 8, 9, 10 (dims 4,900 / 15,876 / 63,504): FP32-mixed within 1e-4
    of FP64, per cluster."""
    from paper_2506_09551_gb300 import api
    models = [api.model(8, 4, 4), api.model(9, 5, 4), api.model(10, 5, 5)]
    w_in = np.linspace(-4, 12, 16)
    w = np.linspace(-1, 10, 200)
    p64 = api.map_params(Gamma=0.3, eta=0.1, solve_tol=1e-10, cf_tol=1e-10, precision=0)
    p32 = api.map_params(Gamma=0.3, eta=0.1, solve_tol=1e-7, cf_tol=1e-8, precision=1)
    I64, E64, _, st64 = api.rixs_map_clusters(models, p64, w_in, w)
    I32, E32, _, st32 = api.rixs_map_clusters(models, p32, w_in, w)
    assert st64 == 0 and st32 == 0
    np.testing.assert_allclose(E32, E64, rtol=1e-11)
    for c in range(len(models)):
        err = orixs.relative_l2(I32[c], I64[c])
        assert err <= 1e-4, (c, err)
        assert I64[c].min() >= -1e-10 * I64[c].max()
