"""GPU parity of the whole RIXS map (Eqs. 1-2) and of the continued fraction."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import hubbard, rixs as orixs, solvers, spectrum
import workloads

pytestmark = pytest.mark.gpu


def _params(api, prec=0, **kw):
    base = dict(Gamma=0.3, eta=0.1, solve_tol=1e-12, cf_tol=1e-12, precision=prec)
    base.update(kw)
    return api.map_params(**base)


@pytest.fixture(scope="module")
def chain8_oracle():
    wl = workloads.CHAIN8
    return wl, orixs.rixs_map(wl.L, wl.n_up, wl.n_dn, 1.0, 8.0, 4.0, 0, wl.Gamma, wl.eta, wl.w_in, wl.w,
                              cf_tol=1e-13, gs_start=workloads.lanczos_start(4900, 1))


def test_continued_fraction_matches_oracle(cuda, chain8_oracle):
    from paper_2506_09551_gb300 import api
    wl, ref = chain8_oracle
    op = api.Operator.hubbard(api.model(wl.L, wl.n_up, wl.n_dn))
    rows = [0, 13, 20, 40]
    phi = torch.tensor(ref.phi[rows], dtype=torch.complex128, device="cuda")
    I, depth = op.continued_fraction(phi, ref.E_G, wl.w, wl.eta, cf_tol=1e-12)
    for i, k in enumerate(rows):
        assert np.max(np.abs(I[i] - ref.I[k])) <= 1e-9 * np.max(ref.I[k]), k
    assert (depth > 0).all()


def test_chain8_map_fp64(cuda, chain8_oracle):
    """The L = 8 workload in full: relative L2 map error <= 1e-8 (FP64 path)."""
    from paper_2506_09551_gb300 import api
    wl, ref = chain8_oracle
    I, info, st = api.rixs_map(api.model(wl.L, wl.n_up, wl.n_dn), _params(api, solve_tol=1e-10, cf_tol=1e-10),
                               wl.w_in, wl.w)
    assert st == 0
    assert abs(info["E_G"] - ref.E_G) <= 1e-12 * abs(ref.E_G)
    err = orixs.relative_l2(I, ref.I)
    assert err <= 1e-8, err
    assert I.min() >= -1e-12 * I.max()
    assert info["n_converged"] == wl.n_in


def test_chain8_map_mixed(cuda, chain8_oracle):
    from paper_2506_09551_gb300 import api
    wl, ref = chain8_oracle
    I, info, st = api.rixs_map(api.model(wl.L, wl.n_up, wl.n_dn), _params(api, 1, solve_tol=1e-6, cf_tol=1e-8),
                               wl.w_in, wl.w)
    err = orixs.relative_l2(I, ref.I)
    assert err <= 1e-4, err


@pytest.mark.parametrize("L,nu,nd,periodic", [(4, 2, 2, True), (6, 3, 3, True), (5, 3, 2, False)])
def test_tiny_maps_vs_lehmann(cuda, L, nu, nd, periodic):
    from paper_2506_09551_gb300 import api
    om = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, 1, periodic)
    w_in = np.linspace(-4, 12, 11)
    w = np.linspace(-1, 10, 60)
    I, info, st = api.rixs_map(api.model(L, nu, nd, core_site=1, periodic=periodic), _params(api), w_in, w)
    ev, V = np.linalg.eigh(om.H.toarray())
    G = V[:, 0]
    I_l = spectrum.lehmann_map(om.H, om.Hp, om.O2, om.O1, G, ev[0], w_in, w, 0.3, 0.1)
    assert orixs.relative_l2(I, I_l) <= 1e-9


def test_atomic_limit_map_with_user_ground_state(cuda):
    from paper_2506_09551_gb300 import api
    L, U, Uc, Gamma, eta = 6, 8.0, 4.0, 0.3, 0.1
    om = hubbard.RixsModel(L, 3, 3, 0.0, U, Uc, 2)
    sec = om.gsec
    mask = ((sec.u & sec.d) == 0) & ((sec.u | sec.d) == (1 << L) - 1)
    G = np.where(mask, workloads.lanczos_start(sec.dim, 7), 0.0)
    G /= np.linalg.norm(G)
    w_in = np.linspace(-4, 12, 13)
    w = np.linspace(-1, 10, 50)
    I, info, st = api.rixs_map(api.model(L, 3, 3, t=0.0, core_site=2), _params(api), w_in, w,
                               G=torch.tensor(G, device="cuda"), E_G=0.0)
    wgt = np.linalg.norm(om.O2 @ G) ** 2
    ref = (wgt / np.abs(U - 2 * Uc - w_in - 1j * Gamma) ** 2)[:, None] * (eta / (w ** 2 + eta ** 2))[None, :] / np.pi
    assert orixs.relative_l2(I, ref) <= 1e-12


def test_seed_choice_does_not_change_the_map(cuda, chain8_oracle):
    from paper_2506_09551_gb300 import api
    wl, ref = chain8_oracle
    m = api.model(wl.L, wl.n_up, wl.n_dn)
    I0, _, _ = api.rixs_map(m, _params(api, seed_index=-1), wl.w_in, wl.w)
    I1, _, _ = api.rixs_map(m, _params(api, seed_index=0), wl.w_in, wl.w)
    I2, _, _ = api.rixs_map(m, _params(api, seed_index=40), wl.w_in, wl.w)
    assert orixs.relative_l2(I1, I0) <= 1e-8 and orixs.relative_l2(I2, I0) <= 1e-8


def test_translation_and_spin_invariance(cuda):
    from paper_2506_09551_gb300 import api
    w_in = np.linspace(-4, 12, 9)
    w = np.linspace(-1, 10, 30)
    maps = [api.rixs_map(api.model(8, 4, 4, core_site=j), _params(api), w_in, w)[0] for j in (0, 3, 7)]
    for I in maps[1:]:
        assert orixs.relative_l2(I, maps[0]) <= 1e-9


def test_map_sites_batched_right_hand_sides(cuda, chain8_oracle):
    """One call for every core site of the L = 8 ring (the batched workload's shape):
    each site's map equals the single-site call, all sites agree by translation
    invariance, and site 0 matches the oracle."""
    from paper_2506_09551_gb300 import api
    wl, ref = chain8_oracle
    m = api.model(wl.L, wl.n_up, wl.n_dn)
    p = _params(api, solve_tol=1e-10, cf_tol=1e-10)
    sites = list(range(wl.L))
    I, info, st = api.rixs_map_sites(m, p, sites, wl.w_in, wl.w)
    assert st == 0 and I.shape == (wl.L, wl.n_in, wl.n_w)
    assert orixs.relative_l2(I[0], ref.I) <= 1e-8
    single, _, _ = api.rixs_map(api.model(wl.L, wl.n_up, wl.n_dn, core_site=3), p, wl.w_in, wl.w)
    assert orixs.relative_l2(I[3], single) <= 1e-9
    for j in sites[1:]:
        assert orixs.relative_l2(I[j], I[0]) <= 1e-8, j


@pytest.mark.parametrize("L,nu,nd,periodic", [(8, 4, 4, True), (7, 3, 3, False), (10, 5, 5, True)])
def test_continued_fraction_fp32(cuda, L, nu, nd, periodic):
    """FP32 second step vs the oracle's FP64 fraction on the same phi (even D_dn uses the
    two-elements-per-thread kernel, odd D_dn the general one)."""
    from paper_2506_09551_gb300 import api
    om = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, 0, periodic)
    E_G, G, _ = solvers.ground_state(om.H, workloads.lanczos_start(om.H.shape[0], 1))
    n = om.Hp.shape[0]
    A = (om.Hp - (E_G + 0.3j) * sp.identity(n)).tocsr()
    X, _ = solvers.solve_shifted(A, om.O2 @ G, np.array([-2.0, 0.0, 4.0]), tol=1e-12)
    phi = np.ascontiguousarray((om.O1 @ X.T).T)
    w = np.linspace(-1, 10, 60)
    op = api.Operator.hubbard(api.model(L, nu, nd, periodic=periodic))
    I, depth = op.continued_fraction(torch.tensor(phi, dtype=torch.complex64, device="cuda"), E_G, w, 0.1,
                                     cf_tol=1e-7)
    for k in range(3):
        ref, _ = spectrum.lanczos_cf(om.H, phi[k], E_G, w, 0.1)
        assert np.max(np.abs(I[k] - ref)) <= 1e-4 * np.max(ref), k
