"""Parity against the oracle at the full sizes of the L = 14 and L = 12 workloads.

* L = 14 ring, ground sector D = 11,778,624 (the FP32-mixed workload's size): the
  continued fraction of Eq. 1 at a fixed depth K (cf_check = cf_maxdepth = K), in
  FP64 and FP32, against the oracle's Lanczos coefficients and bottom-up fraction at
  the same K, on seeded complex columns.  These are the row-tiled apply kernels the
  L = 14 map runs: rows of 3432 elements (the 256-thread fixed-point FP64 kernel) and
  the bank-aware row placement of the FP32 kernel.
* L = 14 intermediate sector D' = 10,306,296: the multi-shift solve (App. C, Alg. 1)
  capped at 30 iterations against the oracle's MSBiCG capped the same way.
* L = 14 ring with one up and seven down electrons (rows of 3432 elements, D = 48,048,
  D' = 312,312): the whole map in FP64 and FP32-mixed against the plain definition
  (independent solves per incident energy, Eqs. 1-2).
* L = 12 workload (101 x 400 points): five rows spread over the incident grid,
  including the seed row at the atomic resonance, in FP64 and FP32-mixed.

The oracle's H and H' at these sizes are assembled in the Kronecker form
(hubbard.hamiltonian_kron, pinned equal to the generic construction); its rows run
in a spawn process pool (tests/oracle_pool.py).
"""
import numpy as np
import pytest
import torch

from oracle import hubbard, rixs as orixs, solvers, spectrum
import oracle_pool
import workloads

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-8        # relative L2 error of the FP64 path
MIXED_BAR = 1e-4       # relative L2 error of the FP32-mixed path


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def h14():
    return hubbard.hamiltonian_kron(hubbard.Sector(14, 7, 7), 1.0, 8.0)


@pytest.fixture(scope="module")
def hp14():
    return hubbard.hamiltonian_kron(hubbard.Sector(14, 8, 7), 1.0, 8.0, 4.0, 0)


def test_chain14_continued_fraction_fixed_depth(cuda, h14):
    from paper_2506_09551_gb300 import api
    K, E0, eta = 24, -4.6, 0.1
    w = workloads.CHAIN14.w
    D = h14.shape[0]
    phi = workloads.random_complex_vectors(D, 2, seed=0x14CF)
    z = E0 + w + 1j * eta
    ref = []
    for k in range(2):
        n0, a, b = spectrum.lanczos_coefficients(h14, phi[k], K)
        assert len(a) == K
        ref.append(-np.imag(spectrum.cf_green(n0, a, b, z, K)) / np.pi)
    op = api.Operator.hubbard(api.model(14, 7, 7))
    for prec, dt, bar in ((api.FP64, torch.complex128, FP64_BAR), (api.FP32_MIXED, torch.complex64, MIXED_BAR)):
        x = torch.tensor(phi, dtype=dt, device="cuda")
        I, depth = op.continued_fraction(x, E0, w, eta, cf_tol=0.0, cf_check=K, cf_maxdepth=K, prec=prec)
        del x
        assert (depth == K).all()
        for k in range(2):
            err = _rel(I[k], ref[k])
            print(f"L=14 CF depth {K}, precision {prec}, column {k}: relative L2 {err:.2e}")
            assert err <= bar, (prec, k, err)


def test_chain14_solve_capped_iterations(cuda, hp14):
    from paper_2506_09551_gb300 import api, native
    maxit, E0, Gamma = 30, -4.6, 0.3
    n = hp14.shape[0]
    b = workloads.random_complex_vectors(n, 1, seed=0x14B1)[0]
    w_in = np.array([-4.0, -1.0, 0.0, 2.4, 12.0])
    c0 = -(E0 + 1j * Gamma)                    # seed system A = H' - E0 - i Gamma, shifts s_k = w_in_k
    ref = solvers.msbicg(lambda v: hp14 @ v + c0 * v, b, w_in.astype(np.complex128), tol=1e-15, maxit=maxit)
    assert ref["m"] == maxit
    op = api.Operator.hubbard(api.model(14, 7, 7, core_site=0), True)
    assert op.dim == n
    bt = torch.tensor(b, dtype=torch.complex128, device="cuda")
    for prec, bar in ((api.FP64, 1e-10), (api.FP32_MIXED, MIXED_BAR)):
        x, per, info, st = op.multishift_solve(bt, w_in, c0=c0, tol=1e-15, maxit=maxit, prec=prec,
                                               allow_status=(native.MSB_EMAXITER,))
        assert st == native.MSB_EMAXITER and info["iterations"] == maxit
        for k in range(len(w_in)):
            err = _rel(x[k].cpu().numpy().astype(np.complex128), ref["x"][k])
            print(f"L=14 solve, {maxit} iterations, precision {prec}, w_in {w_in[k]}: relative L2 {err:.2e}")
            assert err <= bar, (prec, k, err)
        del x


def _oracle_rows(wl_args, G, E_G, w_in_rows, w, cf_tol=1e-12, solve_tol=1e-12):
    L, nu, nd, core, Gamma, eta = wl_args
    jobs = [(L, nu, nd, core, Gamma, eta, E_G, G, float(x), w, solve_tol, cf_tol) for x in w_in_rows]
    with oracle_pool.pool(len(jobs)) as p:
        return np.array(p.map(oracle_pool.map_row, jobs))


def test_chain14_long_rows_map(cuda):
    """Rows of 3432 elements in a small sector: the whole map against the plain definition."""
    from paper_2506_09551_gb300 import api
    L, nu, nd = 14, 1, 7
    w_in = np.linspace(-4.0, 12.0, 9)
    w = workloads.CHAIN14.w
    sec = hubbard.Sector(L, nu, nd)
    H = hubbard.hamiltonian_kron(sec, 1.0, 8.0)
    E_G, G, _ = solvers.ground_state(H, workloads.lanczos_start(H.shape[0], 1))
    ref = _oracle_rows((L, nu, nd, 0, 0.3, 0.1), G, E_G, w_in, w)
    m = api.model(L, nu, nd)
    I64, info64, st64 = api.rixs_map(m, api.map_params(solve_tol=1e-10, cf_tol=1e-9, precision=api.FP64), w_in, w)
    I32, info32, st32 = api.rixs_map(m, api.map_params(solve_tol=1e-8, cf_tol=1e-5, precision=api.FP32_MIXED),
                                     w_in, w)
    assert st64 == 0 and st32 == 0
    assert abs(info64["E_G"] - E_G) <= 1e-11 * abs(E_G)
    e64, e32 = orixs.relative_l2(I64, ref), orixs.relative_l2(I32, ref)
    print(f"L=14 (1 up, 7 down) map: FP64 {e64:.2e}, FP32-mixed {e32:.2e}")
    assert e64 <= FP64_BAR and e32 <= MIXED_BAR


def test_chain12_rows_against_oracle(cuda):
    """The L = 12 workload on its full grid; the oracle recomputes five rows (the ends,
    the seed row at the atomic resonance w_in = 0, and two more) by independent solves."""
    from paper_2506_09551_gb300 import api
    wl = workloads.CHAIN12
    m = api.model(wl.L, wl.n_up, wl.n_dn)
    I64, info64, st64 = api.rixs_map(m, api.map_params(solve_tol=1e-10, cf_tol=1e-9, precision=api.FP64),
                                     wl.w_in, wl.w)
    I32, info32, st32 = api.rixs_map(m, api.map_params(solve_tol=1e-8, cf_tol=1e-5, precision=api.FP32_MIXED),
                                     wl.w_in, wl.w)
    assert st64 == 0 and info64["n_converged"] == wl.n_in and st32 == 0
    H = hubbard.hamiltonian_kron(hubbard.Sector(wl.L, wl.n_up, wl.n_dn), 1.0, 8.0)
    E_G, G, _ = solvers.ground_state(H, workloads.lanczos_start(H.shape[0], 1), kmax=250)
    assert abs(info64["E_G"] - E_G) <= 1e-11 * abs(E_G)
    rows = [0, workloads.seed_index(wl.w_in), 40, 70, wl.n_in - 1]
    ref = _oracle_rows((wl.L, wl.n_up, wl.n_dn, 0, wl.Gamma, wl.eta), G, E_G, wl.w_in[rows], wl.w)
    for i, k in enumerate(rows):
        e64, e32 = _rel(I64[k], ref[i]), _rel(I32[k], ref[i])
        print(f"L=12 row {k} (w_in {wl.w_in[k]:+.2f}): FP64 {e64:.2e}, FP32-mixed {e32:.2e}")
        assert e64 <= FP64_BAR, (k, e64)
        assert e32 <= MIXED_BAR, (k, e32)
    assert orixs.relative_l2(I64[rows], ref) <= FP64_BAR
