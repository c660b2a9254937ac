"""The per-incident-energy baseline on the GPU: BiCGStab for every shift on its own
(Sec. III, Fig. 4), against the oracle's independent solves and its own BiCGStab."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import hubbard, solvers
import workloads

pytestmark = pytest.mark.gpu


def _system(L, nu, nd):
    om = hubbard.RixsModel(L, nu, nd, 1.0, 8.0, 4.0, 0, True)
    E_G, G, _ = solvers.ground_state(om.H, workloads.lanczos_start(om.H.shape[0], 1))
    n = om.Hp.shape[0]
    A = (om.Hp - (E_G + 0.3j) * sp.identity(n)).tocsr()
    return E_G, A, (om.O2 @ G).astype(np.complex128)


@pytest.mark.parametrize("L,nu,nd", [(8, 4, 4), (10, 5, 5)])
def test_bicgstab_matches_independent_solves(cuda, L, nu, nd):
    from paper_2506_09551_gb300 import api
    E_G, A, b = _system(L, nu, nd)
    w_in = np.linspace(-4.0, 12.0, 9)
    ref, _ = solvers.solve_shifted(A, b, w_in, tol=1e-13, method="lu" if A.shape[0] <= 5000 else "bicgstab")
    op = api.Operator.hubbard(api.model(L, nu, nd), True)
    bt = torch.tensor(b, device="cuda")
    x, per, info, st = op.bicgstab(bt, w_in, c0=-(E_G + 0.3j), tol=1e-12, maxit=20000)
    assert st == 0 and per["converged"].all()
    assert info["matvecs"] == 2 * int(per["iters"].sum()) + int(per["restarts"].sum())
    err = np.linalg.norm(x.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-8, err
    # the oracle's BiCGStab needs a comparable number of products per shift
    n_or = [solvers.bicgstab(lambda v, s=s: A @ v - s * v, b, 1e-12)[1] for s in w_in[::4]]
    n_gpu = 2 * per["iters"][::4]
    assert all(0.5 * a <= g <= 2.0 * a + 10 for a, g in zip(n_or, n_gpu)), (n_or, n_gpu)
    # FP32-mixed vectors
    x32, per32, info32, st32 = op.bicgstab(bt, w_in, c0=-(E_G + 0.3j), tol=1e-6, maxit=20000, prec=api.FP32_MIXED)
    assert per32["converged"].all()
    err32 = np.linalg.norm(x32.cpu().numpy().astype(np.complex128) - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err32.max() <= 1e-4, err32


def test_bicgstab_and_msbicg_agree_and_count(cuda):
    """Same solutions from both methods; MSBiCG needs one product per iteration for all
    shifts, BiCGStab two per iteration per shift (Sec. II)."""
    from paper_2506_09551_gb300 import api
    E_G, A, b = _system(8, 4, 4)
    w_in = np.linspace(-4.0, 12.0, 21)
    seed = workloads.seed_index(w_in)
    op = api.Operator.hubbard(api.model(8, 4, 4), True)
    bt = torch.tensor(b, device="cuda")
    xb, perb, infob, stb = op.bicgstab(bt, w_in, c0=-(E_G + 0.3j), tol=1e-11)
    xm, perm, infom, stm = op.multishift_solve(bt, w_in - w_in[seed], c0=-(E_G + 0.3j + w_in[seed]), tol=1e-11)
    assert stb == 0 and stm == 0
    d = np.linalg.norm(xb.cpu().numpy() - xm.cpu().numpy(), axis=1) / np.linalg.norm(xm.cpu().numpy(), axis=1)
    assert d.max() <= 1e-8
    assert infom["matvecs"] == infom["iterations"]
    assert infob["matvecs"] > 5 * infom["matvecs"]
