"""Spin channels and 2D clusters on the GPU against the oracle (Sec. III's polarisation
channels and lattices at sizes that fit): the spin-flip channel (O2 = c^dag_{j,dn},
O1 = c_{j,up}, final states in another sector), the down-spin channel, and periodic
2D clusters with and without diagonal hopping t'."""
import numpy as np
import pytest
import torch

from oracle import rixs as orixs

pytestmark = pytest.mark.gpu

W_IN = np.linspace(-4.0, 12.0, 9)
W = np.linspace(-1.0, 10.0, 120)


def _oracle(L, nu, nd, j, spin, spin_out, lx, tp):
    return orixs.rixs_map(L, nu, nd, 1.0, 8.0, 4.0, j, 0.3, 0.1, W_IN, W, spin=spin, spin_out=spin_out, lx=lx, tp=tp)


@pytest.mark.parametrize("L,nu,nd,j,o2,o1,lx,tp", [
    (6, 3, 3, 0, 1, 0, 0, 0.0),        # spin flip, chain
    (7, 3, 3, 2, 0, 1, 0, 0.0),        # spin flip the other way, odd ring
    (6, 3, 2, 1, 1, 1, 0, 0.0),        # down-spin channel
    (9, 2, 1, 4, 0, 0, 3, -0.3),       # 3 x 3 cluster with diagonal hopping
    (12, 2, 2, 5, 0, 0, 3, 0.0),       # 3 x 4 cluster, 24 bonds: the row-tiled apply
    (12, 2, 1, 5, 1, 0, 3, 0.25),      # 3 x 4 cluster, t', spin flip
])
def test_channel_and_cluster_maps(cuda, L, nu, nd, j, o2, o1, lx, tp):
    from paper_2506_09551_gb300 import api
    ref = _oracle(L, nu, nd, j, o2, o1, lx, tp)
    m = api.model(L, nu, nd, core_site=j, o2_spin=o2, o1_spin=o1, lx=lx, tp=tp)
    # the library's own ground state (its energy must agree) ...
    _, info0, st0 = api.rixs_map(m, api.map_params(solve_tol=1e-10, cf_tol=1e-9, precision=api.FP64), W_IN, W)
    assert st0 == 0 and abs(info0["E_G"] - ref.E_G) <= 1e-10 * abs(ref.E_G)
    # ... and the maps from the oracle's |G> (open-shell fillings have a degenerate ground
    # level, where each side may pick another vector of it)
    G = torch.tensor(ref.G, dtype=torch.float64, device="cuda")
    I64, info64, st64 = api.rixs_map(m, api.map_params(solve_tol=1e-11, cf_tol=1e-10, precision=api.FP64), W_IN, W,
                                     G=G, E_G=ref.E_G)
    assert st64 == 0
    e64 = orixs.relative_l2(I64, ref.I)
    I32, _, st32 = api.rixs_map(m, api.map_params(solve_tol=1e-8, cf_tol=1e-5, precision=api.FP32_MIXED), W_IN, W,
                                G=G, E_G=ref.E_G)
    e32 = orixs.relative_l2(I32, ref.I)
    print(f"L={L} ({nu},{nd}) O2 spin {o2} O1 spin {o1} lx={lx} t'={tp}: FP64 {e64:.2e}, FP32-mixed {e32:.2e}")
    assert e64 <= 1e-8 and e32 <= 1e-4


def test_final_sector_operator_and_rejections(cuda):
    from paper_2506_09551_gb300 import api, native
    m = api.model(6, 3, 2, o2_spin=1, o1_spin=0)
    Hf = api.Operator.hubbard(m, 2)                      # final sector (2 up, 3 down)
    assert Hf.dim == 15 * 20
    with pytest.raises(native.MsbError):
        api.rixs_map_sites(m, api.map_params(), [0, 1], W_IN, W)   # the site batch is up-spin only
    with pytest.raises(native.MsbError):
        api.Operator.hubbard(api.model(8, 2, 2, lx=2), False)     # 2 x 4 torus doubles its bonds
