"""The method's cost claim (Sec. III, Fig. 4), pinned on the oracle at small size: the
multi-shifted BiCG needs one seed Krylov space for every incident energy, so its
matrix-vector products do not grow with the number of incident energies, while
independent per-energy BiCGStab solves (the paper's baseline) grow linearly."""
import numpy as np
import scipy.sparse as sp

from oracle import hubbard, solvers
import workloads


def test_mvm_counts_vs_number_of_incident_energies():
    om = hubbard.RixsModel(6, 3, 3, 1.0, 8.0, 4.0, 0, True)
    E_G, G, _ = solvers.ground_state(om.H, workloads.lanczos_start(om.H.shape[0], 1))
    n = om.Hp.shape[0]
    A = (om.Hp - (E_G + 0.3j) * sp.identity(n)).tocsr()
    b = (om.O2 @ G).astype(np.complex128)
    ms, stab = {}, {}
    for n_in in (5, 20, 80):
        w_in = np.linspace(-4.0, 12.0, n_in)
        seed = int(np.argmin(np.abs(w_in)))
        res = solvers.msbicg(lambda v: A @ v - w_in[seed] * v, b, w_in - w_in[seed], 1e-10, 5000)
        assert res["converged"].all()
        ms[n_in] = res["m"]                              # one MVM per seed iteration
        total = 0
        for w in w_in:
            _, nmv = solvers.bicgstab(lambda v, w=w: A @ v - w * v, b, 1e-10)
            total += nmv
        stab[n_in] = total
    assert max(ms.values()) <= 1.3 * min(ms.values())   # flat in n_in
    assert stab[80] >= 8 * stab[5] and stab[20] >= 2.5 * stab[5]   # linear in n_in
    assert stab[80] >= 10 * ms[80]                      # an order of magnitude at 80 energies
