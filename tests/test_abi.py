"""The C ABI library builds, loads and exports every symbol of include/msbicg.h.
Host-only calls (sector basis) are checked against the oracle; no GPU needed."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import hubbard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "msbicg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(msb_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2506_09551_gb300 import native
    names = header_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert n in native.SIGNATURES, n
    assert set(native.SIGNATURES) == set(names)


def test_version_and_defaults(lib):
    from paper_2506_09551_gb300 import native
    assert b"sm_103a" in lib.msb_version()
    p = native.msb_map_params()
    lib.msb_map_params_default(C.byref(p))
    assert p.Gamma == 0.3 and p.eta == 0.1 and p.solve_tol == 1e-10 and p.precision == 0


@pytest.mark.parametrize("L,nu,nd", [(4, 2, 2), (8, 4, 4), (12, 7, 6), (14, 8, 7), (16, 8, 8)])
def test_basis_states_match_oracle(lib, L, nu, nd):
    from paper_2506_09551_gb300 import api
    up, dn = api.basis_states(L, nu, nd)
    assert np.array_equal(up, hubbard.sector_states(L, nu))
    assert np.array_equal(dn, hubbard.sector_states(L, nd))


def test_invalid_arguments_are_reported(lib):
    from paper_2506_09551_gb300 import native
    h = C.c_void_p()
    assert lib.msb_basis_create(17, 2, 2, C.byref(h)) == native.MSB_EINVAL
    assert b"L must be" in lib.msb_last_error()
    assert lib.msb_basis_create(4, 5, 2, C.byref(h)) == native.MSB_EINVAL


def test_no_device_fails_loudly(lib):
    """Without a CUDA device the compute entry points refuse with MSB_ECUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2506_09551_gb300 import native
    m = native.msb_model(6, 3, 3, 1, 1.0, 8.0, 4.0, 0)
    h = C.c_void_p()
    assert lib.msb_op_create_hubbard(C.byref(m), 0, C.byref(h)) == native.MSB_ECUDA
    assert b"CUDA" in lib.msb_last_error()
    # the batch entry points refuse the same way (no CPU fallback)
    parts = (C.c_void_p * 1)(None)
    assert lib.msb_op_create_direct_sum(parts, None, 1, C.byref(h)) == native.MSB_ECUDA
    p = native.msb_map_params()
    lib.msb_map_params_default(C.byref(p))
    models = (native.msb_model * 2)(m, m)
    w = (C.c_double * 2)(0.0, 1.0)
    I = (C.c_double * 8)()
    info = native.msb_solve_info()
    assert lib.msb_rixs_map_clusters(models, 2, C.byref(p), w, 2, w, 2, I, None, C.byref(info),
                                     None) == native.MSB_ECUDA
