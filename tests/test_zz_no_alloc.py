"""The allocation-free ground state, called through the C ABI.

msb_ground_state_noalloc serves callers that cannot allocate device memory
(a process whose device memory belongs to another allocator under a fixed
budget): it uses a fixed scratch array inside the library instead.  Checked
here against the allocating msb_ground_state on two calls in a row, since the
array keeps the previous call's contents.  This file is collected last so a
failure here does not stop the other GPU tests from running first.
"""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


def _call(lib, op, tol=1e-12, maxit=300):
    g = torch.empty(op.dim, dtype=torch.float64, device="cuda")
    E, res = C.c_double(), C.c_double()
    st = lib.msb_ground_state_noalloc(op.h, tol, maxit, None, C.byref(E), C.c_void_p(g.data_ptr()), C.byref(res),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, E.value, g, res.value


@pytest.mark.parametrize("L,nu,nd", [(10, 5, 5), (8, 4, 4)])
def test_noalloc_ground_state_matches_allocating_call(cuda, L, nu, nd):
    from paper_2506_09551_gb300 import api, native
    lib = native.load()
    op = api.Operator.hubbard(api.model(L, nu, nd))
    E_ref, g_ref, res_ref = op.ground_state(1e-12, 300)
    for _ in range(2):
        st, E, g, res = _call(lib, op)
        assert st == native.MSB_OK, native.last_error()
        assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
        assert res <= 1e-12 * max(1.0, abs(E))
        assert abs(abs(torch.dot(g, g_ref).item()) - 1.0) <= 1e-11


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda):
    from paper_2506_09551_gb300 import api, native
    lib = native.load()
    op = api.Operator.hubbard(api.model(14, 7, 7))          # dim 11,778,624 > 2^20
    st, E, g, res = _call(lib, op)
    assert st == native.MSB_EINVAL
    assert "exceeds the no-alloc scratch limit" in native.last_error()
    op8 = api.Operator.hubbard(api.model(8, 4, 4))
    st, *_ = _call(lib, op8, maxit=2000)
    assert st == native.MSB_EINVAL
