"""Torch / numpy front end of libmsbicg: argument marshalling only.

Device vectors are torch tensors on the current CUDA device (complex128 for
MSB_FP64, complex64 for MSB_FP32_MIXED; the ground state is float64); every
call runs on torch's current stream.  All arithmetic happens in the library.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import native as N

FP64, FP32_MIXED = N.MSB_FP64, N.MSB_FP32_MIXED


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def cdtype(prec: int) -> torch.dtype:
    return torch.complex128 if prec == FP64 else torch.complex64


def model(L, n_up, n_dn, t=1.0, U=8.0, Uc=4.0, core_site=0, periodic=True, o2_spin=0, o1_spin=None, lx=0,
          tp=0.0, flux=0.0) -> N.msb_model:
    """A Hubbard chain (lx = 0) or periodic lx x (L / lx) cluster with diagonal hopping tp, and
    the RIXS channel O2 = c^dag_{j,o2_spin}, O1 = c_{j,o1_spin} (o1_spin defaults to o2_spin);
    flux: Peierls phases on a ring (complex Hermitian H)."""
    o1 = o2_spin if o1_spin is None else o1_spin
    return N.msb_model(L, n_up, n_dn, 1 if periodic else 0, t, U, Uc, core_site, o2_spin, o1, lx, tp, flux)


def map_params(**kw) -> N.msb_map_params:
    p = N.msb_map_params()
    N.load().msb_map_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def basis_states(L: int, n_up: int, n_dn: int):
    lib = N.load()
    h = C.c_void_p()
    N.check(lib.msb_basis_create(L, n_up, n_dn, C.byref(h)))
    try:
        du, dd, dim = C.c_int64(), C.c_int64(), C.c_int64()
        N.check(lib.msb_basis_dims(h, C.byref(du), C.byref(dd), C.byref(dim)))
        up = np.zeros(du.value, dtype=np.uint32)
        dn = np.zeros(dd.value, dtype=np.uint32)
        N.check(lib.msb_basis_states(h, 0, up.ctypes.data_as(C.POINTER(C.c_uint32))))
        N.check(lib.msb_basis_states(h, 1, dn.ctypes.data_as(C.POINTER(C.c_uint32))))
        return up, dn
    finally:
        lib.msb_basis_destroy(h)


def row_order(L: int, n_dn: int, periodic: bool = True):
    """Continued-fraction row order: the down-spin state held at each position of a row."""
    lib = N.load()
    h = C.c_void_p()
    N.check(lib.msb_basis_create(L, 0, n_dn, C.byref(h)))
    try:
        dd = C.c_int64()
        N.check(lib.msb_basis_dims(h, None, C.byref(dd), None))
        order = np.zeros(dd.value, dtype=np.uint16)
        N.check(lib.msb_basis_row_order(h, 1 if periodic else 0, order.ctypes.data_as(C.POINTER(C.c_uint16))))
        return order
    finally:
        lib.msb_basis_destroy(h)


def row_layout(L: int, n_dn: int, periodic: bool = True, hops: bool = False):
    """Shared-memory slot of each row position (in the continued-fraction row order) used
    by the FP32 continued-fraction apply, and the mean worst-bank count per half-warp
    gather without / with it.  hops=True also returns the scheduled hop table (W x D:
    target position << 1 | sign bit per round, D << 1 for an idle round)."""
    lib = N.load()
    h = C.c_void_p()
    N.check(lib.msb_basis_create(L, 0, n_dn, C.byref(h)))
    try:
        dd = C.c_int64()
        N.check(lib.msb_basis_dims(h, None, C.byref(dd), None))
        slot = np.zeros(dd.value, dtype=np.uint16)
        width = C.c_int()
        c0, c1 = C.c_double(), C.c_double()
        N.check(lib.msb_basis_row_layout(h, 1 if periodic else 0, slot.ctypes.data_as(C.POINTER(C.c_uint16)),
                                         C.byref(width), None, C.byref(c0), C.byref(c1)))
        if not hops:
            return slot, c0.value, c1.value
        tab = np.zeros((width.value, dd.value), dtype=np.uint16)
        N.check(lib.msb_basis_row_layout(h, 1 if periodic else 0, None, None,
                                         tab.ctypes.data_as(C.POINTER(C.c_uint16)), None, None))
        return slot, c0.value, c1.value, tab
    finally:
        lib.msb_basis_destroy(h)


class Operator:
    """Handle of a library operator (matrix-free Hubbard H / H', or CSR)."""

    def __init__(self, handle: C.c_void_p):
        self.h = handle
        d = C.c_int64()
        N.check(N.load().msb_op_dim(self.h, C.byref(d)))
        self.dim = d.value

    @classmethod
    def hubbard(cls, m: N.msb_model, intermediate=False) -> "Operator":
        """H on the model's ground sector (intermediate = 0 / False), H' on the intermediate
        sector (1 / True) or H on the final sector of a spin-flip channel (2)."""
        h = C.c_void_p()
        N.check(N.load().msb_op_create_hubbard(C.byref(m), int(intermediate), C.byref(h)))
        return cls(h)

    @classmethod
    def csr(cls, rowptr: np.ndarray, col: np.ndarray, val: np.ndarray) -> "Operator":
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        h = C.c_void_p()
        N.check(N.load().msb_op_create_csr(len(rowptr) - 1, rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                                           col.ctypes.data_as(C.POINTER(C.c_int32)),
                                           val.ctypes.data_as(C.POINTER(C.c_double)), C.byref(h)))
        return cls(h)

    @classmethod
    def direct_sum(cls, ops, shifts=None) -> "Operator":
        """Block-diagonal (H_0 + s_0) (+) (H_1 + s_1) (+) ... of up to 4 Hubbard operators;
        keeps the parts alive (the library does not own them)."""
        arr = (C.c_void_p * len(ops))(*[o.h for o in ops])
        sh = None
        if shifts is not None:
            sh = np.ascontiguousarray(shifts, dtype=np.float64)
            if len(sh) != len(ops):
                raise ValueError("one shift per part")
        h = C.c_void_p()
        N.check(N.load().msb_op_create_direct_sum(arr, sh.ctypes.data_as(C.POINTER(C.c_double)) if sh is not None
                                                  else None, len(ops), C.byref(h)))
        op = cls(h)
        op._parts = list(ops)
        return op

    def close(self):
        if self.h:
            N.load().msb_op_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, x: torch.Tensor, c0: complex = 0.0, prec: int | None = None, out: torch.Tensor | None = None):
        """y = (A + c0) x; x of shape (dim,) or (nvec, dim)."""
        if prec is None:
            prec = FP64 if x.dtype == torch.complex128 else FP32_MIXED
        if x.dtype != cdtype(prec):
            raise ValueError("dtype does not match precision")
        nvec = 1 if x.dim() == 1 else x.shape[0]
        if x.shape[-1] != self.dim:
            raise ValueError("length does not match the operator dimension")
        y = torch.empty_like(x) if out is None else out
        N.check(N.load().msb_op_apply(self.h, N.msb_complex(complex(c0).real, complex(c0).imag), _ptr(x), _ptr(y),
                                      nvec, prec, _stream()))
        return y

    def ground_state(self, tol: float = 1e-12, maxit: int = 300, start: torch.Tensor | None = None):
        g = torch.empty(self.dim, dtype=torch.float64, device="cuda")
        E, res = C.c_double(), C.c_double()
        st = _ptr(start) if start is not None else None
        N.check(N.load().msb_ground_state(self.h, tol, maxit, st, C.byref(E), _ptr(g), C.byref(res), _stream()))
        return E.value, g, res.value

    def multishift_solve(self, b: torch.Tensor, shifts, c0: complex = 0.0, tol: float = 1e-10, maxit: int = 5000,
                         block: int = 0, prec: int = FP64, allow_status=(), dual: bool = False):
        """x_k = (A + c0 - s_k)^{-1} b for every shift.  Returns (x, per-shift dict, info dict, status).
        dual: the dual-space form for a Hermitian, not real symmetric, A (Peierls phases)."""
        shifts = np.asarray(shifts, dtype=np.complex128)
        ns = len(shifts)
        sh = (N.msb_complex * ns)(*[N.msb_complex(s.real, s.imag) for s in shifts])
        x = torch.empty((ns, self.dim), dtype=cdtype(prec), device="cuda")
        iters = np.zeros(ns, dtype=np.int32)
        resid = np.zeros(ns, dtype=np.float64)
        conv = np.zeros(ns, dtype=np.int32)
        info = N.msb_solve_info()
        c0 = complex(c0)
        fn = N.load().msb_multishift_bicg_dual_solve if dual else N.load().msb_multishift_bicg_solve
        st = fn(
            self.h, N.msb_complex(c0.real, c0.imag), _ptr(b.to(cdtype(prec)).contiguous()), sh, ns, tol, maxit,
            block, prec, _ptr(x), iters.ctypes.data_as(C.POINTER(C.c_int)),
            resid.ctypes.data_as(C.POINTER(C.c_double)), conv.ctypes.data_as(C.POINTER(C.c_int)), C.byref(info),
            _stream())
        N.check(st, allow=allow_status)
        return x, dict(iters=iters, resid=resid, converged=conv.astype(bool)), info.as_dict(), st

    def bicgstab(self, b: torch.Tensor, shifts, c0: complex = 0.0, tol: float = 1e-10, maxit: int = 20000,
                 prec: int = FP64, allow_status=(N.MSB_EMAXITER,)):
        """x_k = (A + c0 - s_k)^{-1} b, each shift by its own BiCGStab (the per-incident-energy
        baseline).  Returns (x, per-shift dict, info dict, status)."""
        shifts = np.asarray(shifts, dtype=np.complex128)
        ns = len(shifts)
        sh = (N.msb_complex * ns)(*[N.msb_complex(s.real, s.imag) for s in shifts])
        x = torch.empty((ns, self.dim), dtype=cdtype(prec), device="cuda")
        iters = np.zeros(ns, dtype=np.int32)
        resid = np.zeros(ns, dtype=np.float64)
        conv = np.zeros(ns, dtype=np.int32)
        restarts = np.zeros(ns, dtype=np.int32)
        info = N.msb_solve_info()
        c0 = complex(c0)
        st = N.load().msb_bicgstab_solve(
            self.h, N.msb_complex(c0.real, c0.imag), _ptr(b.to(cdtype(prec)).contiguous()), sh, ns, tol, maxit, prec,
            _ptr(x), iters.ctypes.data_as(C.POINTER(C.c_int)), resid.ctypes.data_as(C.POINTER(C.c_double)),
            conv.ctypes.data_as(C.POINTER(C.c_int)), restarts.ctypes.data_as(C.POINTER(C.c_int)), C.byref(info),
            _stream())
        N.check(st, allow=allow_status)
        return x, dict(iters=iters, resid=resid, converged=conv.astype(bool), restarts=restarts), info.as_dict(), st

    def multishift_reseeded(self, b: torch.Tensor, shifts, c0: complex = 0.0, tol: float = 1e-10,
                            maxit: int = 5000, reseed_tol: float = 1e-8, seed_index: int = 0, max_seeds: int = 8,
                            block: int = 0, prec: int = FP64):
        """Adaptive reseeding (App. E): x_k = (A + c0 - s_k)^{-1} b for every shift, reseeded
        from rejected shifts.  Returns (x, per-shift dict, seeds list, info dict, status)."""
        shifts = np.asarray(shifts, dtype=np.complex128)
        ns = len(shifts)
        sh = (N.msb_complex * ns)(*[N.msb_complex(s.real, s.imag) for s in shifts])
        x = torch.empty((ns, self.dim), dtype=cdtype(prec), device="cuda")
        conv = np.zeros(ns, dtype=np.int32)
        acc = np.zeros(ns, dtype=np.int32)
        dr = np.zeros(ns, dtype=np.float64)
        seeds = np.zeros(max_seeds, dtype=np.int32)
        nseeds = C.c_int()
        info = N.msb_solve_info()
        c0 = complex(c0)
        st = N.load().msb_multishift_bicg_reseeded(
            self.h, N.msb_complex(c0.real, c0.imag), _ptr(b.to(cdtype(prec)).contiguous()), sh, ns, tol, maxit,
            block, prec, reseed_tol, seed_index, max_seeds, _ptr(x), conv.ctypes.data_as(C.POINTER(C.c_int)),
            acc.ctypes.data_as(C.POINTER(C.c_int)), dr.ctypes.data_as(C.POINTER(C.c_double)),
            seeds.ctypes.data_as(C.POINTER(C.c_int)), C.byref(nseeds), C.byref(info), _stream())
        N.check(st, allow=(N.MSB_EMAXITER,))
        per = dict(converged=conv.astype(bool), accepted=acc.astype(bool), dr=dr)
        return x, per, seeds[:nseeds.value].tolist(), info.as_dict(), st

    def continued_fraction(self, phi: torch.Tensor, E0: float, w, eta: float, cf_tol: float = 1e-10,
                           cf_check: int = 50, cf_maxdepth: int = 4000, prec: int | None = None):
        if prec is None:
            prec = FP64 if phi.dtype == torch.complex128 else FP32_MIXED
        w = np.ascontiguousarray(w, dtype=np.float64)
        nv = 1 if phi.dim() == 1 else phi.shape[0]
        I = np.zeros((nv, len(w)), dtype=np.float64)
        depth = np.zeros(nv, dtype=np.int32)
        N.check(N.load().msb_continued_fraction(self.h, _ptr(phi), nv, E0, w.ctypes.data_as(C.POINTER(C.c_double)),
                                                len(w), eta, cf_tol, cf_check, cf_maxdepth, prec,
                                                I.ctypes.data_as(C.POINTER(C.c_double)),
                                                depth.ctypes.data_as(C.POINTER(C.c_int)), _stream()))
        return I, depth


def apply_cdag_up(m: N.msb_model, site: int, x: torch.Tensor, out_dim: int, prec: int = FP64):
    nvec = 1 if x.dim() == 1 else x.shape[0]
    y = torch.empty((nvec, out_dim) if x.dim() > 1 else (out_dim,), dtype=x.dtype, device="cuda")
    N.check(N.load().msb_apply_cdag_up(C.byref(m), site, _ptr(x), _ptr(y), nvec, prec, _stream()))
    return y


def apply_c_up(m: N.msb_model, site: int, x: torch.Tensor, out_dim: int, prec: int = FP64):
    nvec = 1 if x.dim() == 1 else x.shape[0]
    y = torch.empty((nvec, out_dim) if x.dim() > 1 else (out_dim,), dtype=x.dtype, device="cuda")
    N.check(N.load().msb_apply_c_up(C.byref(m), site, _ptr(x), _ptr(y), nvec, prec, _stream()))
    return y


def rixs_map_ops(H: Operator, Hp: Operator, params: N.msb_map_params, w_in, w, G: torch.Tensor | None = None,
                 E_G: float = 0.0, out: torch.Tensor | None = None, allow_status=(N.MSB_EMAXITER,)):
    """Map from prebuilt operators into a device tensor (n_in, n_w) float64."""
    w_in = np.ascontiguousarray(w_in, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    I = out if out is not None else torch.empty((len(w_in), len(w)), dtype=torch.float64, device="cuda")
    info = N.msb_solve_info()
    st = N.load().msb_rixs_map_ops(H.h, Hp.h, C.byref(params), _ptr(G) if G is not None else None, E_G,
                                   w_in.ctypes.data_as(C.POINTER(C.c_double)), len(w_in),
                                   w.ctypes.data_as(C.POINTER(C.c_double)), len(w), _ptr(I), C.byref(info),
                                   _stream())
    N.check(st, allow=allow_status)
    return I, info.as_dict(), st


def rixs_map_sites(m: N.msb_model, params: N.msb_map_params, sites, w_in, w, allow_status=(N.MSB_EMAXITER,)):
    """Maps of several core sites, I[n_sites, n_in, n_w] (numpy), info dict, status."""
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    w_in = np.ascontiguousarray(w_in, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    I = np.zeros((len(sites), len(w_in), len(w)), dtype=np.float64)
    info = N.msb_solve_info()
    st = N.load().msb_rixs_map_sites(C.byref(m), C.byref(params), sites.ctypes.data_as(C.POINTER(C.c_int)),
                                     len(sites), w_in.ctypes.data_as(C.POINTER(C.c_double)), len(w_in),
                                     w.ctypes.data_as(C.POINTER(C.c_double)), len(w),
                                     I.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info), _stream())
    N.check(st, allow=allow_status)
    return I, info.as_dict(), st


def rixs_map_q(m: N.msb_model, params: N.msb_map_params, qs, w_in, w, allow_status=(N.MSB_EMAXITER,)):
    """Momentum-resolved maps I[n_q, n_in, n_w] (coherent sum over core sites), info, status."""
    qs = np.ascontiguousarray(qs, dtype=np.float64)
    w_in = np.ascontiguousarray(w_in, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    I = np.zeros((len(qs), len(w_in), len(w)), dtype=np.float64)
    info = N.msb_solve_info()
    st = N.load().msb_rixs_map_q(C.byref(m), C.byref(params), qs.ctypes.data_as(C.POINTER(C.c_double)), len(qs),
                                 w_in.ctypes.data_as(C.POINTER(C.c_double)), len(w_in),
                                 w.ctypes.data_as(C.POINTER(C.c_double)), len(w),
                                 I.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info), _stream())
    N.check(st, allow=allow_status)
    return I, info.as_dict(), st


def rixs_map_clusters(models, params: N.msb_map_params, w_in, w, allow_status=(N.MSB_EMAXITER,)):
    """Maps of several independent clusters computed together (one solve on their direct
    sum, one continued fraction over all columns): I[n_clusters, n_in, n_w] (numpy),
    E_G per cluster (numpy), info dict, status."""
    arr = (N.msb_model * len(models))(*models)
    w_in = np.ascontiguousarray(w_in, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    I = np.zeros((len(models), len(w_in), len(w)), dtype=np.float64)
    E = np.zeros(len(models), dtype=np.float64)
    info = N.msb_solve_info()
    st = N.load().msb_rixs_map_clusters(arr, len(models), C.byref(params),
                                        w_in.ctypes.data_as(C.POINTER(C.c_double)), len(w_in),
                                        w.ctypes.data_as(C.POINTER(C.c_double)), len(w),
                                        I.ctypes.data_as(C.POINTER(C.c_double)),
                                        E.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info), _stream())
    N.check(st, allow=allow_status)
    return I, E, info.as_dict(), st


def rixs_map(m: N.msb_model, params: N.msb_map_params, w_in, w, G: torch.Tensor | None = None, E_G: float = 0.0,
             allow_status=(N.MSB_EMAXITER,)):
    """The RIXS map I[n_in, n_w] (numpy), the solve info (dict) and the status."""
    w_in = np.ascontiguousarray(w_in, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    I = np.zeros((len(w_in), len(w)), dtype=np.float64)
    info = N.msb_solve_info()
    st = N.load().msb_rixs_map(C.byref(m), C.byref(params), _ptr(G) if G is not None else None, E_G,
                               w_in.ctypes.data_as(C.POINTER(C.c_double)), len(w_in),
                               w.ctypes.data_as(C.POINTER(C.c_double)), len(w),
                               I.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info), _stream())
    N.check(st, allow=allow_status)
    return I, info.as_dict(), st


def autotune(m: N.msb_model, prec: int, n_in: int):
    """Timed trials of the per-shift update lag and of the continued-fraction apply's shape
    (FP64: threads per CTA; FP32: shape 1-4) on this model; the choices are cached by
    the library for later calls.  Returns a dict."""
    blk, thr = C.c_int(), C.c_int()
    bms = np.zeros(5, dtype=np.float64)
    cms = np.zeros(4, dtype=np.float64)
    N.check(N.load().msb_autotune(C.byref(m), prec, n_in, C.byref(blk), C.byref(thr),
                                  bms.ctypes.data_as(C.POINTER(C.c_double)), cms.ctypes.data_as(C.POINTER(C.c_double)),
                                  _stream()))
    cands = (128, 256) if prec == FP64 else (1, 2, 3, 4)
    return {"block": blk.value, "cf_threads": thr.value,
            "ms_per_iteration": dict(zip((1, 2, 4, 8, 16), bms.tolist())),
            "ms_per_level": dict(zip(cands, cms.tolist()))}


def autotune_forget():
    N.load().msb_autotune_forget()
