"""CPU pins of three arithmetic schemes the GPU path uses in place of the plain forms.

1. The continued fraction is carried forward level by level (modified Lentz
   recurrences) instead of being re-evaluated bottom-up at every convergence check.
   Both give the K-th convergent with a zero tail; here the forward recurrence, written
   out in numpy, is checked against the oracle's bottom-up cf_green on a real Lanczos run.
2. The FP64 Hamiltonian apply of the continued fraction sums its +-1 hop terms in 64-bit
   integer fixed point scaled by the column norm.  Here the conversion is emulated bit for
   bit in Python integers and its claimed properties are checked: |F| < 2^58, a loss below
   2^-55 ||V|| per term, exact sums of up to 2L terms, zeros and subnormals mapped to 0.
3. The FP32-mixed path forms its inner products (the bilinear products of the seed
   recurrence, the norms and the Lanczos products of the second step) from FP32 vectors
   with no FP64 instruction per element: each thread accumulates x*y as an unevaluated
   float pair (hi, lo), the product split exactly by an FMA (TwoProduct) and added by
   Knuth's TwoSum; the pairs are then summed in float-float and rounded to FP64 once.
   Emulated here with IEEE float32 numpy operations and checked against the exact FP64
   dot of the same FP32 data: relative error <= n 2^-46 * sum|x y| / |sum x y|."""
import math
import struct

import numpy as np
import pytest

from oracle import hubbard, solvers, spectrum
import workloads


# ---------------------------------------------------------------------------
# 1. forward convergents
# ---------------------------------------------------------------------------
def _forward_convergents(n0, a, b, z, checks):
    """G at the depths in `checks`, folding in only the new levels each time."""
    out = {}
    g = z - a[0]
    C = g.copy()
    D = np.zeros_like(z)
    j = 1
    for K in checks:
        for jj in range(j, K):
            cj = -b[jj - 1] ** 2                 # b[jj-1] = b_{jj}
            d = z - a[jj]
            D = 1.0 / (d + cj * D)
            C = d + cj / C
            g = g * C * D
        j = K
        out[K] = n0 / g
    return out


def test_forward_convergent_equals_bottom_up():
    om = hubbard.RixsModel(8, 4, 4, 1.0, 8.0, 4.0, 0, True)
    E_G, G, _ = solvers.ground_state(om.H, workloads.lanczos_start(om.H.shape[0], 1))
    phi = om.O1 @ (om.O2 @ G)                   # a real start vector of the N sector
    n0, a, b = spectrum.lanczos_coefficients(om.H, phi, 400)
    z = E_G + np.linspace(-1, 10, 200) + 0.1j
    checks = [k for k in range(50, len(a) + 1, 50)] or [len(a)]
    fwd = _forward_convergents(n0, a, b, z, checks)
    for K in checks:
        ref = spectrum.cf_green(n0, a, b, z, K)
        assert np.max(np.abs(fwd[K] - ref)) <= 1e-12 * np.max(np.abs(ref)), K


# ---------------------------------------------------------------------------
# 2. fixed-point hop sums
# ---------------------------------------------------------------------------
def _bits(v):
    return struct.unpack("<q", struct.pack("<d", v))[0]


def _eB(sig):
    es = (_bits(sig) >> 52) & 0x7FF
    return max(min(2047 - es, 2100), 63)


def _fx(v, eB, neg=0):
    b = _bits(v)
    e = (b >> 52) & 0x7FF
    r = min((eB - e) & 0xFFFFFFFF, 63)          # unsigned minimum, as on the device
    m = ((b & 0x000FFFFFFFFFFFFF) | 0x0010000000000000) << 5
    f = m >> r
    s = (-1 if b < 0 else 0) ^ neg
    return (f ^ s) - s


# Column norms whose square is a normal double (the CF computes ||W|| as the square
# root of a sum of squares; its vectors have norms b_k of order one).
@pytest.mark.parametrize("scale", [1e-120, 1e-8, 1.0, 3.7e5, 1e140])
def test_fixed_point_bounds_and_exact_sums(scale):
    rng = np.random.default_rng(5)
    V = rng.standard_normal(400) * 10.0 ** rng.uniform(-25, 0, 400) * scale
    V[:3] = [0.0, -0.0, 5e-324 if scale < 1 else 0.0]
    sig = 1.0 / float(np.linalg.norm(V))
    eB = _eB(sig)
    unit = 2.0 ** (eB - 1080)
    bound = 1.0 / sig
    for v in V:
        for neg in (0, -1):
            f = _fx(float(v), eB, neg)
            assert abs(f) < 2 ** 58
            want = -float(v) if neg else float(v)
            assert abs(f * unit - want) < 2.0 ** -55 * bound
    for _ in range(50):                          # hop sums of 28 distinct elements (2L, L = 14)
        idx = rng.choice(len(V), 28, replace=False)
        negs = rng.integers(0, 2, 28)
        acc = sum(_fx(float(V[i]), eB, -int(g)) for i, g in zip(idx, negs))
        assert abs(acc) < 2 ** 61
        exact = math.fsum((-V[i] if g else V[i]) for i, g in zip(idx, negs))
        assert abs(acc * unit - exact) <= 28 * 2.0 ** -55 * bound


def test_fixed_point_zero_and_nonfinite_map_to_zero():
    eB = _eB(1.0)
    assert _fx(0.0, eB) == 0 and _fx(-0.0, eB) == 0
    assert _fx(5e-324, eB) == 0                  # subnormal
    assert _fx(float("inf"), eB) == 0 and _fx(float("nan"), eB) == 0


# ---------------------------------------------------------------------------
# 3. float-float products of the FP32 path
# ---------------------------------------------------------------------------
_f32 = np.float32


def _two_prod(x, y):
    p = _f32(x * y)
    # the exact product of two float32 values is a float64; its rounding error is a float32
    pe = _f32(np.float64(x) * np.float64(y) - np.float64(p))
    return p, pe


def _df_add_prod(hi, lo, x, y):
    p, pe = _two_prod(x, y)
    s = _f32(hi + p)
    bb = _f32(s - hi)
    e = _f32(_f32(hi - _f32(s - bb)) + _f32(p - bb))
    return s, _f32(lo + _f32(e + pe))


def _df_add(hi, lo, bh, bl):
    s = _f32(hi + bh)
    bb = _f32(s - hi)
    e = _f32(_f32(hi - _f32(s - bb)) + _f32(bh - bb))
    return s, _f32(lo + _f32(e + bl))


@pytest.mark.parametrize("n,threads,signed", [(4096, 256, False), (20000, 256, True), (777, 32, True)])
def test_float_float_dot_against_fp64(n, threads, signed):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    if not signed:
        y = np.abs(y) * np.sign(x)                      # all products positive: no cancellation
    # per-thread pairs over a grid-stride loop, then the pairs summed in float-float
    pairs = []
    for t in range(threads):
        hi, lo = _f32(0), _f32(0)
        for i in range(t, n, threads):
            hi, lo = _df_add_prod(hi, lo, x[i], y[i])
        pairs.append((hi, lo))
    hi, lo = _f32(0), _f32(0)
    for bh, bl in pairs:
        hi, lo = _df_add(hi, lo, bh, bl)
    got = np.float64(hi) + np.float64(lo)
    exact = math.fsum(float(np.float64(a) * np.float64(b)) for a, b in zip(x, y))
    mag = math.fsum(abs(float(np.float64(a) * np.float64(b))) for a, b in zip(x, y))
    bound = n * 2.0 ** -46 * mag
    assert abs(got - exact) <= bound, (got, exact, bound)
    # and far better than a plain FP32 sum
    plain = _f32(0)
    for a, b in zip(x, y):
        plain = _f32(plain + _f32(a * b))
    assert abs(got - exact) <= 1e-3 * max(abs(float(plain) - exact), 1e-300) or abs(got - exact) <= 1e-12 * mag
