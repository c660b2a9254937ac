"""Oracle: ground state and the shifted linear systems (TEST INFRASTRUCTURE ONLY).

What is computed, and where the paper defines it
------------------------------------------------
* ground_state: |G>, E_G of H (Sec. III; the paper uses Arnoldi, here a plain
  Lanczos with full reorthogonalisation, restarted from its Ritz vector until
  the true eigen-residual ||H G - E_G G|| <= tol * max(1, |E_G|)).
* solve_shifted: Psi_k = (A - w_k I)^{-1} E for every shift independently
  (Eq. 2 rewritten as Eq. A1, A = H' - E_G - i Gamma).  Small systems use a
  sparse LU factorisation (the plain definition); larger ones use BiCGStab,
  the paper's per-w_in baseline (Sec. III), restarted until the true residual
  meets the tolerance.
* msbicg: the multi-shifted BiCG of Eqs. (4)-(8), App. C and Alg. 1 in
  corrected form (bilinear products; the App. C beta convention; the
  (1 - alpha s) sign that systems (A - s I) require; Alg. 1's statements in
  dependency order).  It exists to pin the recurrences themselves; the map
  oracle does not use it.
* dual_bicg: BiCG with an explicitly propagated dual residual in the
  A^dagger space (App. A), used to pin the simplification r~_m = conj(r_m).
* residual_polynomial: P_m(s) from the seed three-term recurrence (Eqs. C6-C7),
  which the paper equates with zeta_m (Eq. C3).
* msbicg_reseeded: the adaptive reseeding of App. E around msbicg (the deviation
  Delta r between the true and the recursive residual of each shift; a rejected
  shift becomes the next seed).

Parity: pinned by tests/test_oracle_solvers.py (dense eigh and the two-site
closed form for the ground state; sparse LU vs BiCGStab vs dense solve; the
MSBiCG solutions against independent solves; zeta_m = P_m(s); collinearity;
r~ = conj(r); finite termination; the 2x2 toy of Fig. 2c).  msbicg_reseeded: by
tests/test_oracle_reseeding.py (a no-op on an accurate run; planted round-off in the
shifted recursions detected by Delta r and repaired by reseeding, checked against
independent solves; shifts left unconverged by maxit reseeded and solved).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def bilinear(u: np.ndarray, v: np.ndarray) -> complex:
    """(u, v) = sum_i u_i v_i with no conjugation: the product that the BiCG
    conditions reduce to once the dual residual is conj(r) (App. A, Eq. A12)."""
    return complex(np.sum(u * v))


def hermitian(u: np.ndarray, v: np.ndarray) -> complex:
    """<u|v> = sum_i conj(u_i) v_i."""
    return complex(np.vdot(u, v))


# ---------------------------------------------------------------------------
# Ground state
# ---------------------------------------------------------------------------
def ground_state(H: sp.spmatrix, v0: np.ndarray, tol: float = 1e-12, kmax: int = 400,
                 max_restarts: int = 20):
    """Lowest eigenpair of real symmetric H by Lanczos with full reorthogonalisation.

    Returns (E_G, G, true_residual) with ||G|| = 1 and G real.
    """
    n = H.shape[0]
    v = np.asarray(v0, dtype=np.float64).copy()
    v /= np.linalg.norm(v)
    for _ in range(max_restarts):
        V = np.zeros((min(kmax, n) + 1, n))
        alpha, beta = [], []
        V[0] = v
        k_used = 0
        for k in range(min(kmax, n)):
            w = H @ V[k]
            a = float(V[k] @ w)
            w = w - a * V[k] - (beta[-1] * V[k - 1] if k > 0 else 0.0)
            # full reorthogonalisation, twice
            for _r in range(2):
                w -= V[:k + 1].T @ (V[:k + 1] @ w)
            b = float(np.linalg.norm(w))
            alpha.append(a)
            beta.append(b)
            k_used = k + 1
            theta, Y = sla.eigh_tridiagonal(np.array(alpha), np.array(beta[:-1]))
            est = abs(b * Y[-1, 0])
            if est <= 0.01 * tol * max(1.0, abs(theta[0])) or b < 1e-300 or k_used == n:
                break
            V[k + 1] = w / b
        theta, Y = sla.eigh_tridiagonal(np.array(alpha), np.array(beta[:k_used - 1]))
        g = V[:k_used].T @ Y[:, 0]
        g /= np.linalg.norm(g)
        E = float(g @ (H @ g))
        res = float(np.linalg.norm(H @ g - E * g))
        if res <= tol * max(1.0, abs(E)):
            return E, g, res
        v = g
    raise RuntimeError(f"ground state did not converge: residual {res:.3e}")


# ---------------------------------------------------------------------------
# Independent shifted solves (the result MSBiCG must reproduce)
# ---------------------------------------------------------------------------
def bicgstab(matvec, b: np.ndarray, tol: float, maxit: int = 20000, x0: np.ndarray | None = None,
             restarts: int = 50, strict: bool = True):
    """BiCGStab (van der Vorst, 1992) for a complex system; shadow residual r0.

    Restarts from the current iterate until the *true* residual
    ||b - A x|| <= tol ||b||.  Returns (x, matvec_count).  With strict=False
    it returns the last iterate instead of raising when `restarts` runs of
    `maxit` iterations do not reach the tolerance (a bounded run, for timing).
    """
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    nmv = 0
    for _restart in range(restarts):
        r = b - matvec(x) if np.any(x) else b.copy()
        nmv += 1 if np.any(x) else 0
        if np.linalg.norm(r) <= tol * nb:
            return x, nmv
        rhat = r.copy()
        rho = alpha = omega = 1.0 + 0j
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        for _ in range(maxit):
            rho_new = hermitian(rhat, r)
            if rho_new == 0:
                break
            beta = (rho_new / rho) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = matvec(p); nmv += 1
            alpha = rho_new / hermitian(rhat, v)
            s = r - alpha * v
            if np.linalg.norm(s) <= 0.1 * tol * nb:
                x = x + alpha * p
                break
            t = matvec(s); nmv += 1
            omega = hermitian(t, s) / hermitian(t, t)
            x = x + alpha * p + omega * s
            r = s - omega * t
            rho = rho_new
            if np.linalg.norm(r) <= 0.1 * tol * nb:
                break
        nmv += 1
        if np.linalg.norm(b - matvec(x)) <= tol * nb:
            return x, nmv
    if not strict:
        return x, nmv
    raise RuntimeError("BiCGStab did not reach the tolerance")


def solve_shifted(A: sp.spmatrix, b: np.ndarray, shifts: np.ndarray, tol: float = 1e-13,
                  method: str = "auto"):
    """x_k = (A - s_k I)^{-1} b for every shift s_k, each solved on its own.

    method: "lu" (sparse LU, the plain definition), "bicgstab" (the paper's
    per-shift baseline), or "auto" (LU for n <= 1000, else BiCGStab).
    Returns (X of shape (n_shifts, n), total matvec count).
    """
    n = A.shape[0]
    if method == "auto":
        method = "lu" if n <= 1000 else "bicgstab"
    A = sp.csc_matrix(A, dtype=np.complex128)
    I = sp.identity(n, dtype=np.complex128, format="csc")
    X = np.zeros((len(shifts), n), dtype=np.complex128)
    nmv = 0
    for k, s in enumerate(shifts):
        M = (A - s * I).tocsc()
        if method == "lu":
            X[k] = spla.splu(M).solve(np.asarray(b, dtype=np.complex128))
        elif method == "bicgstab":
            Mr = M.tocsr()
            X[k], c = bicgstab(lambda v: Mr @ v, np.asarray(b, dtype=np.complex128), tol)
            nmv += c
        else:
            raise ValueError(method)
    return X, nmv


# ---------------------------------------------------------------------------
# The multi-shifted BiCG (App. C, Alg. 1), corrected
# ---------------------------------------------------------------------------
def msbicg(A, b: np.ndarray, shifts: np.ndarray, tol: float, maxit: int,
           zeta_sign: float = -1.0, product: str = "bilinear", record: bool = False,
           keep_residuals: bool = False, zeta_noise: float = 0.0, noise_seed: int = 0):
    """Solve (A - s_k I) x_k = b for all k from one seed recurrence on A.

    A is complex symmetric (A^T = A); `A` may be a sparse matrix or a callable.
    Seed (App. A, Eqs. A13-A15 with the App. C beta convention):
        v = A p_m; alpha_m = (r_m, r_m) / (p_m, v); r_{m+1} = r_m - alpha_m v;
        beta_{m+1} = (r_{m+1}, r_{m+1}) / (r_m, r_m); p_{m+1} = r_{m+1} + beta_{m+1} p_m.
    Shifts (Eqs. C8, C11-C13), with beta_m the coefficient that built p_m:
        zeta_{m+1} = (1 + zeta_sign * alpha_m s) zeta_m + (alpha_m beta_m / alpha_{m-1}) (zeta_m - zeta_{m-1})
        alpha_m^s = (zeta_m / zeta_{m+1}) alpha_m,  beta_m^s = (zeta_{m-1} / zeta_m)^2 beta_m
        p_m^s = r_m / zeta_m + beta_m^s p_{m-1}^s,  x_{m+1}^s = x_m^s + alpha_m^s p_m^s.
    zeta_sign = -1 is the sign that systems (A - s I) require; +1 is the sign
    as printed in Eq. (5) / (C8), kept so a test can show it is wrong; likewise
    product="hermitian" replaces the bilinear products by <u|v> to show that
    the unconjugated form is the one the method needs.
    A shift is frozen when ||r_m|| / |zeta_m| <= tol ||b|| (the shifted residual
    norm by Eq. 4); the loop ends when every shift is frozen or r_m = 0.

    Returns dict(x=(n_shifts, n), iters=per-shift iteration at freeze,
    converged=bool array, m=iterations, and, if record, the seed scalars and
    zeta history).  keep_residuals adds rrec=(n_shifts, n): each shift's recursive
    residual r_m / zeta_m (Eq. 4) at its freeze (or at the last iteration).
    zeta_noise > 0 is a planted fault for tests: each zeta_{m+1} is multiplied by
    1 + zeta_noise |s| (g1 + i g2) with Gaussian g, an emulation of the round-off
    that accumulates in the shifted recursions far from the seed (Sec. III, App. E).
    """
    mv = A if callable(A) else (lambda v: A @ v)
    dot = bilinear if product == "bilinear" else hermitian
    s = np.asarray(shifts, dtype=np.complex128)
    ns, n = len(s), len(b)
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros((ns, n), dtype=np.complex128)
    ps = np.zeros((ns, n), dtype=np.complex128)     # p_{m-1}^s
    r = b.copy()
    p = b.copy()
    rho = dot(r, r)
    zeta_prev = np.ones(ns, dtype=np.complex128)    # zeta_{m-1}
    zeta = np.ones(ns, dtype=np.complex128)         # zeta_m
    alpha_prev = 1.0 + 0j                           # alpha_{-1}
    beta = 0.0 + 0j                                 # beta_0 (p_0 = r_0)
    active = np.ones(ns, dtype=bool)
    iters = np.zeros(ns, dtype=np.int64)
    rrec = np.zeros((ns, n), dtype=np.complex128) if keep_residuals else None
    noise = np.random.default_rng(noise_seed) if zeta_noise > 0 else None
    hist = dict(alpha=[], beta=[], zeta=[zeta.copy()], rnorm=[np.linalg.norm(r)])
    m = 0
    # shifts already converged at m = 0 (only if b = 0)
    rn = np.linalg.norm(r)
    active &= ~(rn <= tol * nb)
    while m < maxit and active.any() and rn > 0:
        v = mv(p)
        mu = dot(p, v)
        if mu == 0:
            raise ZeroDivisionError("seed breakdown: (p, A p) = 0")
        alpha = rho / mu
        idx = np.nonzero(active)[0]
        zeta_next = ((1 + zeta_sign * alpha * s[idx]) * zeta[idx]
                     + (alpha * beta / alpha_prev) * (zeta[idx] - zeta_prev[idx]))
        if noise is not None:
            g = noise.standard_normal(len(idx)) + 1j * noise.standard_normal(len(idx))
            zeta_next = zeta_next * (1 + zeta_noise * np.abs(s[idx]) * g)
        if np.any(zeta_next == 0):
            raise ZeroDivisionError("shift breakdown: zeta_{m+1} = 0")
        alpha_s = (zeta[idx] / zeta_next) * alpha
        beta_s = (zeta_prev[idx] / zeta[idx]) ** 2 * beta
        ps[idx] = r[None, :] / zeta[idx, None] + beta_s[:, None] * ps[idx]
        x[idx] += alpha_s[:, None] * ps[idx]
        zeta_prev[idx] = zeta[idx]
        zeta[idx] = zeta_next
        r = r - alpha * v
        rho_next = dot(r, r)
        beta = rho_next / rho
        rho = rho_next
        p = r + beta * p
        alpha_prev = alpha
        m += 1
        rn = np.linalg.norm(r)
        iters[idx] = m
        done = rn / np.abs(zeta[idx]) <= tol * nb
        if keep_residuals:
            rrec[idx[done]] = r[None, :] / zeta[idx[done], None]
        active[idx[done]] = False
        if record:
            hist["alpha"].append(alpha); hist["beta"].append(beta)
            hist["zeta"].append(zeta.copy()); hist["rnorm"].append(rn)
    converged = ~active | (rn == 0)
    out = dict(x=x, iters=iters, converged=converged, m=m, r=r, zeta=zeta)
    if keep_residuals:
        rest = np.nonzero(active)[0]
        rrec[rest] = r[None, :] / zeta[rest, None]
        out["rrec"] = rrec
    if record:
        out["hist"] = hist
    return out


def msbicg_reseeded(A, b: np.ndarray, shifts: np.ndarray, tol: float, maxit: int, reseed_tol: float,
                    seed_index: int = 0, max_seeds: int = 8, **kw):
    """Adaptive reseeding (App. E) around msbicg.

    Solve (A - s_k I) x_k = b for all k.  Start from the seed system A - s_{seed} I.
    After a run, compare for every shift the true residual r_t = b - (A - s_k I) x_k (one
    MVM per shift) with the recursive residual r / zeta that MSBiCG carried (Eq. 4):
    Delta r_k = ||r_t - r / zeta||.  A shift whose Delta r_k exceeds reseed_tol ||b||, or
    that did not converge within maxit, is not accepted.  The rejected shift closest to
    the current seed becomes the next seed, and the rejected shifts are solved again
    from it; accepted shifts keep their solution.  Stops when every shift is accepted or
    after max_seeds seeds.  Reading of "promote the corresponding w_in": with several
    rejected shifts, the one next to the seed's accurate region (closest to the seed),
    as in the paper's example (seed -4t, then 0).

    Returns dict(x, seeds=list of seed indices, dr=Delta r per shift (last run that
    solved it), accepted=bool array, runs=list of (seed, shifts solved)).
    """
    mv = A if callable(A) else (lambda v: A @ v)
    s = np.asarray(shifts, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ns, n = len(s), len(b)
    nb = np.linalg.norm(b)
    x = np.zeros((ns, n), dtype=np.complex128)
    dr = np.full(ns, np.inf)
    accepted = np.zeros(ns, dtype=bool)
    seeds, runs = [], []
    todo = np.arange(ns)
    s0 = int(seed_index)
    while todo.size and len(seeds) < max_seeds:
        seeds.append(s0)
        runs.append((s0, todo.copy()))
        sigma = s[s0]
        res = msbicg(lambda v, sigma=sigma: mv(v) - sigma * v, b, s[todo] - sigma, tol, maxit,
                     keep_residuals=True, **kw)
        rejected = []
        for j, k in enumerate(todo):
            xk = res["x"][j]
            rt = b - (mv(xk) - s[k] * xk)
            dr[k] = np.linalg.norm(rt - res["rrec"][j])
            x[k] = xk
            ok = bool(res["converged"][j]) and dr[k] <= reseed_tol * nb
            accepted[k] = ok
            if not ok:
                rejected.append(int(k))
        if not rejected:
            break
        s0 = min(rejected, key=lambda k: abs(s[k] - sigma))
        todo = np.array(rejected)
    return dict(x=x, seeds=seeds, dr=dr, accepted=accepted, runs=runs)


def residual_polynomial(alphas, betas, z: complex, m: int) -> complex:
    """P_m(z) of Eq. (C1) from the seed three-term recurrence (Eqs. C6-C7):
    P_{k+1}(z) = -alpha_k z P_k + (1 + alpha_k beta_k / alpha_{k-1}) P_k
                 - (alpha_k beta_k / alpha_{k-1}) P_{k-1},  P_0 = 1, P_{-1} = 1,
    where beta_k is the coefficient that built p_k (beta_0 = 0, alpha_{-1} = 1).
    `alphas[k]` = alpha_k; `betas[k]` = coefficient computed after step k, i.e.
    the one that builds p_{k+1}."""
    P_prev, P = 1.0 + 0j, 1.0 + 0j
    a_prev = 1.0 + 0j
    for k in range(m):
        bk = betas[k - 1] if k > 0 else 0.0
        c = alphas[k] * bk / a_prev
        P_prev, P = P, -alphas[k] * z * P + (1 + c) * P - c * P_prev
        a_prev = alphas[k]
    return P


def dual_bicg(A: np.ndarray, b: np.ndarray, m: int):
    """BiCG with an explicitly propagated dual system (App. A, Eqs. A4-A11):
    primal r, p on A and dual r~, p~ on A^dagger, Hermitian products
    <r~_j | r_i>.  Returns the lists of primal and dual residuals."""
    A = np.asarray(A)
    Ad = A.conj().T
    r = b.astype(np.complex128).copy()
    rt = b.astype(np.complex128).copy()           # r~_0 = b - A^dag * 0 (Eq. A6)
    p, pt = r.copy(), rt.copy()
    R, RT = [r.copy()], [rt.copy()]
    for _ in range(m):
        rho = hermitian(rt, r)
        v = A @ p
        alpha = rho / hermitian(pt, v)
        r = r - alpha * v
        rt = rt - np.conj(alpha) * (Ad @ pt)
        beta = hermitian(rt, r) / rho
        p = r + beta * p
        pt = rt + np.conj(beta) * pt
        R.append(r.copy()); RT.append(rt.copy())
    return R, RT
