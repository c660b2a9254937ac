// Multi-shifted BiCG on the device (App. C; Alg. 1 in corrected form).
//
// Systems (A - s_k I) x_k = b, A complex symmetric (A = H' - E_G - i Gamma
// - w_seed in the RIXS map).  One seed recurrence on A, shared by all shifts:
//
//   v = A p_m; mu = (p_m, v); alpha_m = rho_m / mu           (MVM, bilinear product)
//   zeta^k_{m+1} = (1 - alpha_m s_k) zeta^k_m
//                  + (alpha_m beta_m / alpha_{m-1}) (zeta^k_m - zeta^k_{m-1})        (Eq. 5, sign fixed)
//   r_{m+1} = r_m - alpha_m v; rho_{m+1} = (r_{m+1}, r_{m+1}); beta_{m+1} = rho_{m+1}/rho_m
//   p_{m+1} = r_{m+1} + beta_{m+1} p_m
//
// (.,.) is the bilinear product sum u_i v_i (App. A: the dual residual is
// conj(r), so the BiCG conditions need no conjugation).  beta_m is the
// coefficient that built p_m (App. C convention).
//
// Per shift (Eqs. 6-8), with the search direction stored rescaled as
// P^k_m = zeta^k_m p^k_m so that no 1/zeta multiply touches the vectors:
//   p^k_m = r_m / zeta^k_m + beta^k_m p^k_{m-1},  beta^k_m = (zeta^k_{m-1}/zeta^k_m)^2 beta_m
//     =>  P^k_m = r_m + gamma^k_m P^k_{m-1},      gamma^k_m = beta_m zeta^k_{m-1} / zeta^k_m
//   x^k_{m+1} = x^k_m + alpha^k_m p^k_m,           alpha^k_m = (zeta^k_m / zeta^k_{m+1}) alpha_m
//     =>  x^k_{m+1} = x^k_m + c^k_m P^k_m,         c^k_m = alpha_m / zeta^k_{m+1}
// A shift is frozen when ||r_{m+1}|| / |zeta^k_{m+1}| <= tol ||b|| (Eq. 4).
//
// Lagged fused update (the GB300 layout of Eqs. 7-8): the scalars gamma, c
// of up to `B` consecutive iterations are kept per shift, the seed residuals
// r_{m0..m0+B-1} are kept in a ring, and one kernel then advances P^k and
// x^k over those B iterations in registers: one read and one write of each
// per-shift vector per B iterations instead of per iteration.  The arithmetic
// and its order are exactly those of the per-iteration update.
//
// Exponent management.  The seed residual of a well-placed seed falls far
// faster than the residuals of distant shifts (1e-160 after ~1000 iterations
// at L = 8), so r_m and zeta^k_m leave the FP32 range long before the shifts
// converge, and the FP64 range on long runs.  Everything is linear, so the
// seed vectors r, p, v are stored as S_m times their true values and each
// shift's (zeta_m, zeta_{m-1}) as g_k times theirs, with S_m and g_k powers of
// two (exact scaling: no rounding changes).  Only the scalars see the scales:
//   gamma~ = gamma * S_m / S_{m-1},   c~ = c / S_m = alpha 2^{E_k} / zeta~_{m+1},
//   ||r^k_m|| = ||r~_m|| 2^{E_k} / |zeta~_m|,      E_k = log2(g_k / S_m).
#include <chrono>
#include <cmath>
#include <memory>

#include "kernels.cuh"
#include "msbicg_impl.cuh"
#include "profile.cuh"

namespace msb {

constexpr int kScalarThreads = 256;

// ---------------------------------------------------------------------------
// Device state
// ---------------------------------------------------------------------------
struct SeedState {
    double2 rho;          // rho_m = (r_m, r_m)
    double2 alpha;        // alpha_m of the current iteration
    double2 alpha_prev;   // alpha_{m-1} (1 before the first iteration)
    double2 beta;         // beta_m: built p_m (0 at m = 0)
    double rnorm;         // ||r_m||
    double bnorm;         // ||b||
    double tol;
    int m;                // iteration count
    int m0;               // iteration at the start of the current block
    int j;                // iterations in the current block
    int slot;             // ring slot holding r_m
    int done;
    int status;           // msb_status of the recurrence
    int maxit;
    int nactive;
    int fexp;             // r~_m, p~_m were rescaled by 2^fexp after r_m was formed
    int sexp;             // log2 S_m (for reporting the true seed residual)
    int flush_J, flush_cnt, flush_first;   // work of the last fused update (profiling)
};

// ---------------------------------------------------------------------------
// Kernels of one iteration.  All of them return at once once state->done.
// ---------------------------------------------------------------------------

// v = A p (A = op + c0), partial mu = (p, v).
// Dual form (pt != null, App. A): mu = <p~|v> (Hermitian) instead of (p, v).
template <class View, typename V>
__global__ void __launch_bounds__(256) k_mvm_dot(View op, const V* __restrict__ p, V* __restrict__ v,
                                                 int64_t n, double c0r, double c0i,
                                                 const SeedState* __restrict__ st, double* part,
                                                 const V* __restrict__ pt) {
    if (st->done) return;
    __shared__ double sm[2 * 32];
    double acc[2] = {0.0, 0.0};
    DF4 df;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x) {
        const V ps = p[s];
        const V h = op.hx(s, p, ps);
        const V vs = vadd(h, cscale(c0r, c0i, ps));
        v[s] = vs;
        if (pt) {
            if constexpr (std::is_same<V, float2>::value) her_acc_df(pt[s], vs, df);
            else her_acc(pt[s], vs, acc[0], acc[1]);
        } else {
            if constexpr (std::is_same<V, float2>::value) bil_acc_df(ps, vs, df);
            else bil_acc(ps, vs, acc[0], acc[1]);
        }
    }
    if constexpr (std::is_same<V, float2>::value) {
        acc[0] = df_value(df.rh, df.rl);
        acc[1] = df_value(df.ih, df.il);
    }
    store_partials<2>(acc, sm, part);
}

// Dual-space product v~ = (A + c0*) p~ = (A + c0)^dagger p~ for Hermitian A (App. A).
template <class View, typename V>
__global__ void __launch_bounds__(256) k_dual_mvm(View op, const V* __restrict__ pt, V* __restrict__ vt, int64_t n,
                                                  double c0r, double c0i, const SeedState* __restrict__ st) {
    if (st->done) return;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        const V ps = pt[s];
        vt[s] = vadd(op.hx(s, pt, ps), cscale(c0r, -c0i, ps));
    }
}

// alpha, and every active shift's zeta / gamma / c for block position j.
template <typename C>
__global__ void __launch_bounds__(kScalarThreads) k_scalar_a(SeedState* st, const double* part, int nblk,
                                                             ShiftArrays sh, int ns, int B) {
    if (st->done) return;
    __shared__ double sm[2 * 32];
    __shared__ double2 s_alpha;
    __shared__ int s_bad;
    double mu[2];
    reduce_partials<2>(part, nblk, mu, sm);
    if (threadIdx.x == 0) {
        const double2 m2 = make_double2(mu[0], mu[1]);
        s_bad = 0;
        if (!cfinite(m2)) {
            st->status = MSB_ENONFINITE; st->done = 1; s_bad = 1;
        } else if (m2.x == 0.0 && m2.y == 0.0) {
            st->status = MSB_EBREAKDOWN; st->done = 1; s_bad = 1;
        } else {
            const double2 a = cdiv(st->rho, m2);
            if (!cfinite(a)) { st->status = MSB_ENONFINITE; st->done = 1; s_bad = 1; }
            st->alpha = a;
            s_alpha = a;
        }
    }
    __syncthreads();
    if (s_bad) return;
    const double2 alpha = s_alpha;
    const double2 beta = st->beta;
    const double2 ab_over = cdiv(cmul(alpha, beta), st->alpha_prev);   // alpha_m beta_m / alpha_{m-1}
    const int j = st->j;
    const int fexp = st->fexp;
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        if (!sh.active[k]) continue;
        const double2 z = sh.zeta[k], zp = sh.zeta_prev[k], s = sh.shift[k];
        // (1 - alpha s) z + (alpha beta / alpha_prev)(z - zp)
        const double2 one_m = make_double2(1.0 - (alpha.x * s.x - alpha.y * s.y), -(alpha.x * s.y + alpha.y * s.x));
        const double2 zn = cadd(cmul(one_m, z), cmul(ab_over, csub(z, zp)));
        if (!(zn.x != 0.0 || zn.y != 0.0) || !cfinite(zn)) {
            // shift breakdown: freeze it, not converged
            sh.active[k] = 0;
            sh.broken[k] = 1;
            continue;
        }
        // beta_m zeta_{m-1} / zeta_m, times S_m / S_{m-1}
        double2 gamma = cdiv(cmul(beta, zp), z);
        gamma = make_double2(ldexp(gamma.x, fexp), ldexp(gamma.y, fexp));
        // alpha_m / zeta_{m+1} / S_m
        double2 c = cdiv(alpha, zn);
        c = make_double2(ldexp(c.x, sh.zexp[k]), ldexp(c.y, sh.zexp[k]));
        const int64_t o = int64_t(k) * B + j;
        sh.coef64[2 * o] = gamma;
        sh.coef64[2 * o + 1] = c;
        reinterpret_cast<C*>(sh.coefv)[2 * o] = from_d2<C>(gamma);
        reinterpret_cast<C*>(sh.coefv)[2 * o + 1] = from_d2<C>(c);
        sh.nblk[k] = j + 1;
        // keep zeta~ near 1: rescale the pair (zeta_{m+1}, zeta_m) by 2^q
        const double mag = fmax(fabs(zn.x), fabs(zn.y));
        int q = 0;
        if (mag < 0x1p-30 || mag > 0x1p30) q = -ilogb(mag);
        sh.zeta_prev[k] = make_double2(ldexp(z.x, q), ldexp(z.y, q));
        sh.zeta[k] = make_double2(ldexp(zn.x, q), ldexp(zn.y, q));
        sh.zexp[k] += q;
    }
}

// r_{m+1} = r_m - alpha v (into the next ring slot); partials (r,r), ||r||^2.
// Dual form (rt != null): also r~ <- r~ - conj(alpha) v~, and rho = <r~|r> (Hermitian).
template <typename V>
__global__ void __launch_bounds__(256) k_seed_update(V* ring, const V* __restrict__ v, int64_t n, int nslot,
                                                     const SeedState* __restrict__ st, double* part,
                                                     V* __restrict__ rt, const V* __restrict__ vt) {
    if (st->done) return;
    __shared__ double sm[3 * 32];
    const int cur = st->slot, nxt = (cur + 1) % nslot;
    const V* __restrict__ r = ring + int64_t(cur) * n;
    V* __restrict__ rn = ring + int64_t(nxt) * n;
    const double2 a = st->alpha;
    double acc[3] = {0.0, 0.0, 0.0};
    DF4 df;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x) {
        const V x = vsub(r[s], cscale(a.x, a.y, v[s]));
        rn[s] = x;
        if (rt) {
            const V y = vsub(rt[s], cscale(a.x, -a.y, vt[s]));
            rt[s] = y;
            if constexpr (std::is_same<V, float2>::value) {
                her_acc_df(y, x, df);
                norm_acc_df(x, df);
            } else {
                her_acc(y, x, acc[0], acc[1]);
                acc[2] += norm2(x);
            }
            continue;
        }
        if constexpr (std::is_same<V, float2>::value) {
            bil_acc_df(x, x, df);
            norm_acc_df(x, df);
        } else {
            bil_acc(x, x, acc[0], acc[1]);
            acc[2] += norm2(x);
        }
    }
    if constexpr (std::is_same<V, float2>::value) {
        acc[0] = df_value(df.rh, df.rl);
        acc[1] = df_value(df.ih, df.il);
        acc[2] = df_value(df.nh, df.nl);
    }
    store_partials<3>(acc, sm, part);
}

// beta, convergence of every shift, iteration bookkeeping, seed rescaling.
// The rescale 2^f of r~_{m+1} is committed only if the solve goes on (a finished
// solve keeps r~ as it is), so that fz_coef, the factor from the stored r~_{m+1}
// to each tested shift's recursive residual, matches what the ring holds.
__global__ void __launch_bounds__(kScalarThreads) k_scalar_b(SeedState* st, const double* part, int nblk,
                                                             ShiftArrays sh, int ns, int nslot) {
    if (st->done) return;
    __shared__ double sm[3 * 32];
    __shared__ double s_rn;      // ||r~_{m+1}|| (stored scale S_m)
    __shared__ double2 s_rho;    // (r~_{m+1}, r~_{m+1}) at scale S_m
    __shared__ int s_m, s_stop, s_f;
    double v[3];
    reduce_partials<3>(part, nblk, v, sm);
    if (threadIdx.x == 0) {
        const double2 rho_new = make_double2(v[0], v[1]);
        const double rn = sqrt(v[2]);
        st->slot = (st->slot + 1) % nslot;
        st->m += 1;
        st->j += 1;
        st->alpha_prev = st->alpha;
        s_stop = 0;
        int f = 0;
        if (!cfinite(rho_new) || !isfinite(rn)) {
            st->status = MSB_ENONFINITE; s_stop = 1;
        } else if (rn == 0.0) {
            st->beta = make_double2(0.0, 0.0);        // exact solution: every shift converged
        } else if (rho_new.x == 0.0 && rho_new.y == 0.0) {
            st->status = MSB_EBREAKDOWN; s_stop = 1;   // (r, r) = 0 with r != 0
        } else {
            st->beta = cdiv(rho_new, st->rho);
            // bring ||r~|| back near ||b|| once it drifts by more than 2^20
            const double ratio = rn / st->bnorm;
            if (ratio < 0x1p-20 || ratio > 0x1p20) f = -ilogb(ratio);
        }
        st->rnorm = ldexp(rn, -st->sexp);
        s_rn = rn;
        s_rho = rho_new;
        s_f = f;
        s_m = st->m;
    }
    __syncthreads();
    const double thr = st->tol * st->bnorm;
    int still = 0;
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        if (!sh.active[k]) continue;
        // ||r^k_{m+1}|| = ||r~_{m+1}|| 2^{E_k} / |zeta~_{m+1}|
        const double rk = ldexp(s_rn / cabs(sh.zeta[k]), sh.zexp[k]);
        sh.iters[k] = s_m;
        sh.resid[k] = rk / st->bnorm;
        const double2 iz = cdiv(make_double2(1.0, 0.0), sh.zeta[k]);
        sh.fz_coef[k] = make_double2(ldexp(iz.x, sh.zexp[k]), ldexp(iz.y, sh.zexp[k]));
        sh.fz_iter[k] = s_m;
        if (rk <= thr) { sh.active[k] = 0; sh.conv[k] = 1; }
        else ++still;
    }
    double cnt[1] = {double(still)};
    block_sum<1>(cnt, sm);
    if (threadIdx.x == 0) {
        st->nactive = int(cnt[0]);
        if (s_stop || cnt[0] == 0.0 || s_m >= st->maxit) {
            st->done = 1;
            s_f = 0;                                   // nothing follows: keep r~ unscaled
        }
        const int f = s_f;
        st->rho = make_double2(ldexp(s_rho.x, 2 * f), ldexp(s_rho.y, 2 * f));
        st->fexp = f;
        st->sexp += f;
    }
    __syncthreads();
    if (s_f != 0) {
        // S_{m+1} = S_m 2^f: exponents and residual factors of the shifts tested here
        for (int k = threadIdx.x; k < ns; k += blockDim.x) {
            if (sh.fz_iter[k] != s_m) continue;
            sh.zexp[k] -= s_f;
            const double2 c = sh.fz_coef[k];
            sh.fz_coef[k] = make_double2(ldexp(c.x, -s_f), ldexp(c.y, -s_f));
        }
    }
}

// p = 2^f (r_{m+1} + beta p), r_{m+1} <- 2^f r_{m+1} (exact power-of-two rescale)
// Dual form (rt != null): also p~ = 2^f (r~ + conj(beta) p~), r~ <- 2^f r~.
template <typename V>
__global__ void __launch_bounds__(256) k_update_p(V* ring, V* __restrict__ p, int64_t n,
                                                  const SeedState* __restrict__ st, V* __restrict__ rt,
                                                  V* __restrict__ pt) {
    if (st->done) return;
    V* __restrict__ r = ring + int64_t(st->slot) * n;
    const double2 b = st->beta;
    const int f = st->fexp;
    if (f == 0) {
        for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
             s += int64_t(gridDim.x) * blockDim.x) {
            p[s] = vadd(r[s], cscale(b.x, b.y, p[s]));
            if (rt) pt[s] = vadd(rt[s], cscale(b.x, -b.y, pt[s]));
        }
    } else {
        const double sc = ldexp(1.0, f);
        for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
             s += int64_t(gridDim.x) * blockDim.x) {
            const V rs = r[s];
            p[s] = cscale(sc, 0.0, vadd(rs, cscale(b.x, b.y, p[s])));
            r[s] = cscale(sc, 0.0, rs);
            if (rt) {
                const V ts = rt[s];
                pt[s] = cscale(sc, 0.0, vadd(ts, cscale(b.x, -b.y, pt[s])));
                rt[s] = cscale(sc, 0.0, ts);
            }
        }
    }
}

// Start of a block of iterations: nothing pending for any shift.
__global__ void k_block_begin(SeedState* st, ShiftArrays sh, int ns) {
    for (int k = threadIdx.x; k < ns; k += blockDim.x) sh.nblk[k] = 0;
    if (threadIdx.x == 0) {
        st->m0 = st->m;
        st->j = 0;
    }
}

// Lagged fused per-shift update over the block's iterations (Eqs. 7-8):
// for every shift with pending iterations, P <- r_i + gamma_i P; x <- x + c_i P
// for i = 0 .. nblk[k]-1, P and x held in registers, r_i from the ring.
// Optional row map: element e of the per-shift vectors is seed element
// rows[e / rowlen] * rowlen + e % rowlen (only the rows the caller needs).
// rrec (optional): for a shift that froze in this block, or for every shift with
// pending iterations once the solve is done, its recursive residual at its last
// tested iteration, fz_coef[k] * r~_{fz_iter[k]} (r~ from the ring).
template <typename V, int BMAX>
__global__ void __launch_bounds__(256) k_flush(const V* __restrict__ ring, int nslot, int64_t n_seed,
                                               V* __restrict__ P, V* __restrict__ X, int64_t n_out,
                                               const int32_t* __restrict__ rows, int64_t rowlen,
                                               ShiftArrays sh, int ns, SeedState* __restrict__ st,
                                               V* __restrict__ rrec) {
    __shared__ int s_list[kMaxShifts];
    __shared__ int s_cnt;
    const int m0 = st->m0;
    const int slot0 = ((st->slot - st->j) % nslot + nslot) % nslot;   // slot of r_{m0}
    if (threadIdx.x == 0) {
        int c = 0;
        for (int k = 0; k < ns; ++k)
            if (sh.nblk[k] > 0) s_list[c++] = k;
        s_cnt = c;
        if (blockIdx.x == 0) {
            st->flush_J = st->j;
            st->flush_cnt = c;
            st->flush_first = m0 == 0;
        }
    }
    __syncthreads();
    const int cnt = s_cnt;
    if (cnt == 0) return;
    const bool first = (m0 == 0);
    const V* __restrict__ coef = reinterpret_cast<const V*>(sh.coefv);
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n_out;
         e += int64_t(gridDim.x) * blockDim.x) {
        int64_t src = e;
        if (rows) {
            const int64_t row = e / rowlen;
            src = int64_t(__ldg(rows + row)) * rowlen + (e - row * rowlen);
        }
        V r[BMAX];
#pragma unroll
        for (int i = 0; i < BMAX; ++i) {
            const int sl = (slot0 + i) % nslot;
            r[i] = (i < st->j) ? ring[int64_t(sl) * n_seed + src] : vzero(V{});
        }
        for (int q = 0; q < cnt; ++q) {
            const int k = s_list[q];
            const int J = sh.nblk[k];
            V* __restrict__ Pk = P + int64_t(k) * n_out;
            V* __restrict__ Xk = X + int64_t(k) * n_out;
            V pk = first ? vzero(V{}) : Pk[e];
            V xk = first ? vzero(V{}) : Xk[e];
            const V* ck = coef + int64_t(k) * BMAX * 2;
#pragma unroll
            for (int i = 0; i < BMAX; ++i) {
                if (i < J) {
                    const V g = ck[2 * i], c = ck[2 * i + 1];
                    pk = cfma(g, pk, r[i]);    // P = r_i + gamma_i P
                    xk = cfma(c, pk, xk);      // x = x + c_i P
                }
            }
            Pk[e] = pk;
            Xk[e] = xk;
            if (rrec && (!sh.active[k] || st->done)) {
                const int i = sh.fz_iter[k] - m0;                // 1 .. j
                const V rf = ring[int64_t((slot0 + i) % nslot) * n_seed + src];
                const double2 cf = sh.fz_coef[k];
                rrec[int64_t(k) * n_out + e] = cscale(cf.x, cf.y, rf);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Initialisation: rho = (b,b), ||b||, r_0 = b in ring slot 0, p = b.
// ---------------------------------------------------------------------------
// Dual form (rt != null): r~_0 = p~_0 = b, rho = <b|b>.
template <typename V>
__global__ void __launch_bounds__(256) k_init_vectors(const V* __restrict__ b, V* __restrict__ ring,
                                                      V* __restrict__ p, int64_t n, double* part,
                                                      V* __restrict__ rt, V* __restrict__ pt) {
    __shared__ double sm[3 * 32];
    double acc[3] = {0.0, 0.0, 0.0};
    DF4 df;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x) {
        const V x = b[s];
        ring[s] = x;
        p[s] = x;
        if (rt) {
            rt[s] = x;
            pt[s] = x;
            if constexpr (std::is_same<V, float2>::value) {
                her_acc_df(x, x, df);
                norm_acc_df(x, df);
            } else {
                her_acc(x, x, acc[0], acc[1]);
                acc[2] += norm2(x);
            }
            continue;
        }
        if constexpr (std::is_same<V, float2>::value) {
            bil_acc_df(x, x, df);
            norm_acc_df(x, df);
        } else {
            bil_acc(x, x, acc[0], acc[1]);
            acc[2] += norm2(x);
        }
    }
    if constexpr (std::is_same<V, float2>::value) {
        acc[0] = df_value(df.rh, df.rl);
        acc[1] = df_value(df.ih, df.il);
        acc[2] = df_value(df.nh, df.nl);
    }
    store_partials<3>(acc, sm, part);
}

__global__ void __launch_bounds__(kScalarThreads) k_init_state(SeedState* st, const double* part, int nblk,
                                                               ShiftArrays sh, const double2* shifts, int ns,
                                                               double tol, int maxit) {
    __shared__ double sm[3 * 32];
    double v[3];
    reduce_partials<3>(part, nblk, v, sm);
    __shared__ double s_bn;
    if (threadIdx.x == 0) {
        const double bn = sqrt(v[2]);
        st->rho = make_double2(v[0], v[1]);
        st->alpha = make_double2(1.0, 0.0);
        st->alpha_prev = make_double2(1.0, 0.0);
        st->beta = make_double2(0.0, 0.0);
        st->rnorm = bn;
        st->bnorm = bn;
        st->tol = tol;
        st->m = 0; st->m0 = 0; st->j = 0; st->slot = 0;
        st->status = MSB_OK;
        st->maxit = maxit;
        st->done = (bn == 0.0 || maxit <= 0) ? 1 : 0;
        if (bn != 0.0 && st->rho.x == 0.0 && st->rho.y == 0.0) { st->status = MSB_EBREAKDOWN; st->done = 1; }
        st->nactive = bn == 0.0 ? 0 : ns;
        st->fexp = 0;
        st->sexp = 0;
        s_bn = bn;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        sh.shift[k] = shifts[k];
        sh.zeta[k] = make_double2(1.0, 0.0);
        sh.zeta_prev[k] = make_double2(1.0, 0.0);
        sh.active[k] = s_bn == 0.0 ? 0 : 1;
        sh.conv[k] = s_bn == 0.0 ? 1 : 0;
        sh.broken[k] = 0;
        sh.nblk[k] = 0;
        sh.iters[k] = 0;
        sh.resid[k] = 0.0;
        sh.zexp[k] = 0;
        sh.fz_coef[k] = make_double2(1.0, 0.0);
        sh.fz_iter[k] = 0;
    }
}

// Zero-fill of the per-shift solutions when the solve ends before any iteration.
template <typename V>
__global__ void k_zero(V* x, int64_t n) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x)
        x[s] = vzero(V{});
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
template <typename V>
struct SolverImpl {
    using C = V;
    const SolveProblem& pr;
    cudaStream_t st;
    int nslot, B, grid_vec, grid_flush;
    DevBuf<V> ring, p, v, Pbuf;
    DevBuf<V> rt, pt, vt;     // dual-space vectors (App. A), allocated only for the dual form
    DevBuf<double> part;
    DevBuf<SeedState> state;
    DevBuf<double2> zeta, zeta_prev, shift, coef64;
    DevBuf<C> coefv;
    DevBuf<int> active, conv, broken, nblk, iters, zexp, fz_iter;
    DevBuf<double2> fz_coef;
    DevBuf<double> resid;
    DevBuf<double2> shifts_dev;
    ShiftArrays sh{};
    int64_t launches = 0;

    SolverImpl(const SolveProblem& p_, cudaStream_t s) : pr(p_), st(s) {}

    const msb_op* op = nullptr;
    size_t csz = sizeof(V);

    template <class View>
    void iteration(const View& view) {
        const int64_t n = pr.n;
        const double nb = double(n) * csz;
        {
            ProfScope ps("seed_mvm", st, 2 * nb + op->matrix_bytes(csz), op->hx_flops() + 16.0 * n);
            k_mvm_dot<View, V><<<grid_vec, 256, 0, st>>>(view, p.p, v.p, n, pr.c0.x, pr.c0.y, state.p, part.p, pt.p);
        }
        {
            ProfScope ps("shift_scalars", st, 0, 0);
            k_scalar_a<C><<<1, kScalarThreads, 0, st>>>(state.p, part.p, grid_vec, sh, pr.ns, B);
        }
        if (pr.dual) {
            ProfScope ps("seed_mvm", st, 2 * nb + op->matrix_bytes(csz), op->hx_flops() + 8.0 * n);
            k_dual_mvm<View, V><<<grid_vec, 256, 0, st>>>(view, pt.p, vt.p, n, pr.c0.x, pr.c0.y, state.p);
        }
        {
            ProfScope ps("seed_update", st, (pr.dual ? 6 : 3) * nb, 20.0 * n);
            k_seed_update<V><<<grid_vec, 256, 0, st>>>(ring.p, v.p, n, nslot, state.p, part.p, rt.p, vt.p);
        }
        {
            ProfScope ps("shift_scalars", st, 0, 0);
            k_scalar_b<<<1, kScalarThreads, 0, st>>>(state.p, part.p, grid_vec, sh, pr.ns, nslot);
        }
        {
            ProfScope ps("seed_p", st, 3 * nb, 8.0 * n);
            k_update_p<V><<<grid_vec, 256, 0, st>>>(ring.p, p.p, n, state.p, rt.p, pt.p);
        }
    }

    void flush() {
        ProfScope ps("shift_update", st, 0, 0);
        switch (B) {
#define MSB_FLUSH_CASE(BB)                                                                          \
    case BB:                                                                                        \
        k_flush<V, BB><<<grid_flush, 256, 0, st>>>(ring.p, nslot, pr.n, Pbuf.p, (V*)pr.x, pr.n_out, \
                                                   pr.rows, pr.rowlen, sh, pr.ns, state.p,          \
                                                   (V*)pr.rrec);                                    \
        break;
            MSB_FLUSH_CASE(1) MSB_FLUSH_CASE(2) MSB_FLUSH_CASE(4) MSB_FLUSH_CASE(8) MSB_FLUSH_CASE(16)
#undef MSB_FLUSH_CASE
            default: fail(MSB_EINVAL, "block must be 1, 2, 4, 8 or 16");
        }
    }

    template <class View>
    void one_block_direct(const View& view) {
        {
            ProfScope ps("shift_scalars", st, 0, 0);
            k_block_begin<<<1, kScalarThreads, 0, st>>>(state.p, sh, pr.ns);
        }
        for (int i = 0; i < B; ++i) iteration(view);
        flush();
    }

    template <class View>
    void run(const msb_op* op_, const View& view, SolveResult& out) {
        op = op_;
        const int64_t n = pr.n, ns = pr.ns;
        B = pr.block;
        nslot = B + 1;
        grid_vec = grid_for(n, 256, 8);
        grid_flush = grid_for(pr.n_out, 256, 8);
        ring.alloc(size_t(nslot) * n);
        p.alloc(n);
        v.alloc(n);
        if (pr.dual) { rt.alloc(n); pt.alloc(n); vt.alloc(n); }
        Pbuf.alloc(size_t(ns) * pr.n_out);
        part.alloc(size_t(grid_vec) * 4);
        state.alloc(1);
        zeta.alloc(ns); zeta_prev.alloc(ns); shift.alloc(ns);
        coef64.alloc(size_t(ns) * B * 2);
        coefv.alloc(size_t(ns) * B * 2);
        active.alloc(ns); conv.alloc(ns); broken.alloc(ns); nblk.alloc(ns); iters.alloc(ns); zexp.alloc(ns);
        fz_iter.alloc(ns); fz_coef.alloc(ns);
        resid.alloc(ns);
        shifts_dev.alloc(ns);
        shifts_dev.upload(pr.shifts.data(), ns, st);
        sh = ShiftArrays{zeta.p, zeta_prev.p, shift.p, coef64.p, (void*)coefv.p,
                         active.p, conv.p, broken.p, nblk.p, iters.p, resid.p, zexp.p, fz_coef.p, fz_iter.p};

        {
            ProfScope ps("seed_init", st, 3.0 * n * csz, 12.0 * n);
            k_init_vectors<V><<<grid_vec, 256, 0, st>>>((const V*)pr.b, ring.p, p.p, n, part.p, rt.p, pt.p);
        }
        {
            ProfScope ps("shift_scalars", st, 0, 0);
            k_init_state<<<1, kScalarThreads, 0, st>>>(state.p, part.p, grid_vec, sh, shifts_dev.p, int(ns),
                                                        pr.tol, pr.maxit);
        }
        launches += 2;
        MSB_LAUNCH_CHECK();
        const int64_t per_block = 2 + (pr.dual ? 6 : 5) * int64_t(B);   // kernels per block of iterations
        const int64_t max_blocks = (int64_t(pr.maxit) + B - 1) / B + 1;
        int64_t blocks = 0;
        if (prof_on()) {
            // Profiled: direct launches, one sync per block to attribute the
            // fused update's work (shifts and iterations it carried).
            SeedState hs;
            for (;;) {
                one_block_direct(view);
                launches += per_block;
                ++blocks;
                MSB_CUDA(cudaMemcpyAsync(&hs, state.p, sizeof(SeedState), cudaMemcpyDeviceToHost, st));
                MSB_CUDA(cudaStreamSynchronize(st));
                const double no = double(pr.n_out) * csz;
                prof_patch_last("shift_update", hs.flush_J * no + hs.flush_cnt * (hs.flush_first ? 2.0 : 4.0) * no,
                                16.0 * hs.flush_cnt * hs.flush_J * double(pr.n_out));
                if (hs.done || blocks > max_blocks + 2) break;
            }
            prof_collect();
            out.flushes = blocks;
        } else {

        // One block of B iterations + the fused per-shift update, captured once.
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        MSB_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        k_block_begin<<<1, kScalarThreads, 0, st>>>(state.p, sh, int(ns));
        for (int i = 0; i < B; ++i) iteration(view);
        flush();
        MSB_CUDA(cudaStreamEndCapture(st, &graph));
        MSB_CUDA(cudaGraphInstantiate(&exec, graph, 0));

        HostBuf<SeedState> hstate(2);
        cudaEvent_t ev[2];
        MSB_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        MSB_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        bool finished = false;
        // Two blocks in flight: launch block i, then look at the state copied
        // after block i-1.  Blocks launched after convergence return at once.
        while (!finished) {
            MSB_CUDA(cudaGraphLaunch(exec, st));
            launches += per_block;
            const int slot = int(blocks & 1);
            MSB_CUDA(cudaMemcpyAsync(&hstate.p[slot], state.p, sizeof(SeedState), cudaMemcpyDeviceToHost, st));
            MSB_CUDA(cudaEventRecord(ev[slot], st));
            if (blocks >= 1) {
                MSB_CUDA(cudaEventSynchronize(ev[slot ^ 1]));
                if (hstate.p[slot ^ 1].done) finished = true;
            }
            ++blocks;
            if (blocks > max_blocks + 2) break;
        }
        MSB_CUDA(cudaStreamSynchronize(st));
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        out.flushes = blocks;
        }

        SeedState fs;
        MSB_CUDA(cudaMemcpyAsync(&fs, state.p, sizeof(SeedState), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaStreamSynchronize(st));
        if (fs.m == 0) {   // no iteration ran: solutions are zero
            k_zero<V><<<grid_for(ns * pr.n_out, 256, 8), 256, 0, st>>>((V*)pr.x, ns * pr.n_out);
            launches += 1;
        }
        out.iterations = fs.m;
        out.seed_residual = fs.bnorm > 0 ? fs.rnorm / fs.bnorm : 0.0;
        out.bnorm = fs.bnorm;
        out.iters.resize(ns);
        out.resid.resize(ns);
        out.conv.resize(ns);
        std::vector<int> brk(ns);
        MSB_CUDA(cudaMemcpyAsync(out.iters.data(), iters.p, ns * sizeof(int), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaMemcpyAsync(out.resid.data(), resid.p, ns * sizeof(double), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaMemcpyAsync(out.conv.data(), conv.p, ns * sizeof(int), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaMemcpyAsync(brk.data(), broken.p, ns * sizeof(int), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaStreamSynchronize(st));
        out.status = msb_status(fs.status);
        int nconv = 0;
        for (int k = 0; k < ns; ++k) nconv += out.conv[k];
        out.n_converged = nconv;
        bool any_broken = false;
        for (int k = 0; k < ns; ++k) any_broken |= brk[k] != 0;
        if (out.status == MSB_OK && any_broken) out.status = MSB_EBREAKDOWN;
        if (out.status == MSB_OK && nconv < ns) out.status = MSB_EMAXITER;
        out.launches = launches;
    }
};

void multishift_solve(msb_op* op, const SolveProblem& pr, SolveResult& out, cudaStream_t st) {
    MSB_REQUIRE(pr.ns >= 1 && pr.ns <= kMaxShifts, "n_shifts must be in 1..4096");
    MSB_REQUIRE(pr.dual || !op_has_flux(op),
                "the operator is complex Hermitian (Peierls phases), not complex symmetric: use the dual solver");
    if (pr.prec == MSB_FP64) {
        SolverImpl<double2> s(pr, st);
        if (op->kind == 0) s.run(op, op->hub, out);
        else if (op->kind == 1) s.run(op, op->csr, out);
        else s.run(op, op->sum, out);
    } else {
        SolverImpl<float2> s(pr, st);
        if (op->kind == 0) s.run(op, op->hub, out);
        else if (op->kind == 1) s.run(op, op->csr, out);
        else s.run(op, op->sum, out);
    }
}

int pick_block(int block, msb_precision prec, int64_t n, int ns) {
    if (block == 0) {
        const int t = n > 0 ? tuned_block(n, ns, prec) : 0;
        return t ? t : (prec == MSB_FP64 ? 4 : 8);
    }
    MSB_REQUIRE(block == 1 || block == 2 || block == 4 || block == 8 || block == 16,
                "block must be 0 (auto), 1, 2, 4, 8 or 16");
    return block;
}

}  // namespace msb

// ----------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------
static msb_status solve_entry(const char* fname, bool dual, msb_op* A, msb_complex c0, const void* b,
                              const msb_complex* shifts, int n_shifts, double tol, int maxit, int block,
                              msb_precision prec, void* x, int* iters, double* resid, int* converged,
                              msb_solve_info* info, void* stream) {
    msb_status result = MSB_OK;
    msb_status g = msb::guard(fname, [&] {
        msb::require_device();
        MSB_REQUIRE(A != nullptr && b != nullptr && x != nullptr && shifts != nullptr, "NULL argument");
        MSB_REQUIRE(prec == MSB_FP64 || prec == MSB_FP32_MIXED, "unknown precision");
        MSB_REQUIRE(tol >= 0.0, "tol must be >= 0");
        MSB_REQUIRE(maxit >= 0, "maxit must be >= 0");
        auto t0 = std::chrono::steady_clock::now();
        msb::g_alloc_bytes = 0;
        msb::SolveProblem pr;
        pr.n = A->dim;
        pr.ns = n_shifts;
        pr.b = b;
        pr.x = x;
        pr.n_out = A->dim;
        pr.c0 = make_double2(c0.re, c0.im);
        pr.tol = tol;
        pr.maxit = maxit;
        pr.block = msb::pick_block(block, prec, A->dim, n_shifts);
        pr.prec = prec;
        pr.dual = dual;
        pr.shifts.resize(n_shifts);
        for (int k = 0; k < n_shifts; ++k) pr.shifts[k] = make_double2(shifts[k].re, shifts[k].im);
        msb::SolveResult out;
        msb::StreamScope scope((cudaStream_t)stream);
        msb::multishift_solve(A, pr, out, scope.s);
        scope.finish();
        if (iters) for (int k = 0; k < n_shifts; ++k) iters[k] = out.iters[k];
        if (resid) for (int k = 0; k < n_shifts; ++k) resid[k] = out.resid[k];
        if (converged) for (int k = 0; k < n_shifts; ++k) converged[k] = out.conv[k];
        if (info) {
            *info = msb_solve_info{};
            info->iterations = out.iterations;
            info->n_converged = out.n_converged;
            info->matvecs = (dual ? 2 : 1) * int64_t(out.iterations);
            info->flushes = out.flushes;
            info->seed_residual = out.seed_residual;
            double mx = 0;
            for (double r : out.resid) mx = r > mx ? r : mx;
            info->max_shift_residual = mx;
            info->seconds_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            info->seconds_total = info->seconds_solve;
            info->device_bytes = msb::g_alloc_bytes;
            info->kernel_launches = out.launches;
        }
        result = out.status;
        if (result != MSB_OK)
            msb::set_error_message(std::string(fname) + ": recurrence ended with status " + std::to_string(int(result)));
    });
    return g != MSB_OK ? g : result;
}

extern "C" msb_status msb_multishift_bicg_solve(msb_op* A, msb_complex c0, const void* b,
                                                const msb_complex* shifts, int n_shifts, double tol,
                                                int maxit, int block, msb_precision prec, void* x,
                                                int* iters, double* resid, int* converged,
                                                msb_solve_info* info, void* stream) {
    return solve_entry("msb_multishift_bicg_solve", false, A, c0, b, shifts, n_shifts, tol, maxit, block, prec, x,
                       iters, resid, converged, info, stream);
}

extern "C" msb_status msb_multishift_bicg_dual_solve(msb_op* A, msb_complex c0, const void* b,
                                                     const msb_complex* shifts, int n_shifts, double tol,
                                                     int maxit, int block, msb_precision prec, void* x,
                                                     int* iters, double* resid, int* converged,
                                                     msb_solve_info* info, void* stream) {
    return solve_entry("msb_multishift_bicg_dual_solve", true, A, c0, b, shifts, n_shifts, tol, maxit, block, prec, x,
                       iters, resid, converged, info, stream);
}
