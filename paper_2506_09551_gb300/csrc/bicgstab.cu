// Per-incident-energy BiCGStab on the device: the paper's baseline method for
// Eq. 2 (Sec. III, Fig. 4), one independent Krylov space per shift.
//
// Systems (A + c0 - s_k I) x_k = b, solved by BiCGStab (van der Vorst, 1992) with
// x_0 = 0 and the shadow residual r^ = r_0 = b.  All shifts advance together (each
// kernel launch covers every active shift, blockIdx.y = shift), each with its own
// scalars:
//   rho = <r^|r>;  beta = (rho / rho_prev)(alpha / omega);  p = r + beta (p - omega v)
//   v = A_k p;      alpha = rho / <r^|v>;                    s = r - alpha v
//   t = A_k s;      omega = <t|s> / <t|t>;                   x += alpha p + omega s;  r = s - omega t
// with Hermitian products, and a shift stops once ||r|| <= tol ||b||.  On a
// breakdown (<r^|v> or <r^|r> vanishing against ||r^|| ||v||, omega = 0, or a
// non-finite scalar) the shift restarts from its current iterate: r = b - A_k x
// (one more product), r^ = p = r, as the oracle's BiCGStab does; each shift keeps
// its own shadow vector for that.  Two operator applications per iteration per
// shift: the MVM count the paper compares with MSBiCG's one per iteration for all
// shifts (Sec. II).
#include <chrono>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "msbicg_impl.cuh"
#include "profile.cuh"

namespace msb {

struct BcgShift {
    double2 rho, rho_prev, alpha, omega;
    double rnorm, hnorm;   // ||r||, ||r^||
    int active, conv, broken, iters;
    int fresh;             // 1: p = r at the next iteration (start or restart)
    int restart;           // 1: restart from the current iterate before the next iteration
    int restarts;
};

constexpr int kMaxRestarts = 64;
constexpr double kBreakdown = 1e-14;       // relative size of a vanishing product

// Hermitian product <u|v> of FP64 or FP32 vectors, accumulated in FP64.
__device__ __forceinline__ void hdot(double2 u, double2 v, double& re, double& im) { her_acc(u, v, re, im); }
__device__ __forceinline__ void hdot(float2 u, float2 v, double& re, double& im) {
    her_acc(make_double2(u.x, u.y), make_double2(v.x, v.y), re, im);
}

// p = r + beta (p - omega v) (beta = 0 at the first iteration: p = r).
template <typename V>
__global__ void __launch_bounds__(256) k_bcg_p(const V* __restrict__ r, V* __restrict__ p, const V* __restrict__ v,
                                               int64_t n, const BcgShift* __restrict__ sh) {
    const int k = blockIdx.y;
    if (!sh[k].active) return;
    const int64_t off = int64_t(k) * n;
    const bool first = sh[k].fresh;
    double2 beta = make_double2(0.0, 0.0);
    if (!first) beta = cmul(cdiv(sh[k].rho, sh[k].rho_prev), cdiv(sh[k].alpha, sh[k].omega));
    const double2 om = sh[k].omega;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        if (first) {
            p[off + s] = r[off + s];
        } else {
            const V t = vsub(p[off + s], cscale(om.x, om.y, v[off + s]));
            p[off + s] = vadd(r[off + s], cscale(beta.x, beta.y, t));
        }
    }
}

// y = (A + c0 - s_k) x for every active shift; partial <r^|y>, or (<y|z>, ||y||^2)
// with mode 1 (z = the vector the product was taken of).
// mode 2: only the shifts flagged for a restart, no products.
template <class View, typename V>
__global__ void __launch_bounds__(256) k_bcg_apply(View op, const V* __restrict__ x, V* __restrict__ y,
                                                   const V* __restrict__ rhat_all, int64_t n, double c0r, double c0i,
                                                   const double2* __restrict__ shifts,
                                                   const BcgShift* __restrict__ sh, int mode, double* part) {
    __shared__ double sm[3 * 32];
    const int k = blockIdx.y;
    double acc[3] = {0.0, 0.0, 0.0};
    if (mode == 2 && !(sh[k].active && sh[k].restart)) return;
    if (sh[k].active && (mode == 2) == bool(sh[k].restart)) {
        const int64_t off = int64_t(k) * n;
        const V* __restrict__ rhat = rhat_all + off;
        const double er = c0r - shifts[k].x, ei = c0i - shifts[k].y;
        const V* __restrict__ xk = x + off;
        for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
             s += int64_t(gridDim.x) * blockDim.x) {
            const V xs = xk[s];
            const V ys = vadd(op.hx(s, xk, xs), cscale(er, ei, xs));
            y[off + s] = ys;
            if (mode == 0) {
                hdot(rhat[s], ys, acc[0], acc[1]);
                acc[2] += norm2(ys);                   // ||v||^2 for the breakdown test
            } else if (mode == 1) {
                hdot(ys, xs, acc[0], acc[1]);          // <t|s>
                acc[2] += norm2(ys);                   // <t|t>
            }
        }
    }
    if (mode == 2) return;
    store_partials<3>(acc, sm, part);
}

// Restart of the flagged shifts from their current iterate: r = b - y (y = A_k x),
// r^ = r; partial ||r||^2 (the scalar kernel sets rho = ||r||^2, p = r next).
template <typename V>
__global__ void __launch_bounds__(256) k_bcg_restart(const V* __restrict__ b, const V* __restrict__ y,
                                                     V* __restrict__ r, V* __restrict__ rhat, int64_t n,
                                                     const BcgShift* __restrict__ sh, double* part) {
    __shared__ double sm[32];
    const int k = blockIdx.y;
    if (!(sh[k].active && sh[k].restart)) return;
    const int64_t off = int64_t(k) * n;
    double acc[1] = {0.0};
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        const V rs = vsub(b[s], y[off + s]);
        r[off + s] = rs;
        rhat[off + s] = rs;
        acc[0] += norm2(rs);
    }
    store_partials<1>(acc, sm, part);
}

__global__ void k_bcg_restart_scalar(const double* part, int nblk, BcgShift* sh, double thr) {
    __shared__ double sm[32];
    const int k = blockIdx.x;
    if (!(sh[k].active && sh[k].restart)) return;
    double v[1];
    reduce_partials<1>(part + int64_t(k) * nblk, nblk, v, sm);
    if (threadIdx.x != 0) return;
    BcgShift& q = sh[k];
    q.restart = 0;
    q.restarts += 1;
    q.rnorm = sqrt(v[0]);
    q.hnorm = q.rnorm;
    q.rho = make_double2(v[0], 0.0);
    q.rho_prev = make_double2(1.0, 0.0);
    q.alpha = make_double2(1.0, 0.0);
    q.omega = make_double2(1.0, 0.0);
    q.fresh = 1;
    if (q.rnorm <= thr) { q.active = 0; q.conv = 1; }
}

// Per-shift scalar steps.  stage 0: alpha = rho / <r^|v>.  stage 1: omega = <t|s> / <t|t>.
// stage 2: rho_new = <r^|r>, ||r||, convergence, iteration count.
__global__ void k_bcg_scalar(const double* part, int nblk, BcgShift* sh, int stage, double thr, int maxit,
                             int* nactive) {
    __shared__ double sm[3 * 32];
    const int k = blockIdx.x;
    if (!sh[k].active) return;
    double v[3];
    reduce_partials<3>(part + int64_t(k) * nblk * 3, nblk, v, sm);
    if (threadIdx.x != 0) return;
    BcgShift& q = sh[k];
    if (q.restart) {                            // the rest of this iteration is skipped: restart pending
        if (stage == 2 && q.active) atomicAdd(nactive, 1);
        return;
    }
    auto restart = [&] {
        q.restart = 1;
        if (q.restarts >= kMaxRestarts) { q.active = 0; q.broken = 1; }
    };
    if (stage == 0) {
        const double2 d = make_double2(v[0], v[1]);
        if (!cfinite(d) || cabs(d) <= kBreakdown * q.hnorm * sqrt(v[2])) { restart(); return; }
        q.alpha = cdiv(q.rho, d);
        q.fresh = 0;
    } else if (stage == 1) {
        if (!(v[2] > 0.0)) {                    // t = 0: s = 0, x + alpha p is exact
            q.omega = make_double2(0.0, 0.0);
            return;
        }
        q.omega = make_double2(v[0] / v[2], v[1] / v[2]);
    } else {
        q.rho_prev = q.rho;
        q.rho = make_double2(v[0], v[1]);
        q.rnorm = sqrt(v[2]);
        q.iters += 1;
        if (!isfinite(q.rnorm)) { q.active = 0; q.broken = 1; return; }
        if (q.rnorm <= thr) { q.active = 0; q.conv = 1; return; }
        if (q.iters >= maxit) { q.active = 0; return; }
        const bool stall = cabs(q.rho) <= kBreakdown * q.hnorm * q.rnorm || (q.omega.x == 0.0 && q.omega.y == 0.0) ||
                           !cfinite(q.rho);
        if (stall) restart();
        if (q.active) atomicAdd(nactive, 1);
    }
}

// s = r - alpha v (into r).
template <typename V>
__global__ void __launch_bounds__(256) k_bcg_s(V* __restrict__ r, const V* __restrict__ v, int64_t n,
                                               const BcgShift* __restrict__ sh) {
    const int k = blockIdx.y;
    if (!sh[k].active || sh[k].restart) return;
    const int64_t off = int64_t(k) * n;
    const double2 a = sh[k].alpha;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x)
        r[off + s] = vsub(r[off + s], cscale(a.x, a.y, v[off + s]));
}

// x += alpha p + omega s;  r = s - omega t (s is held in r); partials <r^|r>, ||r||^2.
template <typename V>
__global__ void __launch_bounds__(256) k_bcg_update(V* __restrict__ x, V* __restrict__ r, const V* __restrict__ p,
                                                    const V* __restrict__ t, const V* __restrict__ rhat, int64_t n,
                                                    const BcgShift* __restrict__ sh, double* part) {
    __shared__ double sm[3 * 32];
    const int k = blockIdx.y;
    double acc[3] = {0.0, 0.0, 0.0};
    if (sh[k].active && !sh[k].restart) {
        const int64_t off = int64_t(k) * n;
        const double2 a = sh[k].alpha, o = sh[k].omega;
        for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
             s += int64_t(gridDim.x) * blockDim.x) {
            const V ss = r[off + s];   // s, held in r
            x[off + s] = vadd(x[off + s], vadd(cscale(a.x, a.y, p[off + s]), cscale(o.x, o.y, ss)));
            const V rn = vsub(ss, cscale(o.x, o.y, t[off + s]));
            r[off + s] = rn;
            hdot(rhat[off + s], rn, acc[0], acc[1]);
            acc[2] += norm2(rn);
        }
    }
    store_partials<3>(acc, sm, part);
}

// x = 0, r = b, rho = <b|b>, every shift active.
template <typename V>
__global__ void __launch_bounds__(256) k_bcg_init(const V* __restrict__ b, V* __restrict__ x, V* __restrict__ r,
                                                  V* __restrict__ rhat, int64_t n) {
    const int k = blockIdx.y;
    const int64_t off = int64_t(k) * n;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        x[off + s] = vzero(V{});
        r[off + s] = b[s];
        rhat[off + s] = b[s];
    }
}

__global__ void k_bcg_state(BcgShift* sh, int ns, double bnorm2) {
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        BcgShift q{};
        q.rho = make_double2(bnorm2, 0.0);
        q.rho_prev = make_double2(1.0, 0.0);
        q.alpha = make_double2(1.0, 0.0);
        q.omega = make_double2(1.0, 0.0);
        q.rnorm = sqrt(bnorm2);
        q.hnorm = q.rnorm;
        q.fresh = 1;
        q.active = bnorm2 > 0.0 ? 1 : 0;
        q.conv = bnorm2 > 0.0 ? 0 : 1;
        sh[k] = q;
    }
}

template <typename V>
__global__ void __launch_bounds__(256) k_bcg_norm(const V* __restrict__ b, int64_t n, double* part) {
    __shared__ double sm[32];
    double acc[1] = {0.0};
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x)
        acc[0] += norm2(b[s]);
    store_partials<1>(acc, sm, part);
}

struct BcgResult {
    std::vector<int> iters, conv, restarts;
    std::vector<double> resid;
    int max_iters = 0;
    int64_t matvecs = 0, launches = 0;
    double bnorm = 0;
};

template <typename V, class View>
static void bicgstab_impl(const msb_op* op, const View& view, double2 c0, const void* b,
                          const std::vector<double2>& shifts, double tol, int maxit, void* xout, BcgResult& out,
                          cudaStream_t st) {
    const int64_t n = op->dim;
    const int ns = int(shifts.size());
    const int grid = grid_for(n, 256, 2);
    const double vb = double(n) * sizeof(V);
    V* x = static_cast<V*>(xout);
    DevBuf<V> r(size_t(ns) * n), p(size_t(ns) * n), v(size_t(ns) * n), t(size_t(ns) * n), rh(size_t(ns) * n);
    DevBuf<double2> sh_dev(ns);
    DevBuf<BcgShift> sh(ns);
    DevBuf<double> part(size_t(ns) * grid * 3);
    DevBuf<int> nact(1);
    sh_dev.upload(shifts.data(), ns, st);
    k_bcg_norm<V><<<grid, 256, 0, st>>>((const V*)b, n, part.p);
    std::vector<double> hp(grid);
    MSB_CUDA(cudaMemcpyAsync(hp.data(), part.p, grid * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSB_CUDA(cudaStreamSynchronize(st));
    double b2 = 0;
    for (double q : hp) b2 += q;
    out.bnorm = std::sqrt(b2);
    const double thr = tol * out.bnorm;
    k_bcg_state<<<1, 256, 0, st>>>(sh.p, ns, b2);
    k_bcg_init<V><<<dim3(grid, ns), 256, 0, st>>>((const V*)b, x, r.p, rh.p, n);
    out.launches += 3;
    MSB_LAUNCH_CHECK();
    const dim3 g(grid, ns);
    const double hxf = op->hx_flops();
    int it = 0;
    const int poll = 8;
    int active = b2 > 0.0 ? ns : 0;
    while (active > 0 && it < maxit) {
        MSB_CUDA(cudaMemsetAsync(nact.p, 0, sizeof(int), st));
        for (int j = 0; j < poll && it < maxit; ++j, ++it) {
            {
                // restarts (breakdowns of the previous iteration): r = b - A_k x, r^ = r
                ProfScope ps("bicgstab_restart", st, 0, 0);
                k_bcg_apply<View, V><<<g, 256, 0, st>>>(view, x, v.p, rh.p, n, c0.x, c0.y, sh_dev.p, sh.p, 2, part.p);
                k_bcg_restart<V><<<g, 256, 0, st>>>((const V*)b, v.p, r.p, rh.p, n, sh.p, part.p);
                k_bcg_restart_scalar<<<ns, 256, 0, st>>>(part.p, grid, sh.p, thr);
            }
            { ProfScope ps("bicgstab_vec", st, 3 * vb * active, 0); k_bcg_p<V><<<g, 256, 0, st>>>(r.p, p.p, v.p, n, sh.p); }
            {
                ProfScope ps("bicgstab_mvm", st, 2 * vb * active, hxf * active);
                k_bcg_apply<View, V><<<g, 256, 0, st>>>(view, p.p, v.p, rh.p, n, c0.x, c0.y, sh_dev.p, sh.p, 0,
                                                        part.p);
            }
            { ProfScope ps("bicgstab_scalar", st, 0, 0); k_bcg_scalar<<<ns, 256, 0, st>>>(part.p, grid, sh.p, 0, thr, maxit, nact.p); }
            { ProfScope ps("bicgstab_vec", st, 3 * vb * active, 0); k_bcg_s<V><<<g, 256, 0, st>>>(r.p, v.p, n, sh.p); }
            {
                ProfScope ps("bicgstab_mvm", st, 2 * vb * active, hxf * active);
                k_bcg_apply<View, V><<<g, 256, 0, st>>>(view, r.p, t.p, rh.p, n, c0.x, c0.y, sh_dev.p, sh.p, 1,
                                                        part.p);
            }
            { ProfScope ps("bicgstab_scalar", st, 0, 0); k_bcg_scalar<<<ns, 256, 0, st>>>(part.p, grid, sh.p, 1, thr, maxit, nact.p); }
            { ProfScope ps("bicgstab_vec", st, 6 * vb * active, 0); k_bcg_update<V><<<g, 256, 0, st>>>(x, r.p, p.p, t.p, rh.p, n, sh.p, part.p); }
            if (j == poll - 1 || it == maxit - 1) MSB_CUDA(cudaMemsetAsync(nact.p, 0, sizeof(int), st));
            { ProfScope ps("bicgstab_scalar", st, 0, 0); k_bcg_scalar<<<ns, 256, 0, st>>>(part.p, grid, sh.p, 2, thr, maxit, nact.p); }
            out.launches += 11;
            out.matvecs += 2 * int64_t(active);
            MSB_LAUNCH_CHECK();
        }
        MSB_CUDA(cudaMemcpyAsync(&active, nact.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<BcgShift> hs(ns);
    MSB_CUDA(cudaMemcpyAsync(hs.data(), sh.p, ns * sizeof(BcgShift), cudaMemcpyDeviceToHost, st));
    MSB_CUDA(cudaStreamSynchronize(st));
    out.iters.resize(ns);
    out.conv.resize(ns);
    out.resid.resize(ns);
    out.restarts.resize(ns);
    out.matvecs = 0;
    for (int k = 0; k < ns; ++k) {
        out.iters[k] = hs[k].iters;
        out.conv[k] = hs[k].conv;
        out.resid[k] = out.bnorm > 0 ? hs[k].rnorm / out.bnorm : 0.0;
        out.restarts[k] = hs[k].restarts;
        out.max_iters = std::max(out.max_iters, hs[k].iters);
        out.matvecs += 2 * int64_t(hs[k].iters) + hs[k].restarts;
    }
}

}  // namespace msb

extern "C" msb_status msb_bicgstab_solve(msb_op* A, msb_complex c0, const void* b, const msb_complex* shifts,
                                         int n_shifts, double tol, int maxit, msb_precision prec, void* x,
                                         int* iters, double* resid, int* converged, int* restarts,
                                         msb_solve_info* info, void* stream) {
    msb_status result = MSB_OK;
    msb_status g = msb::guard("msb_bicgstab_solve", [&] {
        msb::require_device();
        MSB_REQUIRE(A != nullptr && b != nullptr && x != nullptr && shifts != nullptr, "NULL argument");
        MSB_REQUIRE(prec == MSB_FP64 || prec == MSB_FP32_MIXED, "unknown precision");
        MSB_REQUIRE(n_shifts >= 1 && n_shifts <= 65535, "n_shifts must be in 1..65535");
        MSB_REQUIRE(tol >= 0.0 && maxit >= 0, "tol and maxit must be >= 0");
        auto t0 = std::chrono::steady_clock::now();
        msb::g_alloc_bytes = 0;
        std::vector<double2> s(n_shifts);
        for (int k = 0; k < n_shifts; ++k) s[k] = make_double2(shifts[k].re, shifts[k].im);
        msb::BcgResult out;
        msb::StreamScope scope((cudaStream_t)stream);
        const double2 c = make_double2(c0.re, c0.im);
        if (prec == MSB_FP64) {
            if (A->kind == 0) msb::bicgstab_impl<double2>(A, A->hub, c, b, s, tol, maxit, x, out, scope.s);
            else if (A->kind == 1) msb::bicgstab_impl<double2>(A, A->csr, c, b, s, tol, maxit, x, out, scope.s);
            else msb::bicgstab_impl<double2>(A, A->sum, c, b, s, tol, maxit, x, out, scope.s);
        } else {
            if (A->kind == 0) msb::bicgstab_impl<float2>(A, A->hub, c, b, s, tol, maxit, x, out, scope.s);
            else if (A->kind == 1) msb::bicgstab_impl<float2>(A, A->csr, c, b, s, tol, maxit, x, out, scope.s);
            else msb::bicgstab_impl<float2>(A, A->sum, c, b, s, tol, maxit, x, out, scope.s);
        }
        msb::prof_collect();
        scope.finish();
        int nconv = 0;
        double mx = 0;
        for (int k = 0; k < n_shifts; ++k) {
            if (iters) iters[k] = out.iters[k];
            if (resid) resid[k] = out.resid[k];
            if (converged) converged[k] = out.conv[k];
            if (restarts) restarts[k] = out.restarts[k];
            nconv += out.conv[k];
            mx = std::max(mx, out.resid[k]);
        }
        if (info) {
            *info = msb_solve_info{};
            info->iterations = out.max_iters;
            info->n_converged = nconv;
            info->matvecs = out.matvecs;
            info->max_shift_residual = mx;
            info->seconds_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            info->seconds_total = info->seconds_solve;
            info->device_bytes = msb::g_alloc_bytes;
            info->kernel_launches = out.launches;
        }
        if (nconv < n_shifts) {
            result = MSB_EMAXITER;
            msb::set_error_message("msb_bicgstab_solve: " + std::to_string(n_shifts - nconv) +
                                   " shift(s) did not converge");
        }
    });
    return g != MSB_OK ? g : result;
}
