// Adaptive reseeding around the multi-shift solve (App. E, Fig. 5).
//
// The shifted residuals of MSBiCG are never formed: they follow from the seed
// residual through the zeta recurrence (Eq. 4), whose round-off accumulates for
// shifts far from the seed.  After a solve, every shift's true residual
// b - (A + c0 - s_k) x_k (one operator application per shift) is compared with
// the recursive residual r_m / zeta_m^k that the recurrence carried:
//     Delta r_k = || (b - (A + c0 - s_k) x_k) - r_m / zeta_m^k ||.
// A shift is accepted when it converged and Delta r_k <= reseed_tol ||b||.  The
// rejected shift closest to the current seed becomes the next seed, and the
// rejected shifts are solved again from it (accepted shifts keep their
// solutions), until every shift is accepted or max_seeds seeds were used.
#include <chrono>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "msbicg_impl.cuh"
#include "profile.cuh"

namespace msb {

// Per shift k (blockIdx.y): t = b - (A + c0 - s_k) x_k and d = t - R_k; partial
// sums of ||d||^2 and ||t||^2 in FP64.
template <class View, typename V>
__global__ void __launch_bounds__(256) k_true_resid(View op, const V* __restrict__ b, const V* __restrict__ X,
                                                    const V* __restrict__ R, int64_t n, double c0r, double c0i,
                                                    const double2* __restrict__ shifts, double* part) {
    __shared__ double sm[2 * 32];
    const int k = blockIdx.y;
    const V* __restrict__ xk = X + int64_t(k) * n;
    const V* __restrict__ rk = R + int64_t(k) * n;
    const double2 sk = shifts[k];
    const double er = c0r - sk.x, ei = c0i - sk.y;
    double acc[2] = {0.0, 0.0};
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        const V xs = xk[s];
        const double2 ax = to_d2(vadd(op.hx(s, xk, xs), cscale(er, ei, xs)));
        const double2 bs = to_d2(b[s]), rs = to_d2(rk[s]);
        const double2 t = make_double2(bs.x - ax.x, bs.y - ax.y);
        const double2 d = make_double2(t.x - rs.x, t.y - rs.y);
        acc[0] += norm2(d);
        acc[1] += norm2(t);
    }
    store_partials<2>(acc, sm, part);
}

struct ReseedResult {
    std::vector<int> conv, accepted, seeds;
    std::vector<double> dr, true_resid;
    int iterations = 0;
    int64_t matvecs = 0, launches = 0, flushes = 0;
    double bnorm = 0;
};

template <typename V, class View>
static void true_residuals(const View& view, const void* b, const V* X, const V* R, int64_t n, double2 c0,
                           const std::vector<double2>& sk, std::vector<double>& dr, std::vector<double>& tr,
                           int64_t& launches, cudaStream_t st) {
    const int ns = int(sk.size());
    const int grid = grid_for(n, 256, 2);
    DevBuf<double2> sh(ns);
    DevBuf<double> part(size_t(ns) * grid * 2);
    sh.upload(sk.data(), ns, st);
    {
        ProfScope ps("true_residual", st, 3.0 * double(n) * sizeof(V) * ns, 0.0);
        k_true_resid<View, V><<<dim3(grid, ns), 256, 0, st>>>(view, (const V*)b, X, R, n, c0.x, c0.y, sh.p, part.p);
    }
    ++launches;
    MSB_LAUNCH_CHECK();
    std::vector<double> hp(size_t(ns) * grid * 2);
    MSB_CUDA(cudaMemcpyAsync(hp.data(), part.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSB_CUDA(cudaStreamSynchronize(st));
    dr.assign(ns, 0.0);
    tr.assign(ns, 0.0);
    for (int k = 0; k < ns; ++k) {
        double a = 0, c = 0;
        for (int g = 0; g < grid; ++g) {
            a += hp[(size_t(k) * grid + g) * 2];
            c += hp[(size_t(k) * grid + g) * 2 + 1];
        }
        dr[k] = std::sqrt(a);
        tr[k] = std::sqrt(c);
    }
}

template <typename V>
static void reseeded_impl(msb_op* A, double2 c0, const void* b, const std::vector<double2>& s, double tol, int maxit,
                          int block, msb_precision prec, double reseed_tol, int seed0, int max_seeds, void* x,
                          ReseedResult& out, cudaStream_t st) {
    const int ns = int(s.size());
    const int64_t n = A->dim;
    out.conv.assign(ns, 0);
    out.accepted.assign(ns, 0);
    out.dr.assign(ns, INFINITY);
    out.true_resid.assign(ns, INFINITY);
    std::vector<int> todo(ns);
    for (int k = 0; k < ns; ++k) todo[k] = k;
    int sidx = seed0;
    DevBuf<V> Xt(size_t(ns) * n), Rt(size_t(ns) * n);
    while (!todo.empty() && int(out.seeds.size()) < max_seeds) {
        out.seeds.push_back(sidx);
        const double2 sig = s[sidx];
        const int nt = int(todo.size());
        SolveProblem pr;
        pr.n = n;
        pr.ns = nt;
        pr.b = b;
        pr.x = Xt.p;
        pr.n_out = n;
        pr.rrec = Rt.p;
        pr.c0 = make_double2(c0.x - sig.x, c0.y - sig.y);
        pr.tol = tol;
        pr.maxit = maxit;
        pr.block = block;
        pr.prec = prec;
        std::vector<double2> sk(nt);
        pr.shifts.resize(nt);
        for (int j = 0; j < nt; ++j) {
            sk[j] = s[todo[j]];
            pr.shifts[j] = make_double2(sk[j].x - sig.x, sk[j].y - sig.y);
        }
        SolveResult res;
        multishift_solve(A, pr, res, st);
        if (res.status == MSB_ENONFINITE) fail(MSB_ENONFINITE, "non-finite recurrence scalar in a reseeded run");
        out.iterations += res.iterations;
        out.matvecs += res.iterations + nt;
        out.launches += res.launches;
        out.flushes += res.flushes;
        out.bnorm = res.bnorm;
        std::vector<double> dr, tr;
        if (res.iterations == 0) {
            // nothing ran (b = 0 or maxit = 0): x = 0 and the recursive residual is b
            for (int j = 0; j < nt; ++j)
                MSB_CUDA(cudaMemcpyAsync(Rt.p + size_t(j) * n, b, n * sizeof(V), cudaMemcpyDeviceToDevice, st));
        }
        if (A->kind == 0) true_residuals<V>(A->hub, b, Xt.p, Rt.p, n, c0, sk, dr, tr, out.launches, st);
        else if (A->kind == 1) true_residuals<V>(A->csr, b, Xt.p, Rt.p, n, c0, sk, dr, tr, out.launches, st);
        else true_residuals<V>(A->sum, b, Xt.p, Rt.p, n, c0, sk, dr, tr, out.launches, st);
        std::vector<int> rejected;
        for (int j = 0; j < nt; ++j) {
            const int k = todo[j];
            MSB_CUDA(cudaMemcpyAsync(static_cast<V*>(x) + size_t(k) * n, Xt.p + size_t(j) * n, n * sizeof(V),
                                     cudaMemcpyDeviceToDevice, st));
            out.conv[k] = res.conv[j];
            out.dr[k] = dr[j];
            out.true_resid[k] = tr[j];
            const bool ok = res.conv[j] != 0 && dr[j] <= reseed_tol * res.bnorm;
            out.accepted[k] = ok ? 1 : 0;
            if (!ok) rejected.push_back(k);
        }
        if (rejected.empty()) break;
        // the rejected shift closest to the current seed (first in order on a tie)
        int best = rejected[0];
        double bd = std::hypot(s[best].x - sig.x, s[best].y - sig.y);
        for (int k : rejected) {
            const double d = std::hypot(s[k].x - sig.x, s[k].y - sig.y);
            if (d < bd) { bd = d; best = k; }
        }
        sidx = best;
        todo = rejected;
    }
    MSB_CUDA(cudaStreamSynchronize(st));
}

}  // namespace msb

extern "C" msb_status msb_multishift_bicg_reseeded(msb_op* A, msb_complex c0, const void* b,
                                                   const msb_complex* shifts, int n_shifts, double tol, int maxit,
                                                   int block, msb_precision prec, double reseed_tol, int seed_index,
                                                   int max_seeds, void* x, int* converged, int* accepted, double* dr,
                                                   int* seeds, int* n_seeds, msb_solve_info* info, void* stream) {
    msb_status result = MSB_OK;
    msb_status g = msb::guard("msb_multishift_bicg_reseeded", [&] {
        msb::require_device();
        MSB_REQUIRE(A != nullptr && b != nullptr && x != nullptr && shifts != nullptr, "NULL argument");
        MSB_REQUIRE(prec == MSB_FP64 || prec == MSB_FP32_MIXED, "unknown precision");
        MSB_REQUIRE(n_shifts >= 1 && n_shifts <= msb::kMaxShifts, "n_shifts must be in 1..4096");
        MSB_REQUIRE(tol >= 0.0 && maxit >= 0, "tol and maxit must be >= 0");
        MSB_REQUIRE(reseed_tol > 0.0, "reseed_tol must be > 0");
        MSB_REQUIRE(seed_index >= 0 && seed_index < n_shifts, "seed_index out of range");
        MSB_REQUIRE(max_seeds >= 1, "max_seeds must be >= 1");
        auto t0 = std::chrono::steady_clock::now();
        msb::g_alloc_bytes = 0;
        std::vector<double2> s(n_shifts);
        for (int k = 0; k < n_shifts; ++k) s[k] = make_double2(shifts[k].re, shifts[k].im);
        msb::ReseedResult out;
        msb::StreamScope scope((cudaStream_t)stream);
        const int B = msb::pick_block(block, prec, A->dim, n_shifts);
        if (prec == MSB_FP64)
            msb::reseeded_impl<double2>(A, make_double2(c0.re, c0.im), b, s, tol, maxit, B, prec, reseed_tol,
                                        seed_index, max_seeds, x, out, scope.s);
        else
            msb::reseeded_impl<float2>(A, make_double2(c0.re, c0.im), b, s, tol, maxit, B, prec, reseed_tol,
                                       seed_index, max_seeds, x, out, scope.s);
        scope.finish();
        int n_acc = 0;
        for (int k = 0; k < n_shifts; ++k) {
            if (converged) converged[k] = out.conv[k];
            if (accepted) accepted[k] = out.accepted[k];
            if (dr) dr[k] = out.dr[k];
            n_acc += out.accepted[k];
        }
        if (seeds) for (size_t i = 0; i < out.seeds.size(); ++i) seeds[i] = out.seeds[i];
        if (n_seeds) *n_seeds = int(out.seeds.size());
        if (info) {
            *info = msb_solve_info{};
            info->iterations = out.iterations;
            info->n_converged = n_acc;
            info->matvecs = out.matvecs;
            info->flushes = out.flushes;
            double mx = 0;
            for (double r : out.true_resid) mx = std::isfinite(r) && r > mx ? r : mx;
            info->max_shift_residual = out.bnorm > 0 ? mx / out.bnorm : 0.0;
            info->seconds_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            info->seconds_total = info->seconds_solve;
            info->device_bytes = msb::g_alloc_bytes;
            info->kernel_launches = out.launches;
        }
        if (n_acc < n_shifts) {
            result = MSB_EMAXITER;
            msb::set_error_message("msb_multishift_bicg_reseeded: " + std::to_string(n_shifts - n_acc) +
                                   " shift(s) not accepted after " + std::to_string(out.seeds.size()) + " seed(s)");
        }
    });
    return g != MSB_OK ? g : result;
}
