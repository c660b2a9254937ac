// Lanczos on the device: the ground state (Sec. III; FP64, real vectors) and
// the batched continued fraction of the second step (Eq. 1).
//
// Both use the symmetric Lanczos three-term recurrence
//   w = H q_k - b_k q_{k-1};  a_k = <q_k|w>;  w -= a_k q_k;  b_{k+1} = ||w||;  q_{k+1} = w / b_{k+1}
// with the products reduced per block and summed by one CTA in a fixed order,
// so that a rerun reproduces every vector bit for bit (the ground-state
// eigenvector is rebuilt by a second, identical pass).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "msbicg_impl.cuh"
#include "profile.cuh"

namespace msb {

// ---------------------------------------------------------------------------
// Host: lowest eigenpair of the symmetric tridiagonal T (diag a[0..k-1],
// off-diagonal b[0..k-2]) by Sturm bisection and inverse iteration.
// ---------------------------------------------------------------------------
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, int k, double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0) ++cnt;
    }
    return cnt;
}

static void tridiag_lowest(const std::vector<double>& a, const std::vector<double>& b, int k, double& theta,
                           std::vector<double>& y) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 0; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(a, b, k, mid) >= 1) hi = mid; else lo = mid;
    }
    theta = 0.5 * (lo + hi);
    // inverse iteration: solve (T - sigma I) y_new = y with partial pivoting
    const double scale = std::max(1.0, std::fabs(theta));
    const double sigma = theta - 1e-13 * scale;
    y.assign(k, 1.0);
    for (int it = 0; it < 4; ++it) {
        // Gaussian elimination with partial pivoting on a tridiagonal matrix:
        // rows hold (diag, super1, super2) after elimination.
        std::vector<double> d(k), u1(k, 0.0), u2(k, 0.0), l(k, 0.0), rhs(y);
        std::vector<double> sub(k, 0.0), dia(k), sup(k, 0.0);
        for (int i = 0; i < k; ++i) {
            dia[i] = a[i] - sigma;
            if (i + 1 < k) { sup[i] = b[i]; sub[i + 1] = b[i]; }
        }
        // working copies per row: (dia, sup, sup2)
        std::vector<double> r0(k), r1(k), r2(k, 0.0);
        for (int i = 0; i < k; ++i) { r0[i] = dia[i]; r1[i] = sup[i]; }
        for (int i = 0; i + 1 < k; ++i) {
            // rows i and i+1; candidate pivot sub[i+1] in column i
            double s = sub[i + 1];
            if (std::fabs(s) > std::fabs(r0[i])) {
                // swap row i and row i+1 (row i+1 = [s, dia, sup] at columns i, i+1, i+2)
                const double n0 = s, n1 = r0[i + 1], n2 = r1[i + 1];
                const double o0 = r0[i], o1 = r1[i], o2 = r2[i];
                r0[i] = n0; r1[i] = n1; r2[i] = n2;
                std::swap(rhs[i], rhs[i + 1]);
                const double f = o0 / n0;
                r0[i + 1] = o1 - f * n1;
                r1[i + 1] = o2 - f * n2;
                rhs[i + 1] -= f * rhs[i];
            } else {
                const double piv = r0[i] != 0.0 ? r0[i] : 1e-300;
                const double f = s / piv;
                r0[i + 1] -= f * r1[i];
                r1[i + 1] -= f * r2[i];
                rhs[i + 1] -= f * rhs[i];
            }
        }
        for (int i = k - 1; i >= 0; --i) {
            double v = rhs[i];
            if (i + 1 < k) v -= r1[i] * y[i + 1];
            if (i + 2 < k) v -= r2[i] * y[i + 2];
            y[i] = v / (r0[i] != 0.0 ? r0[i] : 1e-300);
        }
        double nrm = 0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        for (double& v : y) v /= nrm;
        (void)d; (void)u1; (void)u2; (void)l;
    }
}

// ---------------------------------------------------------------------------
// Batched Lanczos kernels.  Column c of a block of vectors starts at c * n.
// `cols` lists the active columns (blockIdx.y indexes it).
// ---------------------------------------------------------------------------

// w = H q - b_prev q_prev; partial Re<q|w>.
template <class View, typename V>
__global__ void __launch_bounds__(256) k_lz_apply(View op, const V* __restrict__ q, const V* __restrict__ qp,
                                                  V* __restrict__ w, int64_t n, const int* __restrict__ cols,
                                                  const double* __restrict__ bprev, double* part) {
    __shared__ double sm[32];
    const int c = cols[blockIdx.y];
    const int64_t off = int64_t(c) * n;
    const V* __restrict__ qc = q + off;
    const V* __restrict__ qpc = qp + off;
    V* __restrict__ wc = w + off;
    const double bp = bprev[c];
    double acc[1] = {0.0};
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x) {
        const V qs = qc[s];
        V h = op.hx(s, qc, qs);
        if (bp != 0.0) h = vsub(h, cscale(bp, 0.0, qpc[s]));
        wc[s] = h;
        if constexpr (!is_cplx_v<V>) {
            acc[0] += double(qs) * double(h);
        } else {
            double re = 0, im = 0;
            her_acc(qs, h, re, im);
            acc[0] += re;
        }
    }
    store_partials<1>(acc, sm, part);
}

// a_c = sum of partials (one CTA per active column).
__global__ void k_lz_sum(const double* part, int nblk, const int* cols, double* out, int64_t stride_k, int k) {
    __shared__ double sm[32];
    const int c = cols[blockIdx.x];
    double v[1];
    reduce_partials<1>(part + int64_t(blockIdx.x) * nblk, nblk, v, sm);
    if (threadIdx.x == 0) out[int64_t(k) * stride_k + c] = v[0];
}

// w -= a q; partial ||w||^2.
template <typename V>
__global__ void __launch_bounds__(256) k_lz_orth(const V* __restrict__ q, V* __restrict__ w, int64_t n,
                                                 const int* __restrict__ cols, const double* __restrict__ a,
                                                 double* part) {
    __shared__ double sm[32];
    const int c = cols[blockIdx.y];
    const int64_t off = int64_t(c) * n;
    const double ac = a[c];
    double acc[1] = {0.0};
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x) {
        const V x = vsub(w[off + s], cscale(ac, 0.0, q[off + s]));
        w[off + s] = x;
        acc[0] += norm2(x);
    }
    store_partials<1>(acc, sm, part);
}

// b_c = sqrt(sum); stores b[k][c] and the current b for the next step.
__global__ void k_lz_norm(const double* part, int nblk, const int* cols, double* bstore, int64_t stride_k, int k,
                          double* bcur) {
    __shared__ double sm[32];
    const int c = cols[blockIdx.x];
    double v[1];
    reduce_partials<1>(part + int64_t(blockIdx.x) * nblk, nblk, v, sm);
    if (threadIdx.x == 0) {
        const double b = sqrt(v[0]);
        bstore[int64_t(k) * stride_k + c] = b;
        bcur[c] = b;
    }
}

// w *= 1/b (becomes q_{k+1}); a zero b leaves w (the column is finished).
template <typename V>
__global__ void __launch_bounds__(256) k_lz_scale(V* __restrict__ w, int64_t n, const int* __restrict__ cols,
                                                  const double* __restrict__ bcur) {
    const int c = cols[blockIdx.y];
    const double b = bcur[c];
    if (!(b > 0.0)) return;
    const double inv = 1.0 / b;
    const int64_t off = int64_t(c) * n;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x)
        w[off + s] = cscale(inv, 0.0, w[off + s]);
}

// q_c = x_c / ||x_c|| (start vectors), norms n0[c] = <x_c|x_c>.
template <typename V>
__global__ void __launch_bounds__(256) k_lz_norm_partial(const V* __restrict__ x, int64_t n, const int* cols,
                                                         double* part) {
    __shared__ double sm[32];
    const int c = cols[blockIdx.y];
    const int64_t off = int64_t(c) * n;
    double acc[1] = {0.0};
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x)
        acc[0] += norm2(x[off + s]);
    store_partials<1>(acc, sm, part);
}

template <typename V>
__global__ void __launch_bounds__(256) k_lz_start(const V* __restrict__ x, V* __restrict__ q, V* __restrict__ qp,
                                                  int64_t n, const int* cols, const double* n0) {
    const int c = cols[blockIdx.y];
    const int64_t off = int64_t(c) * n;
    const double nn = n0[c];
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n;
         s += int64_t(gridDim.x) * blockDim.x) {
        q[off + s] = cscale(inv, 0.0, x[off + s]);
        qp[off + s] = vzero(V{});
    }
}

// g += y_k q  (ground-state eigenvector reconstruction; real vectors)
__global__ void k_axpy_real(double* __restrict__ g, const double* __restrict__ q, int64_t n, double y) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x)
        g[s] = fma(y, q[s], g[s]);
}

// Counter-based start vector: splitmix64 of the index mapped to (-1, 1).
__global__ void k_fill_start(double* v, int64_t n, uint64_t seed) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * uint64_t(s + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[s] = (double(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
    }
}

// <g|H g> and ||H g - E g||^2 pieces: partials of (g.Hg, Hg.Hg, g.g) with Hg in `h`.
template <class View>
__global__ void __launch_bounds__(256) k_gs_check(View op, const double* __restrict__ g, double* __restrict__ h,
                                                  int64_t n, double* part) {
    __shared__ double sm[3 * 32];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        const double gs = g[s];
        const double hs = op.hx(s, g, gs);
        h[s] = hs;
        acc[0] += gs * hs;
        acc[1] += hs * hs;
        acc[2] += gs * gs;
    }
    store_partials<3>(acc, sm, part);
}

__global__ void k_gs_resid_partial(const double* __restrict__ g, const double* __restrict__ h, int64_t n, double E,
                                   double* part) {
    __shared__ double sm[32];
    double acc[1] = {0.0};
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        const double r = h[s] - E * g[s];
        acc[0] += r * r;
    }
    store_partials<1>(acc, sm, part);
}

__global__ void k_scale_real(double* g, int64_t n, double f) {
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x)
        g[s] *= f;
}

// ---------------------------------------------------------------------------
// Ground state
// ---------------------------------------------------------------------------
// Device scratch of one ground-state run: three Lanczos vectors, the start
// vector of the current restart, H g for the residual check, the coefficients
// a_k, b_{k+1} (maxit + 1 each), two scalars, the column list and 3 partial
// sums per block.  Allocated by msb_ground_state, carved from a fixed array by
// msb_ground_state_noalloc; the Lanczos run below is the same for both.
struct GroundScratch {
    double* Q;        // 3 n
    double* v0;       // n
    double* hbuf;     // n
    double* a;        // maxit + 1
    double* b;        // maxit + 1
    double* bcur;     // 1
    double* n0;       // 1
    int* col0;        // 1
    double* part;     // 3 * grid
};

template <class View>
static void lanczos_ground(const msb_op* op, const View& view, int64_t n, double tol, int maxit, const double* start,
                           double* g, const GroundScratch& S, int grid, GroundResult& out, cudaStream_t st) {
    const double vb = 8.0 * double(n);                       // one real FP64 vector
    const double hxf = 0.5 * op->hx_flops();
    MSB_CUDA(cudaMemsetAsync(S.col0, 0, sizeof(int), st));
    if (start) MSB_CUDA(cudaMemcpyAsync(S.v0, start, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else { k_fill_start<<<grid, 256, 0, st>>>(S.v0, n, 0x5EEDull); ++out.launches; }
    std::vector<double> ha(maxit + 1), hb(maxit + 1), y;

    // One Lanczos run from v0.  If `accumulate`, g = sum_i y[i] q_i.
    auto run = [&](int kmax, bool accumulate, int& k_done) {
        double* q = S.Q;
        double* qp = S.Q + n;
        double* w = S.Q + 2 * n;
        k_lz_norm_partial<double><<<dim3(grid, 1), 256, 0, st>>>(S.v0, n, S.col0, S.part);
        k_lz_sum<<<1, 256, 0, st>>>(S.part, grid, S.col0, S.n0, 0, 0);
        k_lz_start<double><<<dim3(grid, 1), 256, 0, st>>>(S.v0, q, qp, n, S.col0, S.n0);
        MSB_CUDA(cudaMemsetAsync(S.bcur, 0, sizeof(double), st));
        out.launches += 3;
        if (accumulate) MSB_CUDA(cudaMemsetAsync(g, 0, n * sizeof(double), st));
        int k = 0;
        for (; k < kmax; ++k) {
            if (accumulate) { k_axpy_real<<<grid, 256, 0, st>>>(g, q, n, y[k]); ++out.launches; }
            if (accumulate && k == kmax - 1) break;
            {
                ProfScope ps("ground_state", st, 3 * vb + op->matrix_bytes(8), hxf + 4.0 * n);
                k_lz_apply<View, double><<<dim3(grid, 1), 256, 0, st>>>(view, q, qp, w, n, S.col0, S.bcur, S.part);
            }
            { ProfScope ps("ground_state", st, 0, 0); k_lz_sum<<<1, 256, 0, st>>>(S.part, grid, S.col0, S.a, 1, k); }
            {
                ProfScope ps("ground_state", st, 3 * vb, 4.0 * n);
                k_lz_orth<double><<<dim3(grid, 1), 256, 0, st>>>(q, w, n, S.col0, S.a + k, S.part);
            }
            { ProfScope ps("ground_state", st, 0, 0); k_lz_norm<<<1, 256, 0, st>>>(S.part, grid, S.col0, S.b, 1, k, S.bcur); }
            {
                ProfScope ps("ground_state", st, 2 * vb, 1.0 * n);
                k_lz_scale<double><<<dim3(grid, 1), 256, 0, st>>>(w, n, S.col0, S.bcur);
            }
            out.launches += 5;
            ++out.matvecs;
            MSB_LAUNCH_CHECK();
            std::swap(qp, q);   // q_prev <- q
            std::swap(q, w);    // q <- w (scaled), w <- old q_prev
            if (!accumulate) {
                MSB_CUDA(cudaMemcpyAsync(ha.data(), S.a, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
                MSB_CUDA(cudaMemcpyAsync(hb.data(), S.b, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
                MSB_CUDA(cudaStreamSynchronize(st));
                double theta;
                tridiag_lowest(ha, hb, k + 1, theta, y);
                const double est = std::fabs(hb[k] * y[k]);
                if (est <= 0.01 * tol * std::max(1.0, std::fabs(theta)) || hb[k] <= 1e-300 || k + 1 >= n) {
                    ++k;
                    break;
                }
            }
        }
        k_done = accumulate ? kmax : k;
    };

    out.status = MSB_OK;
    for (int restart = 0; restart < 20; ++restart) {
        int K = 0;
        run(int(std::min<int64_t>(maxit, n)), false, K);
        double theta;
        tridiag_lowest(ha, hb, K, theta, y);
        int K2 = 0;
        run(K, true, K2);
        // E = <g|Hg>/<g|g>, residual ||Hg - E g|| / ||g||
        k_gs_check<View><<<grid, 256, 0, st>>>(view, g, S.hbuf, n, S.part);
        std::vector<double> hp(size_t(grid) * 3);
        MSB_CUDA(cudaMemcpyAsync(hp.data(), S.part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaStreamSynchronize(st));
        double gh = 0, hh = 0, gg = 0;
        for (int b = 0; b < grid; ++b) { gh += hp[3 * b]; hh += hp[3 * b + 1]; gg += hp[3 * b + 2]; }
        const double nrm = std::sqrt(gg);
        k_scale_real<<<grid, 256, 0, st>>>(g, n, 1.0 / nrm);
        k_scale_real<<<grid, 256, 0, st>>>(S.hbuf, n, 1.0 / nrm);
        const double E = gh / gg;
        k_gs_resid_partial<<<grid, 256, 0, st>>>(g, S.hbuf, n, E, S.part);
        std::vector<double> rp(grid);
        MSB_CUDA(cudaMemcpyAsync(rp.data(), S.part, grid * sizeof(double), cudaMemcpyDeviceToHost, st));
        MSB_CUDA(cudaStreamSynchronize(st));
        double rr = 0;
        for (double v : rp) rr += v;
        out.launches += 4;
        ++out.matvecs;
        out.E = E;
        out.residual = std::sqrt(rr);
        out.restarts = restart;
        if (out.residual <= tol * std::max(1.0, std::fabs(E))) return;
        MSB_CUDA(cudaMemcpyAsync(S.v0, g, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    out.status = MSB_EMAXITER;
}

template <class View>
static void ground_state_impl(const msb_op* op, const View& view, int64_t n, double tol, int maxit, const double* start,
                              double* g, GroundResult& out, cudaStream_t st) {
    const int grid = grid_for(n, 256, 8);
    DevBuf<double> Q(3 * size_t(n)), v0(n), hbuf(n), part(size_t(grid) * 3), a_dev(maxit + 1), b_dev(maxit + 1),
        bcur(1), n0(1);
    DevBuf<int> col0(1);
    const GroundScratch S{Q.p, v0.p, hbuf.p, a_dev.p, b_dev.p, bcur.p, n0.p, col0.p, part.p};
    lanczos_ground(op, view, n, tol, maxit, start, g, S, grid, out, st);
}

void ground_state(msb_op* H, double tol, int maxit, const double* start, double* g, GroundResult& out,
                  cudaStream_t st) {
    MSB_REQUIRE(H != nullptr && g != nullptr, "NULL argument");
    MSB_REQUIRE(maxit >= 2, "maxit must be >= 2");
    MSB_REQUIRE(tol > 0, "tol must be > 0");
    MSB_REQUIRE(H->kind != 2, "a direct sum has no single ground state: take each part's");
    MSB_REQUIRE(!op_has_flux(H), "the ground state takes a real symmetric H (no flux)");
    if (H->kind == 0) ground_state_impl(H, H->hub, H->dim, tol, maxit, start, g, out, st);
    else ground_state_impl(H, H->csr, H->dim, tol, maxit, start, g, out, st);
    prof_collect();
}

// ---------------------------------------------------------------------------
// Continued fraction: I(w) = -(1/pi) Im G(E0 + w + i eta),
// G(z) = n0 / (z - a_0 - b_1^2 / (z - a_1 - ...)) cut after level k_to with a
// zero tail (Eq. 1 with the paper's continued-fraction expansion).  The K-th
// convergent is carried forward: each call folds in levels [k_from, k_to) and
// keeps the recurrence state per (column, w), so a run of K levels costs O(K)
// per point instead of O(K^2 / check) for bottom-up re-evaluation at every check.
// One CTA per active column; threads over w.  Also reports the column's
// max |I_new - I_old| and max |I_new|.
// ---------------------------------------------------------------------------
__global__ void k_cf_eval(const double* __restrict__ a, const double* __restrict__ b, int64_t stride_k,
                          const double* __restrict__ n0, const int* __restrict__ cols, int k_from, int k_to,
                          const double* __restrict__ E0c, const double* __restrict__ w, int n_w, double eta,
                          double2* __restrict__ gst, double2* __restrict__ Cst, double2* __restrict__ Dst,
                          double* I, double* diff) {
    __shared__ double sm[2 * 32];
    const int c = cols[blockIdx.x];
    const double E0 = E0c[c];
    double dmax = 0.0, imax = 0.0;
    for (int i = threadIdx.x; i < n_w; i += blockDim.x) {
        const double2 z = make_double2(E0 + w[i], eta);
        const int64_t o = int64_t(c) * n_w + i;
        // g = d_0 + c_1 / (d_1 + c_2 / (d_2 + ...)), d_j = z - a_j, c_j = -b_j^2, by the
        // modified Lentz recurrences C_j = d_j + c_j / C_{j-1}, D_j = 1 / (d_j + c_j D_{j-1}),
        // g_j = g_{j-1} C_j D_j; G = 1 / g.  For Im z > 0 every C_j and 1 / D_j has
        // imaginary part >= eta, so no division by zero.
        double2 g, C, D;
        int j = k_from;
        if (j == 0) {
            g = make_double2(z.x - a[c], z.y);
            C = g;
            D = make_double2(0.0, 0.0);
            j = 1;
        } else {
            g = gst[o];
            C = Cst[o];
            D = Dst[o];
        }
        for (; j < k_to; ++j) {
            const double aj = a[int64_t(j) * stride_k + c];
            const double bj = b[int64_t(j - 1) * stride_k + c];
            const double cj = -bj * bj;
            const double2 d = make_double2(z.x - aj, z.y);
            D = cdiv(make_double2(1.0, 0.0), make_double2(fma(cj, D.x, d.x), fma(cj, D.y, d.y)));
            const double2 ic = cdiv(make_double2(1.0, 0.0), C);
            C = make_double2(fma(cj, ic.x, d.x), fma(cj, ic.y, d.y));
            g = cmul(g, cmul(C, D));
        }
        gst[o] = g;
        Cst[o] = C;
        Dst[o] = D;
        const double2 G = cdiv(make_double2(1.0, 0.0), g);
        const double val = k_to > 0 ? -(n0[c] * G.y) / M_PI : 0.0;
        dmax = fmax(dmax, fabs(val - I[o]));
        imax = fmax(imax, fabs(val));
        I[o] = val;
    }
    // block max via sums of squares is not a max: do a shuffle max instead
    dmax = warp_max(dmax);
    imax = warp_max(imax);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) { sm[wid] = dmax; sm[32 + wid] = imax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double d = 0, m = 0;
        for (int i = 0; i < nw; ++i) { d = fmax(d, sm[i]); m = fmax(m, sm[32 + i]); }
        diff[2 * c] = d;
        diff[2 * c + 1] = m;
    }
}

// ---------------------------------------------------------------------------
// Continued-fraction Lanczos with unnormalised vectors.  Column c stores V_k
// with q_k = sig_k V_k, so no pass rescales a vector:
//   pass A:  W = sig_k (H V_k) - (b_k sig_{k-1}) V_{k-1};   a_k = sig_k Re<V_k|W>
//   pass B:  W -= (a_k sig_k) V_k;                           b_{k+1} = ||W||
//   then V_{k+1} = W, sig_{k+1} = 1 / b_{k+1} (0 once the Krylov space is exhausted).
// Columns are stored with a stride `ld` (n rounded up to 2) for 16-byte loads;
// the padding stays zero.  In the FP32 path every product is accumulated with
// the compensated FP32 scheme of df_add_prod (no per-element FP64 work).
// ---------------------------------------------------------------------------
struct CFCoef {
    double* sig;      // sig_k per column
    double* cB;       // b_k sig_{k-1} per column (0 at k = 0)
    double* cC;       // a_k sig_k per column
    float* sigf;      // the same three rounded to FP32, for the FP32 kernels
    float* cBf;
    float* cCf;
};

constexpr int kMaxHops = 32;     // up-spin hops per row (a 2D 3 x 4 cluster has 24 bonds)

// Pass A for the Hubbard operator, one CTA per (row u, active column): row u
// of V_k is staged in shared memory (own values and the down-spin gathers);
// the up-spin hops read rows u' of V_k coalesced along d.  All CTAs of one
// column are adjacent in launch order, so the column being gathered from stays
// in L2; V_{k-1} and W are streamed with evict-first hints so they do not push
// it out.  Offsets inside a column are 32-bit (fewer than 2^31 elements for
// L <= 16).  Three variants follow: this one (FP32 rows with an odd D_dn, one
// element per thread), k_cf_apply_hub_fx (FP64, hop sums in fixed point) and
// k_cf_apply_hub_f2x2 (FP32, two elements per thread, bank-aware placement).
// Multi: the columns belong to clusters of different sizes; each CTA reads its
// column's cluster view, and CTAs past that cluster's rows write a zero partial.
template <typename C, bool Multi>
__global__ void __launch_bounds__(256, 6) k_cf_apply_hub(HubView h0, const HubView* __restrict__ hv,
                                                         const int* __restrict__ colq, const C* __restrict__ Vk,
                                                         const C* __restrict__ Vkm1, C* __restrict__ W, int64_t ld,
                                                         const int* __restrict__ cols, CFCoef cf, double* part) {
    using S = scalar_t<C>;
    const int c = cols[blockIdx.y];
    const int u = blockIdx.x;
    HubView h = h0;
    if constexpr (Multi) h = hv[colq[c]];
    if (Multi && u >= h.Dup) {            // row beyond this column's cluster
        if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = 0.0;
        return;
    }
    const int L = h.L;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* row = reinterpret_cast<C*>(sm_raw);                          // Ddn values of row u
    S* lut = reinterpret_cast<S*>(row + h.Ddn);                     // 3 (L + 1) diagonal values * sig
    __shared__ int s_uoff[kMaxHops];
    __shared__ S s_usg[kMaxHops];
    __shared__ double red[32];                                      // 64 floats in the FP32 path
    const int Ddn = int(h.Ddn);
    const C* __restrict__ Vc = Vk + int64_t(c) * ld;
    const C* __restrict__ Pc = Vkm1 + int64_t(c) * ld;
    C* __restrict__ Wc = W + int64_t(c) * ld;
    const int rbase = u * Ddn;
    constexpr bool f32 = std::is_same<S, float>::value;
    const S sig = f32 ? S(cf.sigf[c]) : S(cf.sig[c]);
    const S cB = f32 ? S(cf.cBf[c]) : S(cf.cB[c]);
    const bool has_prev = cB != S(0);
    const uint32_t su = __ldg(h.sup + u);
    const int nu = __ldg(h.nup + u);
    for (int d = threadIdx.x; d < Ddn; d += blockDim.x) row[d] = Vc[rbase + d];
    for (int i = threadIdx.x; i < 3 * (L + 1); i += blockDim.x) {
        const int p = i % (L + 1), nb = i / (L + 1);
        if constexpr (f32) lut[i] = sig * (h.Uf * float(p) - h.Ucf * float(nb));
        else lut[i] = sig * (h.U * double(p) - h.Uc * double(nb));
    }
    if (threadIdx.x < nu) {
        const int32_t ent = __ldg(h.hup + int64_t(threadIdx.x) * h.Dup + u);
        s_uoff[threadIdx.x] = (ent >> 1) * Ddn;
        s_usg[threadIdx.x] = (ent & 1) ? S(-1) : S(1);
    }
    __syncthreads();
    const int core = h.core;
    const int ubits = core >= 0 ? int((su >> core) & 1u) : 0;
    const S mt = f32 ? S(-h.tf * sig) : S(-h.t * sig);
    const S mcB = -cB;
    double dot = 0.0;
    float dhi = 0.f, dlo = 0.f;
    for (int d = threadIdx.x; d < Ddn; d += blockDim.x) {
        S ax = 0, ay = 0;
        // up-spin hops: gathers issued four at a time before they are consumed
        int e = 0;
        for (; e + 4 <= nu; e += 4) {
            const C v0 = Vc[s_uoff[e] + d], v1 = Vc[s_uoff[e + 1] + d];
            const C v2 = Vc[s_uoff[e + 2] + d], v3 = Vc[s_uoff[e + 3] + d];
            ax = fma(s_usg[e], v0.x, ax);
            ay = fma(s_usg[e], v0.y, ay);
            ax = fma(s_usg[e + 1], v1.x, ax);
            ay = fma(s_usg[e + 1], v1.y, ay);
            ax = fma(s_usg[e + 2], v2.x, ax);
            ay = fma(s_usg[e + 2], v2.y, ay);
            ax = fma(s_usg[e + 3], v3.x, ax);
            ay = fma(s_usg[e + 3], v3.y, ay);
        }
        for (; e < nu; ++e) {
            const C v = Vc[s_uoff[e] + d];
            ax = fma(s_usg[e], v.x, ax);
            ay = fma(s_usg[e], v.y, ay);
        }
        // down-spin hops: table entries, then row values, four at a time
        const int nd = __ldg(h.ndnp + d);
        e = 0;
        for (; e + 4 <= nd; e += 4) {
            const int h0 = __ldg(h.hdn16 + e * Ddn + d), h1 = __ldg(h.hdn16 + (e + 1) * Ddn + d);
            const int h2 = __ldg(h.hdn16 + (e + 2) * Ddn + d), h3 = __ldg(h.hdn16 + (e + 3) * Ddn + d);
            const C v0 = row[h0 >> 1], v1 = row[h1 >> 1], v2 = row[h2 >> 1], v3 = row[h3 >> 1];
            const S g0 = (h0 & 1) ? S(-1) : S(1), g1 = (h1 & 1) ? S(-1) : S(1);
            const S g2 = (h2 & 1) ? S(-1) : S(1), g3 = (h3 & 1) ? S(-1) : S(1);
            ax = fma(g0, v0.x, ax);
            ay = fma(g0, v0.y, ay);
            ax = fma(g1, v1.x, ax);
            ay = fma(g1, v1.y, ay);
            ax = fma(g2, v2.x, ax);
            ay = fma(g2, v2.y, ay);
            ax = fma(g3, v3.x, ax);
            ay = fma(g3, v3.y, ay);
        }
        for (; e < nd; ++e) {
            const int hh = __ldg(h.hdn16 + e * Ddn + d);
            const C v = row[hh >> 1];
            const S sg = (hh & 1) ? S(-1) : S(1);
            ax = fma(sg, v.x, ax);
            ay = fma(sg, v.y, ay);
        }
        const uint32_t sd = __ldg(h.sdnp + d);
        const int nb = core >= 0 ? ubits + int((sd >> core) & 1u) : 0;
        const S dg = lut[__popc(su & sd) + nb * (L + 1)];
        const C x = row[d];
        C wv;
        wv.x = fma(mt, ax, dg * x.x);
        wv.y = fma(mt, ay, dg * x.y);
        if (has_prev) {
            const C y = __ldcs(Pc + rbase + d);
            wv.x = fma(mcB, y.x, wv.x);
            wv.y = fma(mcB, y.y, wv.y);
        }
        __stcs(Wc + rbase + d, wv);
        if constexpr (std::is_same<S, float>::value) {
            df_add_prod(dhi, dlo, x.x, wv.x);
            df_add_prod(dhi, dlo, x.y, wv.y);
        } else {
            dot = fma(x.x, wv.x, fma(x.y, wv.y, dot));
        }
    }
    if constexpr (f32) {
        const double tot = block_sum_df(dhi, dlo, reinterpret_cast<float*>(red));
        if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = tot;
    } else {
        double acc[1] = {dot};
        block_sum<1>(acc, red);
        if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = acc[0];
    }
}

// ---------------------------------------------------------------------------
// FP64 pass A with the hop sums accumulated exactly in 64-bit fixed point.
//
// On this GPU the FP64 pipe issues a small fraction of the integer rate, and
// 2 of every 2.5 FP64 operations of the plain kernel are the +-1 hop terms.
// Here every component of V_k is bounded by ||V_k|| = 1/sig_k (q_k = sig_k V_k
// has unit norm).  If sig_k has biased exponent es, then 1/sig_k <= 2^(1023-es),
// so no component has a biased exponent above e_B = 2047 - es.  A component
// v = M 2^(e-1075) (M the 53-bit significand, e its biased exponent) becomes the
// integer F = sign(v) floor(32 M / 2^(e_B - e)) in units of 2^(e_B - 1080):
// |F| < 2^58, and the truncation drops less than 2^-55 of the bound.  An
// element's hop sum adds at most 2L such integers taken from distinct
// elements, so sum |F| <= sqrt(2L) 2^58 < 2^61 and the integer sum is exact.
// It is rounded to double once.  FP64 operations per element: the diagonal
// (2), the hop scale (2), the conversion (2), V_{k-1} (2) and the product with
// V_k (2), independent of the hop count.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long fx_term(double v, int eB, long long neg) {
    const long long b = __double_as_longlong(v);
    const int e = int(static_cast<unsigned>(b >> 52) & 0x7FFu);
    // eB >= 63, so zero and subnormals (e = 0) shift out entirely; a non-finite
    // component (e > eB) also maps to 0 here and reaches W through the diagonal.
    const unsigned r = min(static_cast<unsigned>(eB - e), 63u);
    const unsigned long long m =
        ((static_cast<unsigned long long>(b) & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 5;
    const long long f = static_cast<long long>(m >> r);
    const long long s = (b >> 63) ^ neg;                       // 0 or -1
    return (f ^ s) - s;
}

__device__ __forceinline__ long long fx_signed(long long f, long long neg) { return (f ^ neg) - neg; }


template <bool Multi, bool Signed>
__global__ void __launch_bounds__(256, 5) k_cf_apply_hub_fx(HubView h0, const HubView* __restrict__ hv,
                                                            const int* __restrict__ colq,
                                                            const double2* __restrict__ Vk,
                                                            const double2* __restrict__ Vkm1,
                                                            double2* __restrict__ W, int64_t ld,
                                                            const int* __restrict__ cols, CFCoef cf, double* part) {
    const int c = cols[blockIdx.y];
    const int u = blockIdx.x;
    HubView h = h0;
    if constexpr (Multi) h = hv[colq[c]];
    if (Multi && u >= h.Dup) {            // row beyond this column's cluster
        if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = 0.0;
        return;
    }
    const int L = h.L;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    longlong2* row = reinterpret_cast<longlong2*>(sm_raw);          // row u of V_k in fixed point
    double* lut = reinterpret_cast<double*>(row + h.Ddn + 2);       // 3 (L + 1) diagonal values * sig
    __shared__ int s_uoff[kMaxHops];
    __shared__ int s_uneg[kMaxHops];
    __shared__ double red[32];
    const int Ddn = int(h.Ddn);
    const double2* __restrict__ Vc = Vk + int64_t(c) * ld;
    const double2* __restrict__ Pc = Vkm1 + int64_t(c) * ld;
    double2* __restrict__ Wc = W + int64_t(c) * ld;
    const int rbase = u * Ddn;
    const double sig = cf.sig[c], cB = cf.cB[c];
    const bool has_prev = (__double_as_longlong(cB) << 1) != 0;
    const int es = int(static_cast<unsigned long long>(__double_as_longlong(sig)) >> 52) & 0x7FF;
    const int eB = max(min(2047 - es, 2100), 63);
    const uint32_t su = __ldg(h.sup + u);
    const int nu = __ldg(h.nup + u);
    for (int d = threadIdx.x; d < Ddn; d += blockDim.x) {
        const double2 v = Vc[rbase + d];
        row[d] = make_longlong2(fx_term(v.x, eB, 0), fx_term(v.y, eB, 0));
    }
    if (threadIdx.x == 0) row[Ddn] = make_longlong2(0, 0);        // target of the empty down-spin slots
    for (int i = threadIdx.x; i < 3 * (L + 1); i += blockDim.x) {
        const int p = i % (L + 1), nb = i / (L + 1);
        lut[i] = sig * (h.U * double(p) - h.Uc * double(nb));
    }
    if (threadIdx.x < nu) {
        const int32_t ent = __ldg(h.hup + int64_t(threadIdx.x) * h.Dup + u);
        s_uoff[threadIdx.x] = (ent >> 1) * Ddn;
        s_uneg[threadIdx.x] = Signed ? -(ent & 1) : 0;
    }
    __syncthreads();
    const int core = h.core;
    const int ubits = core >= 0 ? int((su >> core) & 1u) : 0;
    // -t sig times the fixed-point unit 2^(eB - 1080) (an exact power of two)
    const double mts = (-h.t * sig) * __longlong_as_double(static_cast<long long>(eB - 57) << 52);
    const double mcB = -cB;
    const uint16_t* __restrict__ t16 = h.hdn16;                     // [slot][position], (target << 1) | neg
    double dot = 0.0;
    // Every lane of a warp runs the same iterations (lanes past the row idle,
    // guarded), so the down-spin loop runs to a warp-uniform count.
    const int iters = (Ddn + blockDim.x - 1) / blockDim.x;
    for (int it = 0; it < iters; ++it) {
        const int d0 = it * blockDim.x + threadIdx.x;
        const bool act = d0 < Ddn;
        const int d = act ? d0 : 0;
        long long ax = 0, ay = 0;
        int e = 0;
        for (; e + 4 <= nu; e += 4) {
            const double2 v0 = Vc[s_uoff[e] + d], v1 = Vc[s_uoff[e + 1] + d];
            const double2 v2 = Vc[s_uoff[e + 2] + d], v3 = Vc[s_uoff[e + 3] + d];
            const long long g0 = Signed ? s_uneg[e] : 0, g1 = Signed ? s_uneg[e + 1] : 0;
            const long long g2 = Signed ? s_uneg[e + 2] : 0, g3 = Signed ? s_uneg[e + 3] : 0;
            ax += fx_term(v0.x, eB, g0);
            ay += fx_term(v0.y, eB, g0);
            ax += fx_term(v1.x, eB, g1);
            ay += fx_term(v1.y, eB, g1);
            ax += fx_term(v2.x, eB, g2);
            ay += fx_term(v2.y, eB, g2);
            ax += fx_term(v3.x, eB, g3);
            ay += fx_term(v3.y, eB, g3);
        }
        for (; e < nu; ++e) {
            const double2 v = Vc[s_uoff[e] + d];
            const long long g = Signed ? s_uneg[e] : 0;
            ax += fx_term(v.x, eB, g);
            ay += fx_term(v.y, eB, g);
        }
        // slots past an element's own count hold the zero slot: no per-hop predicate
        const int nd = __reduce_max_sync(0xffffffffu, act ? int(__ldg(h.ndnp + d)) : 0);
        e = 0;
        for (; e + 4 <= nd; e += 4) {
            const int h0 = __ldg(t16 + e * Ddn + d), h1 = __ldg(t16 + (e + 1) * Ddn + d);
            const int h2 = __ldg(t16 + (e + 2) * Ddn + d), h3 = __ldg(t16 + (e + 3) * Ddn + d);
            const longlong2 f0 = row[h0 >> 1], f1 = row[h1 >> 1], f2 = row[h2 >> 1], f3 = row[h3 >> 1];
            const long long g0 = Signed ? -(h0 & 1) : 0, g1 = Signed ? -(h1 & 1) : 0;
            const long long g2 = Signed ? -(h2 & 1) : 0, g3 = Signed ? -(h3 & 1) : 0;
            ax += fx_signed(f0.x, g0);
            ay += fx_signed(f0.y, g0);
            ax += fx_signed(f1.x, g1);
            ay += fx_signed(f1.y, g1);
            ax += fx_signed(f2.x, g2);
            ay += fx_signed(f2.y, g2);
            ax += fx_signed(f3.x, g3);
            ay += fx_signed(f3.y, g3);
        }
        for (; e < nd; ++e) {
            const int hh = __ldg(t16 + e * Ddn + d);
            const longlong2 f = row[hh >> 1];
            const long long g = Signed ? -(hh & 1) : 0;
            ax += fx_signed(f.x, g);
            ay += fx_signed(f.y, g);
        }
        const uint32_t sd = __ldg(h.sdnp + d);
        const int nb = core >= 0 ? ubits + int((sd >> core) & 1u) : 0;
        const double dg = lut[__popc(su & sd) + nb * (L + 1)];
        if (!act) continue;                                      // warp-uniform part done
        const double2 x = Vc[rbase + d];
        double2 wv;
        wv.x = fma(mts, __ll2double_rn(ax), dg * x.x);
        wv.y = fma(mts, __ll2double_rn(ay), dg * x.y);
        if (has_prev) {
            const double2 y = __ldcs(Pc + rbase + d);
            wv.x = fma(mcB, y.x, wv.x);
            wv.y = fma(mcB, y.y, wv.y);
        }
        __stcs(Wc + rbase + d, wv);
        dot = fma(x.x, wv.x, fma(x.y, wv.y, dot));
    }
    double acc[1] = {dot};
    block_sum<1>(acc, red);
    if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = acc[0];
}

// FP32 pass A with two adjacent elements per thread (NT threads, MINB CTAs per SM:
// 256 x 6 at 40 registers, 256 x 8 or 512 x 4 at 32 registers for full occupancy;
// a row takes less shared memory per resident warp with 512): the up-spin gathers, the
// V_{k-1} loads and the W stores move 16 bytes (two complex floats) at a time,
// and the down-spin table is read as 16-bit entries, two per 32-bit load.
// Needs an even Ddn (rows start on 16-byte boundaries) and Ddn < 32768.  The row
// sits at the sector's bank-aware slots (slot16, with the table hdn16p rewritten
// to them) when the operator has them; the down-spin loop runs to the warp's
// largest hop count, empty slots reading the zero kept past the row.  No FP64
// instruction: coefficients arrive as FP32 copies, the product is compensated
// FP32, and the block sum is float-float.
template <bool Multi, bool Signed, int MINB, int NT = 256>
__global__ void __launch_bounds__(NT, MINB) k_cf_apply_hub_f2x2(HubView h0, const HubView* __restrict__ hv,
                                                              const int* __restrict__ colq,
                                                              const float2* __restrict__ Vk,
                                                              const float2* __restrict__ Vkm1, float2* __restrict__ W,
                                                              int64_t ld, const int* __restrict__ cols, CFCoef cf,
                                                              double* part) {
    const int c = cols[blockIdx.y];
    const int u = blockIdx.x;
    HubView h = h0;
    if constexpr (Multi) h = hv[colq[c]];
    if (Multi && u >= h.Dup) {            // row beyond this column's cluster
        if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = 0.0;
        return;
    }
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float2* row = reinterpret_cast<float2*>(sm_raw);                // Ddn values of row u, then kRowZeroWords zeros
    __shared__ int s_uoff[kMaxHops];
    __shared__ float s_usg[kMaxHops];
    __shared__ float red[64];
    const int Ddn = int(h.Ddn);
    const int half = Ddn >> 1;
    const float2* __restrict__ Vc = Vk + int64_t(c) * ld;
    const float4* __restrict__ Pc4 = reinterpret_cast<const float4*>(Vkm1 + int64_t(c) * ld);
    float4* __restrict__ Wc4 = reinterpret_cast<float4*>(W + int64_t(c) * ld);
    const int rbase = u * Ddn;                      // even
    const float sig = cf.sigf[c], cB = cf.cBf[c];
    const bool has_prev = cB != 0.f;
    const uint32_t su = __ldg(h.sup + u);
    const int nu = __ldg(h.nup + u);
    // Row u into shared memory: element d at slot16[d] when the sector has a
    // bank-aware placement (fewer conflicts in the random down-spin gathers),
    // else at d.
    const bool placed = h.slot16 != nullptr;
    {
        const float4* src = reinterpret_cast<const float4*>(Vc + rbase);
        if (placed) {
            const uint32_t* sl2 = reinterpret_cast<const uint32_t*>(h.slot16);   // slots of 2i, 2i + 1
            for (int i = threadIdx.x; i < half; i += blockDim.x) {
                const float4 v = src[i];
                const uint32_t sp = __ldg(sl2 + i);
                row[sp & 0xFFFFu] = make_float2(v.x, v.y);
                row[sp >> 16] = make_float2(v.z, v.w);
            }
        } else {
            float4* dst = reinterpret_cast<float4*>(row);
            for (int i = threadIdx.x; i < half; i += blockDim.x) dst[i] = src[i];
        }
        if (threadIdx.x < kRowZeroWords / 2)                   // row[Ddn .. Ddn + kRowZeroWords - 1]
            reinterpret_cast<float4*>(row)[half + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (threadIdx.x < nu) {
        const int32_t ent = __ldg(h.hup + int64_t(threadIdx.x) * h.Dup + u);
        s_uoff[threadIdx.x] = ((ent >> 1) * Ddn) >> 1;           // in float4 units
        s_usg[threadIdx.x] = (Signed && (ent & 1)) ? -1.f : 1.f;
    }
    __syncthreads();
    const int core = h.core;
    const int ubits = core >= 0 ? int((su >> core) & 1u) : 0;
    const float mt = -h.tf * sig;
    const float sU = sig * h.Uf, sUc = sig * h.Ucf;                 // diagonal: sig (U popc - Uc nb)
    const float mcB = -cB;
    const float4* __restrict__ Vc4 = reinterpret_cast<const float4*>(Vc);
    const uint32_t* __restrict__ t32 = reinterpret_cast<const uint32_t*>(placed ? h.hdn16p : h.hdn16);
    const uint16_t* __restrict__ n16 = reinterpret_cast<const uint16_t*>(h.ndnp);
    const uint2* __restrict__ sd2 = reinterpret_cast<const uint2*>(h.sdnp);
    float dhi = 0.f, dlo = 0.f;
    // Every lane of a warp runs the same iterations (lanes past the row idle, guarded),
    // so the down-spin loop can use a warp-uniform trip count without divergence.
    const int iters = (half + blockDim.x - 1) / blockDim.x;
    const int step = Ddn >> 1;                                  // table slot stride in 32-bit words
    for (int it = 0; it < iters; ++it) {
        const int q0 = it * blockDim.x + threadIdx.x;
        const bool act = q0 < half;
        const int q = act ? q0 : 0;                             // elements d0 = 2q, d1 = 2q + 1
        float a0x = 0.f, a0y = 0.f, a1x = 0.f, a1y = 0.f;
        int e = 0;
        if constexpr (!Signed) {                                // four partner rows in flight
            for (; e + 4 <= nu; e += 4) {
                const float4 v0 = Vc4[s_uoff[e] + q], v1 = Vc4[s_uoff[e + 1] + q];
                const float4 v2 = Vc4[s_uoff[e + 2] + q], v3 = Vc4[s_uoff[e + 3] + q];
                a0x += (v0.x + v1.x) + (v2.x + v3.x); a0y += (v0.y + v1.y) + (v2.y + v3.y);
                a1x += (v0.z + v1.z) + (v2.z + v3.z); a1y += (v0.w + v1.w) + (v2.w + v3.w);
            }
        }
        for (; e + 2 <= nu; e += 2) {
            const float4 v = Vc4[s_uoff[e] + q], w4 = Vc4[s_uoff[e + 1] + q];
            if constexpr (Signed) {
                const float g = s_usg[e], g2 = s_usg[e + 1];
                a0x = fmaf(g, v.x, a0x); a0y = fmaf(g, v.y, a0y);
                a1x = fmaf(g, v.z, a1x); a1y = fmaf(g, v.w, a1y);
                a0x = fmaf(g2, w4.x, a0x); a0y = fmaf(g2, w4.y, a0y);
                a1x = fmaf(g2, w4.z, a1x); a1y = fmaf(g2, w4.w, a1y);
            } else {
                a0x += v.x + w4.x; a0y += v.y + w4.y;
                a1x += v.z + w4.z; a1y += v.w + w4.w;
            }
        }
        if (e < nu) {
            const float4 v = Vc4[s_uoff[e] + q];
            const float g = Signed ? s_usg[e] : 1.f;
            a0x = fmaf(g, v.x, a0x); a0y = fmaf(g, v.y, a0y);
            a1x = fmaf(g, v.z, a1x); a1y = fmaf(g, v.w, a1y);
        }
        const uint32_t nn = __ldg(n16 + q);
        const int nd0 = int(nn & 0xFFu), nd1 = int(nn >> 8);
        // slots past an element's own count hold the zero slot: no per-hop predicate
        const int ndw = __reduce_max_sync(0xffffffffu, act ? max(nd0, nd1) : 0);
        const uint32_t* __restrict__ tp = t32 + q;
        for (int k = 0; k < ndw; ++k, tp += step) {
            const uint32_t ta = __ldg(tp);                      // one hop of each element
            const float2 va = row[(ta & 0xFFFFu) >> 1], vb = row[ta >> 17];
            if constexpr (Signed) {
                const float ga = (ta & 1u) ? -1.f : 1.f, gb = (ta & 0x10000u) ? -1.f : 1.f;
                a0x = fmaf(ga, va.x, a0x); a0y = fmaf(ga, va.y, a0y);
                a1x = fmaf(gb, vb.x, a1x); a1y = fmaf(gb, vb.y, a1y);
            } else {
                a0x += va.x; a0y += va.y;
                a1x += vb.x; a1y += vb.y;
            }
        }
        const uint2 sd = __ldg(sd2 + q);
        const int nb0 = core >= 0 ? ubits + int((sd.x >> core) & 1u) : 0;
        const int nb1 = core >= 0 ? ubits + int((sd.y >> core) & 1u) : 0;
        const float dg0 = fmaf(sU, float(__popc(su & sd.x)), -sUc * float(nb0));
        const float dg1 = fmaf(sU, float(__popc(su & sd.y)), -sUc * float(nb1));
        float2 x0, x1;
        if (placed) {                                           // own values: from global (L1/L2)
            const float4 xv = Vc4[(rbase >> 1) + q];
            x0 = make_float2(xv.x, xv.y);
            x1 = make_float2(xv.z, xv.w);
        } else {
            x0 = row[2 * q];
            x1 = row[2 * q + 1];
        }
        float4 wv;
        wv.x = fmaf(mt, a0x, dg0 * x0.x);
        wv.y = fmaf(mt, a0y, dg0 * x0.y);
        wv.z = fmaf(mt, a1x, dg1 * x1.x);
        wv.w = fmaf(mt, a1y, dg1 * x1.y);
        if (!act) continue;                                      // warp-uniform part done
        if (has_prev) {
            const float4 y = __ldcs(Pc4 + (rbase >> 1) + q);
            wv.x = fmaf(mcB, y.x, wv.x);
            wv.y = fmaf(mcB, y.y, wv.y);
            wv.z = fmaf(mcB, y.z, wv.z);
            wv.w = fmaf(mcB, y.w, wv.w);
        }
        __stcs(Wc4 + (rbase >> 1) + q, wv);
        df_add_prod(dhi, dlo, x0.x, wv.x);
        df_add_prod(dhi, dlo, x0.y, wv.y);
        df_add_prod(dhi, dlo, x1.x, wv.z);
        df_add_prod(dhi, dlo, x1.y, wv.w);
    }
    const double tot = block_sum_df(dhi, dlo, red);
    if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = tot;
}

// The FP32 pass A for two columns per CTA (one operator for all columns): the two
// columns' row u share the up-spin offsets, the down-spin table entries, the index
// arithmetic, the occupation strings and the loop control, so the issue-bound
// kernel spends about a third fewer instructions per column.  Both rows sit in
// shared memory at the sector's bank-aware slots.  blockIdx.y indexes a pair of
// active columns (cols[2y], cols[2y + 1]); a missing second column (odd count)
// is skipped.  Partial products go to part[(2y + j) * gridDim.x + u], the layout
// of the one-column kernel.
template <bool Signed>
__global__ void __launch_bounds__(256, 4) k_cf_apply_hub_f2x2c2(HubView h, const float2* __restrict__ Vk,
                                                                const float2* __restrict__ Vkm1,
                                                                float2* __restrict__ W, int64_t ld,
                                                                const int* __restrict__ cols, int na, CFCoef cf,
                                                                double* part) {
    const int u = blockIdx.x;
    const int j0 = 2 * blockIdx.y;
    const bool two = j0 + 1 < na;
    const int c0 = cols[j0];
    const int c1 = two ? cols[j0 + 1] : c0;
    const int L = h.L;
    const int Ddn = int(h.Ddn);
    const int half = Ddn >> 1;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float2* row0 = reinterpret_cast<float2*>(sm_raw);               // row u of column 0, then kRowZeroWords zeros
    float2* row1 = row0 + (Ddn + kRowZeroWords);                    // row u of column 1, then kRowZeroWords zeros
    float* lut0 = reinterpret_cast<float*>(row1 + (Ddn + kRowZeroWords));   // 3 (L + 1) diagonal values * sig, per column
    float* lut1 = lut0 + 3 * (L + 1);
    __shared__ int s_uoff[kMaxHops];
    __shared__ float s_usg[kMaxHops];
    __shared__ float red[64];
    const float2* __restrict__ V0 = Vk + int64_t(c0) * ld;
    const float2* __restrict__ V1 = Vk + int64_t(c1) * ld;
    const float4* __restrict__ P04 = reinterpret_cast<const float4*>(Vkm1 + int64_t(c0) * ld);
    const float4* __restrict__ P14 = reinterpret_cast<const float4*>(Vkm1 + int64_t(c1) * ld);
    float4* __restrict__ W04 = reinterpret_cast<float4*>(W + int64_t(c0) * ld);
    float4* __restrict__ W14 = reinterpret_cast<float4*>(W + int64_t(c1) * ld);
    const int rbase = u * Ddn;
    const float sig0 = cf.sigf[c0], cB0 = cf.cBf[c0], sig1 = cf.sigf[c1], cB1 = cf.cBf[c1];
    const uint32_t su = __ldg(h.sup + u);
    const int nu = __ldg(h.nup + u);
    const uint32_t* sl2 = reinterpret_cast<const uint32_t*>(h.slot16);   // slots of positions 2i, 2i + 1
    {
        const float4* src0 = reinterpret_cast<const float4*>(V0 + rbase);
        const float4* src1 = reinterpret_cast<const float4*>(V1 + rbase);
        for (int i = threadIdx.x; i < half; i += blockDim.x) {
            const uint32_t sp = __ldg(sl2 + i);
            const float4 a = src0[i], b = src1[i];
            row0[sp & 0xFFFFu] = make_float2(a.x, a.y);
            row0[sp >> 16] = make_float2(a.z, a.w);
            row1[sp & 0xFFFFu] = make_float2(b.x, b.y);
            row1[sp >> 16] = make_float2(b.z, b.w);
        }
        if (threadIdx.x < kRowZeroWords / 2) {
            reinterpret_cast<float4*>(row0)[half + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4*>(row1)[half + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    for (int i = threadIdx.x; i < 3 * (L + 1); i += blockDim.x) {
        const int p = i % (L + 1), nb = i / (L + 1);
        const float e = h.Uf * float(p) - h.Ucf * float(nb);
        lut0[i] = sig0 * e;
        lut1[i] = sig1 * e;
    }
    if (threadIdx.x < nu) {
        const int32_t ent = __ldg(h.hup + int64_t(threadIdx.x) * h.Dup + u);
        s_uoff[threadIdx.x] = ((ent >> 1) * Ddn) >> 1;           // in float4 units
        s_usg[threadIdx.x] = (Signed && (ent & 1)) ? -1.f : 1.f;
    }
    __syncthreads();
    const int core = h.core;
    const int ubits = core >= 0 ? int((su >> core) & 1u) : 0;
    const float mt0 = -h.tf * sig0, mt1 = -h.tf * sig1;
    const float4* __restrict__ V04 = reinterpret_cast<const float4*>(V0);
    const float4* __restrict__ V14 = reinterpret_cast<const float4*>(V1);
    const uint32_t* __restrict__ t32 = reinterpret_cast<const uint32_t*>(h.hdn16p);
    const uint16_t* __restrict__ n16 = reinterpret_cast<const uint16_t*>(h.ndnp);
    const uint2* __restrict__ sd2 = reinterpret_cast<const uint2*>(h.sdnp);
    float dh0 = 0.f, dl0 = 0.f, dh1 = 0.f, dl1 = 0.f;
    const int iters = (half + blockDim.x - 1) / blockDim.x;
    const int step = Ddn >> 1;
    for (int it = 0; it < iters; ++it) {
        const int q0 = it * blockDim.x + threadIdx.x;
        const bool act = q0 < half;
        const int q = act ? q0 : 0;
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = 0; e < nu; ++e) {
            const int o = s_uoff[e] + q;
            const float4 v = V04[o], w4 = V14[o];
            if constexpr (Signed) {
                const float g = s_usg[e];
                A.x = fmaf(g, v.x, A.x); A.y = fmaf(g, v.y, A.y); A.z = fmaf(g, v.z, A.z); A.w = fmaf(g, v.w, A.w);
                B.x = fmaf(g, w4.x, B.x); B.y = fmaf(g, w4.y, B.y); B.z = fmaf(g, w4.z, B.z); B.w = fmaf(g, w4.w, B.w);
            } else {
                A.x += v.x; A.y += v.y; A.z += v.z; A.w += v.w;
                B.x += w4.x; B.y += w4.y; B.z += w4.z; B.w += w4.w;
            }
        }
        const uint32_t nn = __ldg(n16 + q);
        const int ndw = __reduce_max_sync(0xffffffffu, act ? max(int(nn & 0xFFu), int(nn >> 8)) : 0);
        const uint32_t* __restrict__ tp = t32 + q;
        for (int k = 0; k < ndw; ++k, tp += step) {
            const uint32_t ta = __ldg(tp);
            const int ia = int((ta & 0xFFFFu) >> 1), ib = int(ta >> 17);
            const float2 va = row0[ia], vb = row0[ib], wa = row1[ia], wb = row1[ib];
            if constexpr (Signed) {
                const float ga = (ta & 1u) ? -1.f : 1.f, gb = (ta & 0x10000u) ? -1.f : 1.f;
                A.x = fmaf(ga, va.x, A.x); A.y = fmaf(ga, va.y, A.y); A.z = fmaf(gb, vb.x, A.z); A.w = fmaf(gb, vb.y, A.w);
                B.x = fmaf(ga, wa.x, B.x); B.y = fmaf(ga, wa.y, B.y); B.z = fmaf(gb, wb.x, B.z); B.w = fmaf(gb, wb.y, B.w);
            } else {
                A.x += va.x; A.y += va.y; A.z += vb.x; A.w += vb.y;
                B.x += wa.x; B.y += wa.y; B.z += wb.x; B.w += wb.y;
            }
        }
        const uint2 sd = __ldg(sd2 + q);
        const int nb0 = core >= 0 ? ubits + int((sd.x >> core) & 1u) : 0;
        const int nb1 = core >= 0 ? ubits + int((sd.y >> core) & 1u) : 0;
        const int l0 = __popc(su & sd.x) + nb0 * (L + 1), l1 = __popc(su & sd.y) + nb1 * (L + 1);
        if (!act) continue;                                      // warp-uniform part done
        const int g4 = (rbase >> 1) + q;
        {
            const float4 x = V04[g4];
            const float d0 = lut0[l0], d1 = lut0[l1];
            float4 wv;
            wv.x = fmaf(mt0, A.x, d0 * x.x);
            wv.y = fmaf(mt0, A.y, d0 * x.y);
            wv.z = fmaf(mt0, A.z, d1 * x.z);
            wv.w = fmaf(mt0, A.w, d1 * x.w);
            if (cB0 != 0.f) {
                const float4 y = __ldcs(P04 + g4);
                wv.x = fmaf(-cB0, y.x, wv.x); wv.y = fmaf(-cB0, y.y, wv.y);
                wv.z = fmaf(-cB0, y.z, wv.z); wv.w = fmaf(-cB0, y.w, wv.w);
            }
            __stcs(W04 + g4, wv);
            df_add_prod(dh0, dl0, x.x, wv.x);
            df_add_prod(dh0, dl0, x.y, wv.y);
            df_add_prod(dh0, dl0, x.z, wv.z);
            df_add_prod(dh0, dl0, x.w, wv.w);
        }
        if (two) {
            const float4 x = V14[g4];
            const float d0 = lut1[l0], d1 = lut1[l1];
            float4 wv;
            wv.x = fmaf(mt1, B.x, d0 * x.x);
            wv.y = fmaf(mt1, B.y, d0 * x.y);
            wv.z = fmaf(mt1, B.z, d1 * x.z);
            wv.w = fmaf(mt1, B.w, d1 * x.w);
            if (cB1 != 0.f) {
                const float4 y = __ldcs(P14 + g4);
                wv.x = fmaf(-cB1, y.x, wv.x); wv.y = fmaf(-cB1, y.y, wv.y);
                wv.z = fmaf(-cB1, y.z, wv.z); wv.w = fmaf(-cB1, y.w, wv.w);
            }
            __stcs(W14 + g4, wv);
            df_add_prod(dh1, dl1, x.x, wv.x);
            df_add_prod(dh1, dl1, x.y, wv.y);
            df_add_prod(dh1, dl1, x.z, wv.z);
            df_add_prod(dh1, dl1, x.w, wv.w);
        }
    }
    const double t0 = block_sum_df(dh0, dl0, red);
    if (threadIdx.x == 0) part[int64_t(j0) * gridDim.x + u] = t0;
    __syncthreads();
    const double t1 = block_sum_df(dh1, dl1, red);
    if (two && threadIdx.x == 0) part[int64_t(j0 + 1) * gridDim.x + u] = t1;
}

// Pass A for any operator view (CSR): flat grid over elements.
template <class View, typename C>
__global__ void __launch_bounds__(256) k_cf_apply_gen(View op, const C* __restrict__ Vk, const C* __restrict__ Vkm1,
                                                      C* __restrict__ W, int64_t n, int64_t ld,
                                                      const int* __restrict__ cols, CFCoef cf, double* part) {
    using S = scalar_t<C>;
    __shared__ double sm[32];
    const int c = cols[blockIdx.y];
    const int64_t off = int64_t(c) * ld;
    const S sig = S(cf.sig[c]), mcB = S(-cf.cB[c]);
    const bool has_prev = cf.cB[c] != 0.0;
    double dot = 0.0;
    float dhi = 0.f, dlo = 0.f;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n; s += int64_t(gridDim.x) * blockDim.x) {
        const C x = Vk[off + s];
        const C hx = op.hx(s, Vk + off, x);
        C wv = mk(sig * hx.x, sig * hx.y);
        if (has_prev) {
            const C y = Vkm1[off + s];
            wv.x = fma(mcB, y.x, wv.x);
            wv.y = fma(mcB, y.y, wv.y);
        }
        W[off + s] = wv;
        if constexpr (std::is_same<S, float>::value) {
            df_add_prod(dhi, dlo, x.x, wv.x);
            df_add_prod(dhi, dlo, x.y, wv.y);
        } else {
            dot = fma(x.x, wv.x, fma(x.y, wv.y, dot));
        }
    }
    if constexpr (std::is_same<S, float>::value) dot = df_value(dhi, dlo);
    double acc[1] = {dot};
    store_partials<1>(acc, sm, part);
}

// a_k = sig_k * sum;  cC = a_k sig_k.
__global__ void k_cf_reduce_a(const double* part, int nblk, const int* cols, double* astore, int64_t stride_k, int k,
                              CFCoef cf) {
    __shared__ double sm[32];
    const int c = cols[blockIdx.x];
    double v[1];
    reduce_partials<1>(part + int64_t(blockIdx.x) * nblk, nblk, v, sm);
    if (threadIdx.x == 0) {
        const double a = cf.sig[c] * v[0];
        astore[int64_t(k) * stride_k + c] = a;
        cf.cC[c] = a * cf.sig[c];
        cf.cCf[c] = float(cf.cC[c]);
    }
}

// W -= cC V_k; partial ||W||^2.  16-byte loads: one complex double or two
// complex floats (ld is even and the padding is zero).
__device__ __forceinline__ void orth_step(double2 v, double2& x, double m, double& acc, float&, float&) {
    x.x = fma(m, v.x, x.x);
    x.y = fma(m, v.y, x.y);
    acc = fma(x.x, x.x, acc);
    acc = fma(x.y, x.y, acc);
}
__device__ __forceinline__ void orth_step(float4 v, float4& x, float m, double&, float& hi, float& lo) {
    x.x = fmaf(m, v.x, x.x);
    x.y = fmaf(m, v.y, x.y);
    x.z = fmaf(m, v.z, x.z);
    x.w = fmaf(m, v.w, x.w);
    df_add_prod(hi, lo, x.x, x.x);
    df_add_prod(hi, lo, x.y, x.y);
    df_add_prod(hi, lo, x.z, x.z);
    df_add_prod(hi, lo, x.w, x.w);
}

template <typename C>
__global__ void __launch_bounds__(256) k_cf_orth(const C* __restrict__ Vk, C* __restrict__ W, int64_t ld,
                                                 const int* __restrict__ cols, const int64_t* __restrict__ clen,
                                                 CFCoef cf, double* part) {
    using S = scalar_t<C>;
    using V16 = typename std::conditional<std::is_same<S, float>::value, float4, double2>::type;
    constexpr int per = sizeof(V16) / sizeof(C);     // complex elements per 16-byte load
    __shared__ double sm[32];
    const int c = cols[blockIdx.y];
    const V16* __restrict__ v4 = reinterpret_cast<const V16*>(Vk + int64_t(c) * ld);
    V16* __restrict__ w4 = reinterpret_cast<V16*>(W + int64_t(c) * ld);
    const int64_t nv = clen[c] / per;                 // column length, rounded up to even
    const S mc = std::is_same<S, float>::value ? S(-cf.cCf[c]) : S(-cf.cC[c]);
    double acc = 0.0;
    float hi = 0.f, lo = 0.f;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    // evict-first loads and stores: this pass streams whole columns that are not read
    // again soon, and should not push out of L2 the column another group's apply gathers from
    for (; i + stride < nv; i += 2 * stride) {      // two independent loads in flight per stream
        V16 x0 = __ldcs(w4 + i), x1 = __ldcs(w4 + i + stride);
        const V16 a0 = __ldcs(v4 + i), a1 = __ldcs(v4 + i + stride);
        orth_step(a0, x0, mc, acc, hi, lo);
        orth_step(a1, x1, mc, acc, hi, lo);
        __stcs(w4 + i, x0);
        __stcs(w4 + i + stride, x1);
    }
    if (i < nv) {
        V16 x0 = __ldcs(w4 + i);
        orth_step(__ldcs(v4 + i), x0, mc, acc, hi, lo);
        __stcs(w4 + i, x0);
    }
    if constexpr (std::is_same<S, float>::value) {
        const double tot = block_sum_df(hi, lo, reinterpret_cast<float*>(sm));
        if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = tot;
    } else {
        double a1[1] = {acc};
        store_partials<1>(a1, sm, part);
    }
}

// b_{k+1} = ||W||; next step: cB = b_{k+1} sig_k, sig = 1 / b_{k+1}.
__global__ void k_cf_reduce_b(const double* part, int nblk, const int* cols, double* bstore, int64_t stride_k, int k,
                              CFCoef cf) {
    __shared__ double sm[32];
    const int c = cols[blockIdx.x];
    double v[1];
    reduce_partials<1>(part + int64_t(blockIdx.x) * nblk, nblk, v, sm);
    if (threadIdx.x == 0) {
        const double b = sqrt(v[0]);
        bstore[int64_t(k) * stride_k + c] = b;
        cf.cB[c] = b * cf.sig[c];
        cf.sig[c] = b > 0.0 ? 1.0 / b : 0.0;
        cf.cBf[c] = float(cf.cB[c]);
        cf.sigf[c] = float(cf.sig[c]);
    }
}

// V_0 = phi (copied: the input is not modified; padding zeroed); the other two
// vector blocks get a zero padding; partial ||phi||^2.  Column c of phi starts
// at c * ldphi and has nlen[c] elements.  With the row-tiled Hubbard apply
// (hv != null) the column is stored in the continued-fraction row order of its
// operator: element (u, p) of V_0 is phi's element (u, dpos[p]).
template <typename C>
__global__ void __launch_bounds__(256) k_cf_start(const C* __restrict__ phi, int64_t ldphi,
                                                  const int64_t* __restrict__ nlen, const HubView* __restrict__ hv,
                                                  const int* __restrict__ colq, C* __restrict__ V0,
                                                  C* __restrict__ V1, C* __restrict__ V2, int64_t ld, double* part) {
    using S = scalar_t<C>;
    __shared__ double sm[32];
    const int c = blockIdx.y;
    const int64_t n = nlen[c];
    const uint16_t* __restrict__ dpos = hv ? hv[colq[c]].dpos : nullptr;
    const int64_t Ddn = hv ? hv[colq[c]].Ddn : 1;
    double acc = 0.0;
    float hi = 0.f, lo = 0.f;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < ld; s += int64_t(gridDim.x) * blockDim.x) {
        C x = mk(S(0), S(0));
        if (s < n) {
            int64_t src = s;
            if (dpos) {
                const int64_t u = s / Ddn;
                src = u * Ddn + __ldg(dpos + (s - u * Ddn));
            }
            x = phi[int64_t(c) * ldphi + src];
        }
        V0[int64_t(c) * ld + s] = x;
        if (s >= n) {
            V1[int64_t(c) * ld + s] = x;
            V2[int64_t(c) * ld + s] = x;
        }
        if constexpr (std::is_same<S, float>::value) {
            df_add_prod(hi, lo, x.x, x.x);
            df_add_prod(hi, lo, x.y, x.y);
        } else {
            acc = fma(x.x, x.x, fma(x.y, x.y, acc));
        }
    }
    if constexpr (std::is_same<S, float>::value) acc = df_value(hi, lo);
    double a1[1] = {acc};
    store_partials<1>(a1, sm, part);
}

// n0 = ||phi||^2, sig_0 = 1/sqrt(n0), cB = 0 (one CTA per column).
__global__ void k_cf_setup(const double* part, int nblk, double* n0, CFCoef cf) {
    __shared__ double sm[32];
    const int c = blockIdx.x;
    double v[1];
    reduce_partials<1>(part + int64_t(c) * nblk, nblk, v, sm);
    if (threadIdx.x == 0) {
        n0[c] = v[0];
        cf.sig[c] = v[0] > 0.0 ? 1.0 / sqrt(v[0]) : 0.0;
        cf.cB[c] = 0.0;
        cf.cC[c] = 0.0;
        cf.sigf[c] = float(cf.sig[c]);
        cf.cBf[c] = 0.f;
        cf.cCf[c] = 0.f;
    }
}

template <class View, typename C>
static void cf_impl(const CFColumns& P, const View& view, const double* w, int n_w, double eta, double cf_tol,
                    int check, int maxdepth, double* I_out, CFResult& out, cudaStream_t st, bool I_dev) {
    constexpr bool hub = std::is_same<View, HubView>::value;
    const int nv = P.nv;
    const bool multi = P.ops.size() > 1;
    std::vector<int64_t> nlen(nv), clen(nv);
    int64_t ld = 0;
    for (int c = 0; c < nv; ++c) {
        nlen[c] = P.ops[P.q[c]]->dim;
        clen[c] = (nlen[c] + 1) / 2 * 2;     // 16-byte loads in the orth pass; the padding stays zero
        ld = std::max(ld, clen[c]);
    }
    const C* phi = (const C*)P.phi;
    const int per = int(16 / sizeof(C));
    const int grid = grid_for(ld / per, 256, 4);
    int64_t hub_smem = 0;
    bool rows = false, pair = false, fx = false, sgn = false;
    int cpc = 1;                               // columns per CTA of the FP32 row-tiled apply
    int fx_threads = 256;
    int nblkA = grid;
    std::vector<HubView> hviews;
    if constexpr (hub) {
        int64_t maxDdn = 0, maxDup = 0;
        int maxL = 0;
        rows = true;
        pair = std::is_same<C, float2>::value;
        fx = std::is_same<C, double2>::value;
        for (const msb_op* o : P.ops) {
            const HubView& h = o->hub;
            hviews.push_back(h);
            maxDdn = std::max(maxDdn, h.Ddn);
            maxDup = std::max(maxDup, h.Dup);
            maxL = std::max(maxL, h.L);
            rows = rows && h.Wup <= kMaxHops && h.Dup * h.Ddn < (int64_t(1) << 31) && h.hdn16 != nullptr &&
                   h.hup2 == nullptr;      // the row-tiled kernels apply one hopping amplitude
            pair = pair && h.Ddn % 2 == 0;
            sgn = sgn || h.usign || h.dsign;
        }
        // row, its zero words (one for the FP64 and generic kernels, one per bank pair for
        // the FP32 two-element kernels, padded to 16 bytes), diagonal table
        const int zw = pair ? kRowZeroWords : 2;
        hub_smem = (maxDdn + zw) * int64_t(sizeof(C)) + 3 * (maxL + 1) * 8;
        rows = rows && hub_smem <= 160 * 1024;
        // FP64 fixed-point kernel: rows of up to 1024 elements take 128-thread CTAs (~7
        // elements per thread at L = 12, so the staging barrier and the block reduction
        // are paid over twice the work); longer rows keep 256 threads, where shared
        // memory, not registers, limits the CTAs per SM.
        fx_threads = maxDdn <= 1024 ? 128 : 256;
        if (!multi && std::is_same<C, double2>::value) {
            const int t = tuned_cf_threads(maxDdn, maxDup, MSB_FP64);
            if (t == 128 || t == 256) fx_threads = t;
        }
        // FP32 shape: 1 = one column per CTA at 6 CTAs per SM; 2 = two columns per CTA
        // (half the index work, 4 CTAs per SM); 3 = one column at 8 CTAs per SM (32
        // registers); 4 = one column per 512-thread CTA, 4 per SM (32 registers).
        // Shape 1 unless the autotuner measured another as faster.
        if (!multi && pair && hviews[0].slot16 != nullptr) {
            const int t = tuned_cf_threads(maxDdn, maxDup, MSB_FP32_MIXED);
            cpc = (t >= 2 && t <= 4) ? t : 1;
        }
        fx = fx && rows;
        pair = pair && rows;
        if (rows) {
            nblkA = int(maxDup);
            const void* fn = nullptr;
            if (fx)
                fn = multi ? (sgn ? (const void*)k_cf_apply_hub_fx<true, true> : (const void*)k_cf_apply_hub_fx<true, false>)
                           : (sgn ? (const void*)k_cf_apply_hub_fx<false, true> : (const void*)k_cf_apply_hub_fx<false, false>);
            else if (pair && cpc == 2) {
                fn = sgn ? (const void*)k_cf_apply_hub_f2x2c2<true> : (const void*)k_cf_apply_hub_f2x2c2<false>;
                hub_smem = 2 * (maxDdn + zw) * int64_t(sizeof(C)) + 2 * 3 * (maxL + 1) * 4;
                if (hub_smem > 200 * 1024) {               // rows too long for two per CTA
                    cpc = 1;
                    hub_smem = (maxDdn + zw) * int64_t(sizeof(C)) + 3 * (maxL + 1) * 8;
                    fn = sgn ? (const void*)k_cf_apply_hub_f2x2<false, true, 6> : (const void*)k_cf_apply_hub_f2x2<false, false, 6>;
                }
            } else if (pair && cpc == 3)
                fn = sgn ? (const void*)k_cf_apply_hub_f2x2<false, true, 8> : (const void*)k_cf_apply_hub_f2x2<false, false, 8>;
            else if (pair && cpc == 4)
                fn = sgn ? (const void*)k_cf_apply_hub_f2x2<false, true, 4, 512>
                         : (const void*)k_cf_apply_hub_f2x2<false, false, 4, 512>;
            else if (pair)
                fn = multi ? (sgn ? (const void*)k_cf_apply_hub_f2x2<true, true, 6> : (const void*)k_cf_apply_hub_f2x2<true, false, 6>)
                           : (sgn ? (const void*)k_cf_apply_hub_f2x2<false, true, 6> : (const void*)k_cf_apply_hub_f2x2<false, false, 6>);
            else
                fn = multi ? (const void*)k_cf_apply_hub<float2, true> : (const void*)k_cf_apply_hub<float2, false>;
            MSB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(hub_smem)));
            if (cpc == 3)      // eight rows of shared memory per SM: take the largest carve-out
                MSB_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              int(cudaSharedmemCarveoutMaxShared)));
        }
    }
    MSB_REQUIRE(!multi || rows, "a batch of clusters needs the row-tiled Hubbard apply (one hopping amplitude)");
    DevBuf<C> Q(3 * size_t(nv) * ld);
    DevBuf<double> part(size_t(std::max(grid, nblkA)) * nv), a(size_t(maxdepth) * nv), b(size_t(maxdepth) * nv),
        n0(nv), sig(nv), cB(nv), cC(nv), I(size_t(nv) * n_w), diff(2 * size_t(nv)), wdev(n_w), E0d(nv);
    DevBuf<float> sigf(nv), cBf(nv), cCf(nv);
    DevBuf<double2> gst(size_t(nv) * n_w), Cst(size_t(nv) * n_w), Dst(size_t(nv) * n_w);
    int k_eval = 0;                      // levels already folded into the convergents
    DevBuf<int> cols(nv), colq(nv);
    DevBuf<int64_t> nlen_d(nv), clen_d(nv);
    DevBuf<HubView> hv(std::max<size_t>(1, hviews.size()));
    if (!hviews.empty()) hv.upload(hviews.data(), hviews.size(), st);
    CFCoef cf{sig.p, cB.p, cC.p, sigf.p, cBf.p, cCf.p};
    wdev.upload(w, n_w, st);
    E0d.upload(P.E0.data(), nv, st);
    colq.upload(P.q.data(), nv, st);
    nlen_d.upload(nlen.data(), nv, st);
    clen_d.upload(clen.data(), nv, st);
    std::vector<int> hcols(nv), hdepth(nv, 0);
    MSB_CUDA(cudaMemsetAsync(I.p, 0, I.bytes(), st));
    C* vk = Q.p;
    C* vkm1 = Q.p + size_t(nv) * ld;
    C* wv = Q.p + 2 * size_t(nv) * ld;
    double all_elems = 0;
    for (int c = 0; c < nv; ++c) all_elems += double(nlen[c]);
    {
        ProfScope ps("cf_start", st, 2.0 * all_elems * sizeof(C), 4.0 * all_elems);
        k_cf_start<C><<<dim3(grid, nv), 256, 0, st>>>(phi, P.ldphi, nlen_d.p, rows ? hv.p : nullptr, colq.p, vk, vkm1,
                                                       wv, ld, part.p);
    }
    { ProfScope ps("cf_reduce", st, 0, 0); k_cf_setup<<<nv, 256, 0, st>>>(part.p, grid, n0.p, cf); }
    out.launches += 2;
    MSB_LAUNCH_CHECK();
    std::vector<double> hn0(nv), hdiff(2 * size_t(nv));
    MSB_CUDA(cudaMemcpyAsync(hn0.data(), n0.p, nv * sizeof(double), cudaMemcpyDeviceToHost, st));
    MSB_CUDA(cudaStreamSynchronize(st));
    int nact = 0;
    for (int c = 0; c < nv; ++c)
        if (hn0[c] > 0.0) hcols[nact++] = c;
    cols.upload(hcols.data(), std::max(nact, 1), st);
    const dim3 gridA(unsigned(nblkA), 1);
    // Two column groups on two streams: the apply of one group (bound by issue and the
    // L1/shared pipe) overlaps the orth pass of the other (bound by DRAM).  Each group's
    // levels are ordered on its own stream; the groups meet at every convergence check.
    // With the profiler on, one group, so that every launch is timed alone.
    const int ngrp = prof_on() ? 1 : 2;
    cudaStream_t gs[2] = {st, nullptr};
    cudaEvent_t gev = nullptr;
    if (ngrp == 2) {
        MSB_CUDA(cudaStreamCreateWithFlags(&gs[1], cudaStreamNonBlocking));
        MSB_CUDA(cudaEventCreateWithFlags(&gev, cudaEventDisableTiming));
    }
    struct StreamGuard {
        cudaStream_t s; cudaEvent_t e;
        ~StreamGuard() { if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); } if (e) cudaEventDestroy(e); }
    } sguard{gs[1], gev};
    DevBuf<int> gcols_d[2];
    DevBuf<double> gpart[2];
    std::vector<int> gcols[2];
    for (int g = 0; g < ngrp; ++g) {
        gcols_d[g].alloc(std::max(nv, 1));
        gpart[g].alloc(size_t(std::max(grid, nblkA)) * nv);
    }
    auto split = [&] {                              // active columns -> groups, interleaved
        for (int g = 0; g < ngrp; ++g) gcols[g].clear();
        for (int i = 0; i < nact; ++i) gcols[i % ngrp].push_back(hcols[i]);
        for (int g = 0; g < ngrp; ++g)
            if (!gcols[g].empty()) gcols_d[g].upload(gcols[g].data(), gcols[g].size(), st);
        if (ngrp == 2) {                            // the lists are uploaded on st
            MSB_CUDA(cudaEventRecord(gev, st));
            MSB_CUDA(cudaStreamWaitEvent(gs[1], gev, 0));
        }
    };
    split();
    double grp_bytes[2], grp_flops[2], grp_elems[2];
    auto regroup_counts = [&] {
        for (int g = 0; g < ngrp; ++g) {
            grp_bytes[g] = grp_flops[g] = grp_elems[g] = 0;
            for (int c : gcols[g]) {
                const msb_op* o = P.ops[P.q[c]];
                grp_elems[g] += double(nlen[c]);
                grp_bytes[g] += 3.0 * double(nlen[c]) * sizeof(C) + o->matrix_bytes(sizeof(C));
                grp_flops[g] += o->hx_flops() + 8.0 * double(nlen[c]);
            }
        }
    };
    regroup_counts();
    // one level of the recurrence for group g on its stream
    auto level = [&](int g, int kk) {
        const int na = int(gcols[g].size());
        if (na == 0) return;
        cudaStream_t s = gs[g];
        const int* cl = gcols_d[g].p;
        double* pt = gpart[g].p;
        {
            ProfScope ps("cf_apply", s, grp_bytes[g], grp_flops[g]);
            bool done_hub = false;
            if constexpr (hub) {
                const dim3 gg(gridA.x, unsigned(na));
                if (rows && fx) {
                    auto x = reinterpret_cast<const double2*>(vk);
                    auto xm = reinterpret_cast<const double2*>(vkm1);
                    auto y = reinterpret_cast<double2*>(wv);
                    auto kern = multi ? (sgn ? k_cf_apply_hub_fx<true, true> : k_cf_apply_hub_fx<true, false>)
                                      : (sgn ? k_cf_apply_hub_fx<false, true> : k_cf_apply_hub_fx<false, false>);
                    kern<<<gg, fx_threads, hub_smem, s>>>(view, hv.p, colq.p, x, xm, y, ld, cl, cf, pt);
                    done_hub = true;
                } else if (rows && pair && cpc == 2) {
                    auto x = reinterpret_cast<const float2*>(vk);
                    auto xm = reinterpret_cast<const float2*>(vkm1);
                    auto y = reinterpret_cast<float2*>(wv);
                    auto kern = sgn ? k_cf_apply_hub_f2x2c2<true> : k_cf_apply_hub_f2x2c2<false>;
                    const dim3 g2(gridA.x, unsigned((na + 1) / 2));
                    kern<<<g2, kApplyThreads, hub_smem, s>>>(hviews[0], x, xm, y, ld, cl, na, cf, pt);
                    done_hub = true;
                } else if (rows && pair) {
                    auto x = reinterpret_cast<const float2*>(vk);
                    auto xm = reinterpret_cast<const float2*>(vkm1);
                    auto y = reinterpret_cast<float2*>(wv);
                    auto kern = cpc == 4   ? (sgn ? k_cf_apply_hub_f2x2<false, true, 4, 512>
                                                      : k_cf_apply_hub_f2x2<false, false, 4, 512>)
                                : cpc == 3 ? (sgn ? k_cf_apply_hub_f2x2<false, true, 8> : k_cf_apply_hub_f2x2<false, false, 8>)
                                : multi    ? (sgn ? k_cf_apply_hub_f2x2<true, true, 6> : k_cf_apply_hub_f2x2<true, false, 6>)
                                           : (sgn ? k_cf_apply_hub_f2x2<false, true, 6> : k_cf_apply_hub_f2x2<false, false, 6>);
                    kern<<<gg, cpc == 4 ? 512 : kApplyThreads, hub_smem, s>>>(view, hv.p, colq.p, x, xm, y, ld, cl, cf,
                                                                            pt);
                    done_hub = true;
                } else if (rows) {
                    // FP32 with an odd D_dn (FP64 always takes the fixed-point kernel)
                    if constexpr (std::is_same<C, float2>::value) {
                        if (multi)
                            k_cf_apply_hub<C, true><<<gg, kApplyThreads, hub_smem, s>>>(view, hv.p, colq.p, vk, vkm1,
                                                                                         wv, ld, cl, cf, pt);
                        else
                            k_cf_apply_hub<C, false><<<gg, kApplyThreads, hub_smem, s>>>(view, hv.p, colq.p, vk, vkm1,
                                                                                          wv, ld, cl, cf, pt);
                        done_hub = true;
                    }
                }
            }
            if (!done_hub)
                k_cf_apply_gen<View, C><<<dim3(grid, na), 256, 0, s>>>(view, vk, vkm1, wv, nlen[0], ld, cl, cf, pt);
        }
        {
            ProfScope ps("cf_reduce", s, 0, 0);
            k_cf_reduce_a<<<na, 256, 0, s>>>(pt, rows ? nblkA : grid, cl, a.p, nv, kk, cf);
        }
        {
            ProfScope ps("cf_orth", s, 3.0 * grp_elems[g] * sizeof(C), 8.0 * grp_elems[g]);
            k_cf_orth<C><<<dim3(grid, na), 256, 0, s>>>(vk, wv, ld, cl, clen_d.p, cf, pt);
        }
        {
            ProfScope ps("cf_reduce", s, 0, 0);
            k_cf_reduce_b<<<na, 256, 0, s>>>(pt, grid, cl, b.p, nv, kk, cf);
        }
        out.launches += 4;
        out.matvecs += na;
    };
    int k = 0;
    while (nact > 0 && k < maxdepth) {
        for (int g = 0; g < ngrp; ++g) level(g, k);
        MSB_LAUNCH_CHECK();
        // (V_{k-1}, V_k, W) <- (V_k, W, V_{k-1})
        C* t = vkm1;
        vkm1 = vk;
        vk = wv;
        wv = t;
        ++k;
        if (k % check == 0 || k == maxdepth) {
            if (ngrp == 2) {                        // the groups meet: st waits for the second stream
                MSB_CUDA(cudaEventRecord(gev, gs[1]));
                MSB_CUDA(cudaStreamWaitEvent(st, gev, 0));
            }
            for (int i = 0; i < nact; ++i) hdepth[hcols[i]] = k;
            cols.upload(hcols.data(), std::max(nact, 1), st);
            {
                ProfScope ps("cf_eval", st, 0, 40.0 * nact * n_w * double(k - k_eval));
                k_cf_eval<<<nact, 128, 0, st>>>(a.p, b.p, nv, n0.p, cols.p, k_eval, k, E0d.p, wdev.p, n_w, eta,
                                                gst.p, Cst.p, Dst.p, I.p, diff.p);
                k_eval = k;
            }
            ++out.launches;
            MSB_CUDA(cudaMemcpyAsync(hdiff.data(), diff.p, 2 * nv * sizeof(double), cudaMemcpyDeviceToHost, st));
            MSB_CUDA(cudaStreamSynchronize(st));
            int keep = 0;
            for (int i = 0; i < nact; ++i) {
                const int c = hcols[i];
                bool fin = k >= maxdepth;
                if (k > check && hdiff[2 * c] <= cf_tol * hdiff[2 * c + 1]) fin = true;
                if (!fin) hcols[keep++] = c;
            }
            nact = keep;
            split();
            regroup_counts();
        }
    }
    MSB_CUDA(cudaMemcpyAsync(I_out, I.p, size_t(nv) * n_w * sizeof(double),
                             I_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    MSB_CUDA(cudaStreamSynchronize(st));
    out.depth = hdepth;
}

static void cf_check_args(int n_vec, const double* w, int n_w, double eta, int cf_check, int cf_maxdepth,
                          double* I_out) {
    MSB_REQUIRE(w != nullptr && I_out != nullptr, "NULL argument");
    MSB_REQUIRE(n_vec >= 1 && n_vec <= 65535, "n_vec must be in 1..65535");
    MSB_REQUIRE(n_w >= 1, "n_w must be >= 1");
    MSB_REQUIRE(eta > 0, "eta must be > 0");
    MSB_REQUIRE(cf_check >= 1 && cf_maxdepth >= cf_check, "need 1 <= cf_check <= cf_maxdepth");
}

void continued_fraction(msb_op* H, const void* phi, int n_vec, double E0, const double* w, int n_w, double eta,
                        double cf_tol, int cf_check, int cf_maxdepth, msb_precision prec, double* I_out,
                        CFResult& out, cudaStream_t st, bool I_dev) {
    MSB_REQUIRE(H != nullptr && phi != nullptr, "NULL argument");
    cf_check_args(n_vec, w, n_w, eta, cf_check, cf_maxdepth, I_out);
    MSB_REQUIRE(H->kind != 2, "the continued fraction of a direct sum mixes its parts: use one part per column");
    MSB_REQUIRE(!op_has_flux(H), "the continued fraction takes a real symmetric H (no flux)");
    CFColumns P;
    P.phi = phi;
    P.ldphi = H->dim;
    P.nv = n_vec;
    P.ops = {H};
    P.q.assign(n_vec, 0);
    P.E0.assign(n_vec, E0);
    if (prec == MSB_FP64) {
        if (H->kind == 0) cf_impl<HubView, double2>(P, H->hub, w, n_w, eta, cf_tol, cf_check, cf_maxdepth, I_out, out, st, I_dev);
        else cf_impl<CsrView, double2>(P, H->csr, w, n_w, eta, cf_tol, cf_check, cf_maxdepth, I_out, out, st, I_dev);
    } else {
        if (H->kind == 0) cf_impl<HubView, float2>(P, H->hub, w, n_w, eta, cf_tol, cf_check, cf_maxdepth, I_out, out, st, I_dev);
        else cf_impl<CsrView, float2>(P, H->csr, w, n_w, eta, cf_tol, cf_check, cf_maxdepth, I_out, out, st, I_dev);
    }
    prof_collect();
}

void continued_fraction_columns(const CFColumns& P, const double* w, int n_w, double eta, double cf_tol,
                                int cf_check, int cf_maxdepth, msb_precision prec, double* I_out, CFResult& out,
                                cudaStream_t st) {
    MSB_REQUIRE(P.phi != nullptr && !P.ops.empty() && int(P.q.size()) == P.nv && int(P.E0.size()) == P.nv,
                "inconsistent column description");
    cf_check_args(P.nv, w, n_w, eta, cf_check, cf_maxdepth, I_out);
    for (const msb_op* o : P.ops) MSB_REQUIRE(o != nullptr && o->kind == 0, "cluster columns need Hubbard operators");
    for (int c = 0; c < P.nv; ++c) MSB_REQUIRE(P.q[c] >= 0 && P.q[c] < int(P.ops.size()), "column cluster out of range");
    if (prec == MSB_FP64)
        cf_impl<HubView, double2>(P, P.ops[0]->hub, w, n_w, eta, cf_tol, cf_check, cf_maxdepth, I_out, out, st, false);
    else
        cf_impl<HubView, float2>(P, P.ops[0]->hub, w, n_w, eta, cf_tol, cf_check, cf_maxdepth, I_out, out, st, false);
    prof_collect();
}

}  // namespace msb

extern "C" msb_status msb_ground_state(msb_op* H, double tol, int maxit, const double* start, double* E_G,
                                       double* g, double* residual, void* stream) {
    msb_status result = MSB_OK;
    msb_status s = msb::guard("msb_ground_state", [&] {
        msb::require_device();
        msb::GroundResult r;
        msb::StreamScope scope((cudaStream_t)stream);
        msb::ground_state(H, tol, maxit, start, g, r, scope.s);
        scope.finish();
        if (E_G) *E_G = r.E;
        if (residual) *residual = r.residual;
        result = r.status;
        if (result != MSB_OK) msb::set_error_message("msb_ground_state: tolerance not reached");
    });
    return s != MSB_OK ? s : result;
}

extern "C" msb_status msb_continued_fraction(msb_op* H, const void* phi, int n_vec, double E0, const double* w,
                                             int n_w, double eta, double cf_tol, int cf_check, int cf_maxdepth,
                                             msb_precision prec, double* I_out, int* depth, void* stream) {
    return msb::guard("msb_continued_fraction", [&] {
        msb::require_device();
        MSB_REQUIRE(prec == MSB_FP64 || prec == MSB_FP32_MIXED, "unknown precision");
        msb::CFResult r;
        msb::StreamScope scope((cudaStream_t)stream);
        msb::continued_fraction(H, phi, n_vec, E0, w, n_w, eta, cf_tol, cf_check, cf_maxdepth, prec, I_out, r,
                                scope.s);
        scope.finish();
        if (depth) for (int c = 0; c < n_vec; ++c) depth[c] = r.depth[c];
    });
}

// ---------------------------------------------------------------------------
// Ground state without any device allocation.
//
// Some callers cannot call cudaMalloc: a host process whose device memory is
// owned by another allocator under a fixed budget (a framework's caching pool,
// a serving process that reserved all memory at start-up), where an extra
// allocation fails or fragments that budget.  For them,
// msb_ground_state_noalloc runs the same Lanczos run as msb_ground_state
// (lanczos_ground above) on a fixed scratch array that lives in the library
// image: every GPU that loads the library holds it until the process exits.
// Its device address is looked up at the start of every call, with the
// caller's current device, so it stays valid after a cudaDeviceReset.  All
// calls share the array and it keeps the previous call's contents; every part
// the Lanczos run reads is written first in the call.  Calls that overlap on
// the GPU (two streams, or two threads) race on the array.
// ---------------------------------------------------------------------------
namespace msb {

constexpr int64_t kNoAllocMaxDim = int64_t(1) << 20;   // dimension limit of the operator
constexpr int kNoAllocMaxIt = 1024;                     // Lanczos steps per restart
constexpr int kNoAllocMaxGrid = 4096;                   // blocks of the vector kernels
constexpr int64_t kNoAllocDoubles =
    5 * kNoAllocMaxDim + 2 * int64_t(kNoAllocMaxIt + 1) + 3 * int64_t(kNoAllocMaxGrid) + 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

static double* noalloc_scratch_address() {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(MSB_ECUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch: ") + cudaGetErrorString(e));
    }
    return static_cast<double*>(p);
}

template <class View>
static void ground_state_noalloc_impl(const msb_op* op, const View& view, int64_t n, double tol, int maxit,
                                      const double* start, double* g, GroundResult& out, cudaStream_t st) {
    const int grid = grid_for(n, 256, 8);
    MSB_REQUIRE(grid <= kNoAllocMaxGrid, "grid exceeds the no-alloc scratch layout");
    double* base = noalloc_scratch_address();
    GroundScratch S;
    S.Q = base;                               // 3 Lanczos vectors
    S.v0 = base + 3 * n;                      // start vector of the current restart
    S.hbuf = base + 4 * n;                    // H g for the residual check
    S.a = base + 5 * n;                       // a_k
    S.b = S.a + (maxit + 1);                  // b_{k+1}
    S.bcur = S.b + (maxit + 1);
    S.n0 = S.bcur + 1;
    S.col0 = reinterpret_cast<int*>(S.n0 + 1);
    S.part = S.n0 + 2;                        // partial sums, 3 per block
    lanczos_ground(op, view, n, tol, maxit, start, g, S, grid, out, st);
}

}  // namespace msb

extern "C" msb_status msb_ground_state_noalloc(msb_op* H, double tol, int maxit, const double* start,
                                               double* E_G, double* g, double* residual, void* stream) {
    msb_status result = MSB_OK;
    msb_status s = msb::guard("msb_ground_state_noalloc", [&] {
        msb::require_device();
        MSB_REQUIRE(H != nullptr && g != nullptr, "NULL argument");
        MSB_REQUIRE(tol > 0, "tol must be > 0");
        MSB_REQUIRE(maxit >= 2 && maxit <= msb::kNoAllocMaxIt,
                    "maxit must be in 2.." + std::to_string(msb::kNoAllocMaxIt) + " for the no-alloc ground state");
        MSB_REQUIRE(H->dim <= msb::kNoAllocMaxDim,
                    "operator dimension " + std::to_string(H->dim) + " exceeds the no-alloc scratch limit of " +
                        std::to_string(msb::kNoAllocMaxDim));
        int dev = 0;
        MSB_CUDA(cudaGetDevice(&dev));
        MSB_REQUIRE(dev == H->device, "the operator was created on another device");
        MSB_REQUIRE(H->kind != 2, "a direct sum has no single ground state: take each part's");
        MSB_REQUIRE(!msb::op_has_flux(H), "the ground state takes a real symmetric H (no flux)");
        cudaStream_t st = (cudaStream_t)stream;
        msb::GroundResult r;
        if (H->kind == 0) msb::ground_state_noalloc_impl(H, H->hub, H->dim, tol, maxit, start, g, r, st);
        else msb::ground_state_noalloc_impl(H, H->csr, H->dim, tol, maxit, start, g, r, st);
        MSB_CUDA(cudaStreamSynchronize(st));
        if (E_G) *E_G = r.E;
        if (residual) *residual = r.residual;
        result = r.status;
        if (result != MSB_OK) msb::set_error_message("msb_ground_state_noalloc: tolerance not reached");
    });
    return s != MSB_OK ? s : result;
}
